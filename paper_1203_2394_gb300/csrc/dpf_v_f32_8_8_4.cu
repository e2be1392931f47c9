// Compiled variant: precision float, d1 = 8, d2 = 8, dy = 4 (the general kernels only).
#include "dpf_variant.cuh"

namespace dpf {
Variant make_v_f32_8_8_4() { return VariantImpl<float, 8, 8, 4, 1>::make(DPF_F32); }
}  // namespace dpf
