// Compiled variant: precision float, d1 = 4, d2 = 12, dy = 4 (the general kernels only).
#include "dpf_variant.cuh"

namespace dpf {
Variant make_v_f32_4_12_4() { return VariantImpl<float, 4, 12, 4, 1>::make(DPF_F32); }
}  // namespace dpf
