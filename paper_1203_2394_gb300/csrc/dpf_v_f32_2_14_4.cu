// Compiled variant: precision float, d1 = 2, d2 = 14, dy = 4 (the general kernels only).
#include "dpf_variant.cuh"

namespace dpf {
Variant make_v_f32_2_14_4() { return VariantImpl<float, 2, 14, 4, 1>::make(DPF_F32); }
}  // namespace dpf
