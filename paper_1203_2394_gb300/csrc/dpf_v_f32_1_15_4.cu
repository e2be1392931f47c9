// Compiled variant: precision float, d1 = 1, d2 = 15, dy = 4 (the general kernels only).
#include "dpf_variant.cuh"

namespace dpf {
Variant make_v_f32_1_15_4() { return VariantImpl<float, 1, 15, 4, 1>::make(DPF_F32); }
}  // namespace dpf
