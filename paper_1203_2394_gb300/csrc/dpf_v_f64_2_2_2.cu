// Compiled variant: precision double, d1 = 2, d2 = 2, dy = 2.
#include "dpf_variant.cuh"

namespace dpf {
Variant make_v_f64_2_2_2() { return VariantImpl<double, 2, 2, 2>::make(DPF_F64); }
}  // namespace dpf
