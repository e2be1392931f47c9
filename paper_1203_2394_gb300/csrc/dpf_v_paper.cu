// Compiled variants: the paper's models 1 and 2 (Table 1), FP32.
#include "dpf_nl.cuh"

namespace dpf {
Variant make_v_paper1() { return PaperVariant<PaperModel1>::make(); }
Variant make_v_paper2() { return PaperVariant<PaperModel2>::make(); }
Variant make_v_paper1s() { return PaperVariant<PaperModel1Swap>::make(); }
}  // namespace dpf
