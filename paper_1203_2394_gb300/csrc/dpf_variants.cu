// The table of compiled (precision, d1, d2, dy) variants.
#include "dpf_internal.h"

namespace dpf {

Variant make_v_f32_2_8_2();
Variant make_v_f64_2_2_2();
Variant make_v_f32_2_2_2();
Variant make_v_f32_1_15_4();
Variant make_v_f32_2_14_4();
Variant make_v_f32_4_12_4();
Variant make_v_f32_8_8_4();
Variant make_v_f32_8_56_8();
Variant make_v_paper1();
Variant make_v_paper2();
Variant make_v_paper1s();

const Variant* find_variant(int prec, int d1, int d2, int dy) {
  static const Variant table[] = {make_v_f32_2_8_2(), make_v_f64_2_2_2(), make_v_f32_2_2_2(),
                                  make_v_f32_1_15_4(), make_v_f32_2_14_4(), make_v_f32_4_12_4(),
                                  make_v_f32_8_8_4(), make_v_f32_8_56_8()};
  for (const Variant& v : table)
    if (v.prec == prec && v.d1 == d1 && v.d2 == d2 && v.dy == dy) return &v;
  return nullptr;
}

const Variant* find_paper_variant(int kind, bool swapped) {
  static const Variant table[] = {make_v_paper1(), make_v_paper2(), make_v_paper1s()};
  if (kind == DPF_MODEL_PAPER1) return &table[swapped ? 2 : 0];
  if (kind == DPF_MODEL_PAPER2 && !swapped) return &table[1];
  return nullptr;
}

}  // namespace dpf
