// Reduction variants whose parameters come from the rule-driven enumeration
// (arXiv 1502.02389, Sec. 7 "Towards Automatic Derivation"): each line of
// derived_variants.inc is a parameter set that a derivation of the op's
// Fig. 5 program by the rules of Fig. 3 and Fig. 4 reaches and that the
// hand-picked list in reduce_f32.cu does not instantiate.  The file is
// written by `python -m paper_1502_02389_gb300.derive --emit`.
#include "reduce_f32.cuh"

namespace lift {

void register_reduce_derived(std::vector<Variant>& asum, std::vector<Variant>& dot) {
  const size_t a0 = asum.size(), d0 = dot.size();
#define LIFT_DERIVED(OPNAME, THREADS, TILE, VW, STRIDE, STAGES, NAME)                          \
  (OPNAME == 0 ? asum : dot)                                                                   \
      .push_back(make_variant<OPNAME == 0 ? LIFT_OP_ASUM : LIFT_OP_DOT, THREADS, TILE, VW,      \
                              STRIDE, STAGES, 1, 1>(NAME));
#include "derived_variants.inc"
#undef LIFT_DERIVED
  for (size_t i = a0; i < asum.size(); ++i) {
    asum[i].info.id = static_cast<int>(i);
    asum[i].fallback = 0;  // t1024_v1_ldg_p1: 4-byte loads only
  }
  for (size_t i = d0; i < dot.size(); ++i) {
    dot[i].info.id = static_cast<int>(i);
    dot[i].fallback = 0;
  }
}

}  // namespace lift
