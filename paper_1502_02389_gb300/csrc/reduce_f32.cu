// fp32 reduction variants: the hand-picked variant space of the templates in
// reduce_f32.cuh (arXiv 1502.02389, Fig. 5, Fig. 8 eq. (8), Fig. 9a).
#include "reduce_f32.cuh"

namespace lift {
namespace {

// The variant space (the sweep of split tile x asVector width x passes,
// plus staging, tree and reorder alternatives).  Order is the variant id.
#define LIFT_REDUCE_VARIANTS(OP, L)                                     \
  L.push_back(make_variant<OP, 256, 1024, 1, true, 0, 1, 1>("t1024_v1_ldg_p1"));  \
  L.push_back(make_variant<OP, 256, 256, 1, true, 0, 1, 1>("t256_v1_ldg_p1"));    \
  L.push_back(make_variant<OP, 256, 256, 1, true, 0, 1, 2>("t256_v1_ldg_p2"));    \
  L.push_back(make_variant<OP, 256, 512, 1, true, 0, 1, 1>("t512_v1_ldg_p1"));    \
  L.push_back(make_variant<OP, 256, 512, 1, true, 0, 1, 2>("t512_v1_ldg_p2"));    \
  L.push_back(make_variant<OP, 256, 1024, 1, true, 0, 1, 2>("t1024_v1_ldg_p2"));  \
  L.push_back(make_variant<OP, 256, 2048, 1, true, 0, 1, 1>("t2048_v1_ldg_p1"));  \
  L.push_back(make_variant<OP, 256, 2048, 1, true, 0, 1, 2>("t2048_v1_ldg_p2"));  \
  L.push_back(make_variant<OP, 256, 4096, 1, true, 0, 1, 1>("t4096_v1_ldg_p1"));  \
  L.push_back(make_variant<OP, 256, 4096, 1, true, 0, 1, 2>("t4096_v1_ldg_p2"));  \
  L.push_back(make_variant<OP, 256, 1024, 4, true, 0, 1, 1>("t1024_v4_ldg_p1"));  \
  L.push_back(make_variant<OP, 256, 1024, 4, true, 0, 1, 2>("t1024_v4_ldg_p2"));  \
  L.push_back(make_variant<OP, 256, 2048, 4, true, 0, 1, 1>("t2048_v4_ldg_p1"));  \
  L.push_back(make_variant<OP, 256, 2048, 4, true, 0, 1, 2>("t2048_v4_ldg_p2"));  \
  L.push_back(make_variant<OP, 256, 4096, 4, true, 0, 1, 1>("t4096_v4_ldg_p1"));  \
  L.push_back(make_variant<OP, 256, 4096, 4, true, 0, 1, 2>("t4096_v4_ldg_p2"));  \
  L.push_back(make_variant<OP, 256, 2048, 8, true, 0, 1, 1>("t2048_v8_ldg_p1"));  \
  L.push_back(make_variant<OP, 256, 2048, 8, true, 0, 1, 2>("t2048_v8_ldg_p2"));  \
  L.push_back(make_variant<OP, 256, 4096, 8, true, 0, 1, 1>("t4096_v8_ldg_p1"));  \
  L.push_back(make_variant<OP, 256, 4096, 8, true, 0, 1, 2>("t4096_v8_ldg_p2"));  \
  L.push_back(make_variant<OP, 256, 1024, 4, true, 4, 1, 1>("t1024_v4_tma4_p1")); \
  L.push_back(make_variant<OP, 256, 1024, 4, true, 4, 1, 2>("t1024_v4_tma4_p2")); \
  L.push_back(make_variant<OP, 256, 2048, 4, true, 4, 1, 1>("t2048_v4_tma4_p1")); \
  L.push_back(make_variant<OP, 256, 2048, 4, true, 4, 1, 2>("t2048_v4_tma4_p2")); \
  L.push_back(make_variant<OP, 256, 4096, 4, true, 4, 1, 1>("t4096_v4_tma4_p1")); \
  L.push_back(make_variant<OP, 256, 4096, 4, true, 4, 1, 2>("t4096_v4_tma4_p2")); \
  L.push_back(make_variant<OP, 256, 2048, 4, true, 2, 1, 1>("t2048_v4_tma2_p1")); \
  L.push_back(make_variant<OP, 256, 2048, 4, true, 6, 1, 1>("t2048_v4_tma6_p1")); \
  L.push_back(make_variant<OP, 256, 4096, 4, true, 2, 1, 1>("t4096_v4_tma2_p1")); \
  L.push_back(make_variant<OP, 32, 256, 8, true, 0, 1, 1>("w32_t256_v8_ldg_p1"));  \
  L.push_back(make_variant<OP, 32, 512, 8, true, 0, 1, 1>("w32_t512_v8_ldg_p1"));  \
  L.push_back(make_variant<OP, 32, 1024, 8, true, 0, 1, 1>("w32_t1024_v8_ldg_p1")); \
  L.push_back(make_variant<OP, 32, 256, 4, true, 0, 1, 1>("w32_t256_v4_ldg_p1"));  \
  L.push_back(make_variant<OP, 32, 512, 4, true, 0, 1, 1>("w32_t512_v4_ldg_p1"));  \
  L.push_back(make_variant<OP, 256, 2048, 4, true, 0, 4, 1>("c4_t2048_v4_ldg_p1")); \
  L.push_back(make_variant<OP, 256, 4096, 4, true, 0, 4, 1>("c4_t4096_v4_ldg_p1")); \
  L.push_back(make_variant<OP, 256, 4096, 8, true, 0, 4, 1>("c4_t4096_v8_ldg_p1")); \
  L.push_back(make_variant<OP, 256, 4096, 4, true, 0, 2, 1>("c2_t4096_v4_ldg_p1")); \
  L.push_back(make_variant<OP, 256, 4096, 4, true, 0, 8, 1>("c8_t4096_v4_ldg_p1")); \
  L.push_back(make_variant<OP, 256, 1024, 4, false, 0, 1, 1>("chunk_t1024_v4_ldg_p1")); \
  L.push_back(make_variant<OP, 256, 4096, 4, false, 0, 1, 1>("chunk_t4096_v4_ldg_p1")); \
  L.push_back(make_variant<OP, 256, 4096, 1, false, 0, 1, 1>("chunk_t4096_v1_ldg_p1")); \
  L.push_back(make_variant<OP, 256, 4096, 4, false, 4, 1, 1>("chunk_t4096_v4_tma4_p1"));

// nrm2 and sum: the same templates with other user functions; a compact
// set of the variants that lead the asum / dot sweeps.
#define LIFT_REDUCE_VARIANTS_SHORT(OP, L)                                   \
  L.push_back(make_variant<OP, 256, 1024, 1, true, 0, 1, 1>("t1024_v1_ldg_p1"));  \
  L.push_back(make_variant<OP, 256, 4096, 4, true, 0, 1, 1>("t4096_v4_ldg_p1"));  \
  L.push_back(make_variant<OP, 256, 4096, 4, true, 0, 1, 2>("t4096_v4_ldg_p2"));  \
  L.push_back(make_variant<OP, 256, 2048, 8, true, 0, 1, 1>("t2048_v8_ldg_p1"));  \
  L.push_back(make_variant<OP, 256, 4096, 4, true, 4, 1, 1>("t4096_v4_tma4_p1")); \
  L.push_back(make_variant<OP, 256, 4096, 4, true, 0, 2, 1>("c2_t4096_v4_ldg_p1")); \
  L.push_back(make_variant<OP, 32, 1024, 8, true, 0, 1, 1>("w32_t1024_v8_ldg_p1"));

}  // namespace

void register_reduce_f32(std::vector<Variant>& asum, std::vector<Variant>& dot,
                         std::vector<Variant>& nrm2, std::vector<Variant>& sum) {
  LIFT_REDUCE_VARIANTS(LIFT_OP_ASUM, asum)
  LIFT_REDUCE_VARIANTS(LIFT_OP_DOT, dot)
  LIFT_REDUCE_VARIANTS_SHORT(LIFT_OP_NRM2, nrm2)
  LIFT_REDUCE_VARIANTS_SHORT(LIFT_OP_SUM, sum)
  for (auto* L : {&asum, &dot, &nrm2, &sum})
    for (size_t i = 0; i < L->size(); ++i) {
      (*L)[i].info.id = static_cast<int>(i);
      (*L)[i].fallback = 0;  // t1024_v1_ldg_p1: 4-byte loads only
    }
}

}  // namespace lift
