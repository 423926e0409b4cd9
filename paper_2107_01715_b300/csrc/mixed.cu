// mixed.cu -- batched form: many roots of mixed depth and action count.
#include "search.cuh"

namespace bcts {
int Ctx::run_mixed(const bcts_state *, const bcts_state *, const int32_t *, const int32_t *, int, int32_t *,
                   float *) {
  return fail(BCTS_ENOKERNEL, "not built yet");
}
}  // namespace bcts

extern "C" int bcts_search_mixed(bcts_ctx *, const bcts_state *, const int32_t *, const int32_t *, int, int32_t *,
                                 float *) {
  return BCTS_ENOKERNEL;
}
