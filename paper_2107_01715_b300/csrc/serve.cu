// serve.cu -- continuous-batching serving form (bcts_submit / bcts_poll).
#include "search.cuh"

namespace bcts {
void serve_shutdown(Ctx *) {}
}  // namespace bcts

extern "C" int bcts_submit(bcts_ctx *, const bcts_state *, int, int, uint64_t *) { return BCTS_ENOKERNEL; }
extern "C" int bcts_poll(bcts_ctx *, uint64_t, int32_t *, float *, int) { return BCTS_ENOKERNEL; }
