// qnet_tc.cu -- tensor-core (tcgen05) Q-network paths.
#include "common.cuh"
#include "kernels.cuh"

namespace bcts {

struct TcWeights {
  int A = 0;
  int precision = 0;
};

size_t tc_scratch_bytes(int64_t, int) { return 256; }

int tc_weights_create(const float *, int, int, TcWeights **out, std::string &err) {
  *out = nullptr;
  err = "tensor-core Q-network not built yet";
  return BCTS_ENOKERNEL;
}

void tc_weights_destroy(TcWeights *w) { delete w; }

int tc_qnet_forward(const TcWeights *, int, const uint8_t *, const bcts_state *, int64_t, float *, float *, void *,
                    cudaStream_t, int *) {
  return BCTS_ENOKERNEL;
}

}  // namespace bcts
