// qnet_static.cu -- Q-network evaluation that allocates no memory.
//
// Some callers cannot allocate device memory at all: code running inside a
// custom allocator or a memory-pool callback, an engine that has reserved the
// whole device before it loads this library, or a host that forbids
// cudaMalloc after start-up so its memory use stays fixed.  bcts_qnet_static
// serves them: it runs the same plain FP32 Q-network kernels as a context with
// BCTS_PREC_FP32_SIMT, but takes its scratch (the weights in the kernels'
// layout and the activation maps of up to BCTS_STATIC_MAX_NODES stacks) from
// one file-scope __device__ array instead of cudaMalloc.  The array belongs to
// this file's device code: a GPU holds it (about 18 MB) from the moment that code
// is loaded on it until the process exits.  The CUDA runtime loads device code
// lazily (on first use) unless CUDA_MODULE_LOADING=EAGER, so the first call on
// each device -- n = 0 is enough -- loads the code this entry point runs and looks
// up the array's address; that call is the one that may allocate, and it must come
// before any allocation limit applies and before any stream capture.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace bcts {
namespace {

constexpr int64_t kStaticNodes = BCTS_STATIC_MAX_NODES;
// Weights for the largest action count, rounded up to a 256-byte boundary.
constexpr size_t kWeightFloats = ((size_t(32) * 256 + 32 + 64 * 512 + 64 + 64 * 576 + 64 + size_t(512) * 3136 +
                                   512 + size_t(kMaxA) * 512 + kMaxA) + 63) / 64 * 64;
constexpr size_t kActFloats = size_t(kStaticNodes) * (kP1 * kC1 + kP2 * kC2 + kP3 * kC3 + kF1);

// The scratch every call shares.  Host code must not pass `g_static_scratch`
// itself to a kernel (on the host it names a stand-in, not device memory); it
// uses the address cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) float g_static_scratch[kWeightFloats + kActFloats];

// PyTorch-order weights -> the CUDA-core kernels' layouts (same mapping as the
// context's host-side conversion, 1/255 folded into conv1 in double precision).
__global__ void static_permute_weights(const float *__restrict__ src, int A, float *__restrict__ dst) {
  const int64_t total = int64_t(32) * 256 + 32 + 64 * 512 + 64 + 64 * 576 + 64 + int64_t(512) * 3136 + 512 +
                        int64_t(A) * 512 + A;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    int64_t j = i, base = 0;
    float v;
    if (j < 32 * 256) {  // conv1: same order, scaled
      v = __double2float_rn(double(src[j]) / 255.0);
    } else if ((j -= 32 * 256) < 32) {
      v = src[32 * 256 + j];
    } else if ((j -= 32) < 64 * 512) {  // conv2: k = (ky*4+kx)*32 + c  <-  [o][c][ky][kx]
      base = 32 * 256 + 32;
      const int o = int(j / 512), k = int(j % 512), kk = k >> 5, c = k & 31;
      v = src[base + ((o * 32 + c) * 4 + (kk >> 2)) * 4 + (kk & 3)];
    } else if ((j -= 64 * 512) < 64) {
      v = src[32 * 256 + 32 + 64 * 512 + j];
    } else if ((j -= 64) < 64 * 576) {  // conv3: k = (ky*3+kx)*64 + c  <-  [o][c][ky][kx]
      base = 32 * 256 + 32 + 64 * 512 + 64;
      const int o = int(j / 576), k = int(j % 576), kk = k >> 6, c = k & 63;
      v = src[base + ((o * 64 + c) * 3 + kk / 3) * 3 + kk % 3];
    } else if ((j -= 64 * 576) < 64) {
      v = src[32 * 256 + 32 + 64 * 512 + 64 + 64 * 576 + j];
    } else if ((j -= 64) < int64_t(512) * 3136) {  // fc1: column (y*7+x)*64 + c  <-  c*49 + y*7 + x
      base = 32 * 256 + 32 + 64 * 512 + 64 + 64 * 576 + 64;
      const int64_t o = j / 3136;
      const int k = int(j % 3136), p = k >> 6, c = k & 63;
      v = src[base + o * 3136 + c * 49 + p];
    } else {  // fc1 bias, fc2 weight and bias: same positions in both layouts
      v = src[i];
    }
    dst[i] = v;
  }
}

std::mutex g_setup_mu;
float *g_scratch_ptr[64] = {};

// Set-up, once per device with that device current: load the kernels this entry
// point launches (the permute kernel here, the plain FP32 network's kernels in
// qnet_simt.cu) and look up the scratch's device address.
int static_scratch(float **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return BCTS_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaFuncAttributes fa;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p ||
        cudaFuncGetAttributes(&fa, static_permute_weights) != cudaSuccess || simt_preload() != BCTS_OK) {
      cudaGetLastError();
      return BCTS_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<float *>(p);
  }
  *out = g_scratch_ptr[dev];
  return BCTS_OK;
}

}  // namespace
}  // namespace bcts

extern "C" int bcts_qnet_static(const float *d_qnet_weights, int A, const uint8_t *d_frames, int64_t n, float *d_q,
                                void *stream) {
  using namespace bcts;
  if (!d_qnet_weights || A < 1 || A > kMaxA || n < 0 || (n > 0 && (!d_frames || !d_q))) {
    set_thread_error("bcts_qnet_static: invalid argument");
    return BCTS_EINVAL;
  }
  if (n > kStaticNodes) {
    set_thread_error("bcts_qnet_static: n = " + std::to_string(n) + " exceeds BCTS_STATIC_MAX_NODES = " +
                     std::to_string(kStaticNodes) + " (split the batch)");
    return BCTS_EINVAL;
  }
  float *scratch = nullptr;
  if (static_scratch(&scratch) != BCTS_OK) {
    set_thread_error("bcts_qnet_static: set-up (loading the kernels, cudaGetSymbolAddress of the static scratch) failed");
    return BCTS_ECUDA;
  }
  if (n == 0) return BCTS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  float *w = scratch;
  float *act = scratch + kWeightFloats;
  static_permute_weights<<<296, 256, 0, st>>>(d_qnet_weights, A, w);
  if (cudaGetLastError() != cudaSuccess) {
    set_thread_error("bcts_qnet_static: weight layout launch failed");
    return BCTS_ECUDA;
  }
  SimtWeights sw;
  sw.c1w = w;
  sw.c1b = sw.c1w + 32 * 256;
  sw.c2w = sw.c1b + 32;
  sw.c2b = sw.c2w + 64 * 512;
  sw.c3w = sw.c2b + 64;
  sw.c3b = sw.c3w + 64 * 576;
  sw.f1w = sw.c3b + 64;
  sw.f1b = sw.f1w + size_t(512) * 3136;
  sw.f2w = sw.f1b + 512;
  sw.f2b = sw.f2w + size_t(A) * 512;
  sw.A = A;
  const int rc = simt_qnet_forward(sw, d_frames, n, d_q, nullptr, act, st);
  if (rc != BCTS_OK) set_thread_error("bcts_qnet_static: Q-network launch failed");
  return rc;
}
