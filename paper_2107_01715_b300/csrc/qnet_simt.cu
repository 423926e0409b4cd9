// qnet_simt.cu -- plain FP32 Nature-DQN on CUDA cores: the unoptimised baseline
// the tensor-core paths are measured against (and the reference for "plain FP32"
// one-root-per-launch search).
//
// Each layer is one register-blocked implicit GEMM  out[M][N] = relu(A[M][K] W[N][K]^T + b)
// whose A operand is gathered on the fly from the previous activation map
// (no im2col buffer): M = nodes * output pixels, K = Cin * kh * kw.  Activations
// are stored NHWC, so a GEMM row-major output is already the next layer's input.
// FC2 and the max over actions (Alg. 1's leaf term max_a Q) run in one warp per node.
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace bcts {
namespace {

struct GeoConv1 {  // frames uint8 [n][4][84][84] -> [n][400][32]
  using In = uint8_t;
  static constexpr int K = kK1, N = kC1, MPL = kP1;
  __device__ static __forceinline__ float load(const In *in, int m, int k) {
    const int leaf = m / MPL, p = m - leaf * MPL;
    const int oy = p / 20, ox = p - oy * 20;
    const int c = k >> 6, ky = (k >> 3) & 7, kx = k & 7;
    return float(__ldg(in + size_t(leaf) * kFrameBytes + c * 7056 + (oy * 4 + ky) * 84 + ox * 4 + kx));
  }
};
struct GeoConv2 {  // [n][20][20][32] -> [n][81][64]
  using In = float;
  static constexpr int K = kK2, N = kC2, MPL = kP2;
  __device__ static __forceinline__ float load(const In *in, int m, int k) {
    const int leaf = m / MPL, p = m - leaf * MPL;
    const int oy = p / 9, ox = p - oy * 9;
    const int kk = k >> 5, c = k & 31, ky = kk >> 2, kx = kk & 3;
    return __ldg(in + size_t(leaf) * (kP1 * kC1) + ((oy * 2 + ky) * 20 + ox * 2 + kx) * kC1 + c);
  }
};
struct GeoConv3 {  // [n][9][9][64] -> [n][49][64]
  using In = float;
  static constexpr int K = kK3, N = kC3, MPL = kP3;
  __device__ static __forceinline__ float load(const In *in, int m, int k) {
    const int leaf = m / MPL, p = m - leaf * MPL;
    const int oy = p / 7, ox = p - oy * 7;
    const int kk = k >> 6, c = k & 63, ky = kk / 3, kx = kk - ky * 3;
    return __ldg(in + size_t(leaf) * (kP2 * kC2) + ((oy + ky) * 9 + ox + kx) * kC2 + c);
  }
};
struct GeoFc1 {  // [n][3136] -> [n][512]
  using In = float;
  static constexpr int K = kKF, N = kF1, MPL = 1;
  __device__ static __forceinline__ float load(const In *in, int m, int k) {
    return __ldg(in + size_t(m) * kKF + k);
  }
};

// Block tile BM x BN, K step BK; each thread owns TM x TN outputs.
template <class Geo, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    simt_gemm(const typename Geo::In *__restrict__ in, const float *__restrict__ W,
              const float *__restrict__ bias, float *__restrict__ out, int M) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int K = Geo::K, N = Geo::N;
  static_assert(K % BK == 0 && N % BN == 0, "tile");
  static_assert((BM * BK) % NT == 0 && (BN * BK) % NT == 0, "loads");
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  constexpr int AL = BM * BK / NT, BL = BN * BK / NT;
  float ra[AL], rb[BL];
  auto load_tiles = [&](int k0) {
#pragma unroll
    for (int i = 0; i < AL; ++i) {
      const int e = tid + i * NT, ki = e % BK, mi = e / BK;
      const int m = m0 + mi;
      ra[i] = (m < M) ? Geo::load(in, m, k0 + ki) : 0.f;
    }
#pragma unroll
    for (int i = 0; i < BL; ++i) {
      const int e = tid + i * NT, ki = e % BK, ni = e / BK;
      rb[i] = __ldg(W + size_t(n0 + ni) * K + k0 + ki);
    }
  };
  load_tiles(0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < AL; ++i) {
      const int e = tid + i * NT;
      As[e % BK][e / BK] = ra[i];
    }
#pragma unroll
    for (int i = 0; i < BL; ++i) {
      const int e = tid + i * NT;
      Bs[e % BK][e / BK] = rb[i];
    }
    __syncthreads();
    if (k0 + BK < K) load_tiles(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty * TM + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx * TN + j;
      const float v = acc[i][j] + __ldg(bias + n);
      out[size_t(m) * N + n] = v > 0.f ? v : 0.f;
    }
  }
}

// FC2 + max over actions: q = W2 h + b2, maxq = max_a q[a].  A persistent grid:
// each block stages W2 (A x 512, at most 36 KB) in shared memory once, with all
// of a thread's loads in flight together (a loop that waits for each load before
// its store costs an L2 round trip per element, tens of microseconds per launch),
// and its warps then take two nodes at a time, so each W2 value read from shared
// memory serves both.  Lane l holds h[4 l + 128 j .. + 3] of each node; its 16
// products per action are summed across the warp by a reduce-scatter butterfly
// (31 shuffles for all actions at once), after which lane a holds q[a].
__global__ void __launch_bounds__(256, 2) fc2_max_kernel(const float *__restrict__ h, const float *__restrict__ W2,
                                                      const float *__restrict__ b2, int A, int64_t n,
                                                      float *__restrict__ q, float *__restrict__ maxq,
                                                      const uint8_t *__restrict__ node_A) {
  __shared__ __align__(16) float w[kMaxA * kF1];
  if ((reinterpret_cast<uintptr_t>(W2) & 15u) == 0) {
    constexpr int NV = kMaxA * kF1 / 4, PER = (NV + 255) / 256;
    float4 v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = threadIdx.x + k * 256;
      v[k] = i < A * (kF1 / 4) ? __ldg(reinterpret_cast<const float4 *>(W2) + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = threadIdx.x + k * 256;
      if (i < NV) reinterpret_cast<float4 *>(w)[i] = v[k];
    }
  } else {
#pragma unroll 12
    for (int i = threadIdx.x; i < A * kF1; i += blockDim.x) w[i] = __ldg(W2 + i);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const float bias = lane < A ? __ldg(b2 + lane) : 0.f;
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x / 32);
  // two nodes per warp pass: each W2 value read from shared memory serves both.
  // The next pass's rows are loaded while this pass computes (measured 0.169 ->
  // 0.159 ms per Atari-scale search; the rest is W2's shared-memory reads and
  // the FMAs)
  float4 xn[2][4];
  auto load_pair = [&](int64_t g2) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t nd = 2 * g2 + u < n ? 2 * g2 + u : n - 1;
      const float4 *hv = reinterpret_cast<const float4 *>(h + nd * kF1);
#pragma unroll
      for (int j = 0; j < 4; ++j) xn[u][j] = __ldg(hv + lane + 32 * j);
    }
  };
  int64_t g = int64_t(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (2 * g < n) load_pair(g);
  for (; 2 * g < n; g += nwarps) {
    const int64_t node0 = 2 * g;
    float x[2][16];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x[u][4 * j] = xn[u][j].x;
        x[u][4 * j + 1] = xn[u][j].y;
        x[u][4 * j + 2] = xn[u][j].z;
        x[u][4 * j + 3] = xn[u][j].w;
      }
    if (2 * (g + nwarps) < n) load_pair(g + nwarps);
    float v[2][32];
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      float s0 = 0.f, s1 = 0.f;
      if (a < kMaxA && a < A) {
        const float4 *wa = reinterpret_cast<const float4 *>(w + a * kF1);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 c = wa[lane + 32 * j];
          s0 = fmaf(x[0][4 * j], c.x, s0);
          s0 = fmaf(x[0][4 * j + 1], c.y, s0);
          s0 = fmaf(x[0][4 * j + 2], c.z, s0);
          s0 = fmaf(x[0][4 * j + 3], c.w, s0);
          s1 = fmaf(x[1][4 * j], c.x, s1);
          s1 = fmaf(x[1][4 * j + 1], c.y, s1);
          s1 = fmaf(x[1][4 * j + 2], c.z, s1);
          s1 = fmaf(x[1][4 * j + 3], c.w, s1);
        }
      }
      v[0][a] = s0;
      v[1][a] = s1;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      // reduce-scatter: at offset o a lane keeps the half of its remaining actions
      // selected by its bit o and receives its partner's partial sums for them
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
          const float send = up ? v[u][i] : v[u][i + o];
          const float keep = up ? v[u][i + o] : v[u][i];
          v[u][i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      const int64_t node = node0 + u;
      if (node >= n) break;
      const float s = v[u][0] + bias;  // q[node][lane] for lane < A
      if (q && lane < A) q[node * A + lane] = s;
      // node_A (batched form): the max runs over this node's own first node_A actions
      const int An = node_A ? int(node_A[node]) : A;
      float best = lane < An ? s : -INFINITY;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
      if (maxq && lane == 0) maxq[node] = best;
    }
  }
}

template <class Geo, int BM, int BN, int TM, int TN>
int run_gemm(int kind, const typename Geo::In *in, const float *W, const float *b, float *out, int64_t nodes,
             cudaStream_t st) {
  const int64_t M = nodes * Geo::MPL;
  if (M > 0x7FFFFFFFLL) return BCTS_EINVAL;
  dim3 grid(unsigned((M + BM - 1) / BM), Geo::N / BN);
  ProfScope ps(kind, st);
  simt_gemm<Geo, BM, BN, 16, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(in, W, b, out, int(M));
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

}  // namespace

// Load every kernel simt_qnet_forward launches on the current device.  The CUDA
// runtime loads device code lazily, on a kernel's first launch, unless
// CUDA_MODULE_LOADING=EAGER; querying a kernel's attributes loads it now.
int simt_preload() {
  cudaFuncAttributes fa;
  const void *fns[] = {reinterpret_cast<const void *>(simt_gemm<GeoConv1, 128, 32, 16, 8, 2>),
                       reinterpret_cast<const void *>(simt_gemm<GeoConv2, 128, 64, 16, 8, 4>),
                       reinterpret_cast<const void *>(simt_gemm<GeoConv3, 128, 64, 16, 8, 4>),
                       reinterpret_cast<const void *>(simt_gemm<GeoFc1, 128, 64, 16, 8, 4>),
                       reinterpret_cast<const void *>(fc2_max_kernel)};
  for (const void *f : fns)
    if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) {
      cudaGetLastError();
      return BCTS_ECUDA;
    }
  return BCTS_OK;
}

size_t simt_scratch_bytes(int64_t chunk) {
  return size_t(chunk) * sizeof(float) * (kP1 * kC1 + kP2 * kC2 + kP3 * kC3 + kF1) + 4096;
}

int simt_qnet_forward(const SimtWeights &w, const uint8_t *frames, int64_t n, float *q, float *maxq,
                      void *scratch, cudaStream_t st, const uint8_t *node_A) {
  if (n <= 0) return BCTS_OK;
  float *a1 = static_cast<float *>(scratch);
  float *a2 = a1 + size_t(n) * kP1 * kC1;
  float *a3 = a2 + size_t(n) * kP2 * kC2;
  float *a4 = a3 + size_t(n) * kP3 * kC3;
  int rc;
  if ((rc = run_gemm<GeoConv1, 128, 32, 8, 2>(K_CONV1, frames, w.c1w, w.c1b, a1, n, st)) != BCTS_OK) return rc;
  if ((rc = run_gemm<GeoConv2, 128, 64, 8, 4>(K_CONV2, a1, w.c2w, w.c2b, a2, n, st)) != BCTS_OK) return rc;
  if ((rc = run_gemm<GeoConv3, 128, 64, 8, 4>(K_CONV3, a2, w.c3w, w.c3b, a3, n, st)) != BCTS_OK) return rc;
  if ((rc = run_gemm<GeoFc1, 128, 64, 8, 4>(K_FC1, a3, w.f1w, w.f1b, a4, n, st)) != BCTS_OK) return rc;
  return launch_fc2_max(a4, w.f2w, w.f2b, w.A, n, q, maxq, st, node_A);
}

int launch_fc2_max(const float *h, const float *W2, const float *b2, int A, int64_t n, float *q, float *maxq,
                   cudaStream_t st, const uint8_t *node_A) {
  if (n <= 0) return BCTS_OK;
  const int warps = 8;
  static int sms = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 148;
  });
  // persistent: two blocks per SM (36 KB of W2 each), never more warps than node pairs
  const int64_t groups = ((n + 1) / 2 + warps - 1) / warps;
  const unsigned grid = unsigned(groups < int64_t(2) * sms ? groups : int64_t(2) * sms);
  ProfScope ps(K_FC2, st);
  fc2_max_kernel<<<grid, warps * 32, 0, st>>>(h, W2, b2, A, n, q, maxq, node_A);
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

}  // namespace bcts
