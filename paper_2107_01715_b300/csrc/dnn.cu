// dnn.cu -- the DNN forward-model workload: Batch-BFS (Alg. 1) and the BCTS
// correction over a randomly initialised network that stands in for a learned
// forward model (Sec. 4, runtime experiments: three hidden layers of width 100
// on a 100-wide state and a one-hot action).
//
// Model (weights in PyTorch [out][in] order, see include/bcts.h):
//   x = [s; onehot(a)], h_k = ReLU(W_k h_{k-1} + b_k) for k = 1..3,
//   o = W_o h_3 + b_o, s' = tanh(o[0..99]), r = o[100];  Q(s) = W_q s + b_q.
// Layer 1 splits as W_1 x = W_1s s + W_1a[:, a]: the state part is one product
// per parent, shared by its A children, which each add their action's column.
// Every layer is FP32 on CUDA cores: K = N = 100 contractions are too narrow to
// feed the tensor cores at FP32 accuracy, and the forward model is the
// simulator, whose arithmetic the search must not change.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstring>
#include <string>
#include <vector>

#include "search.cuh"

namespace bcts {
namespace {

constexpr int kD = 100;  // state width
constexpr int kH = 100;  // hidden width
constexpr int kMaxDnnA = 32;
constexpr int kMaxDnnDepth = 16;
constexpr int64_t kChunkRows = int64_t(1) << 21;  // children per forward-model pass

// ---------------------------------------------------------------------------
// out[m][n] = act(in[m][0..K) . W[n][0..K) + b[n]), m < M, n < N <= 104,
// K <= kXS and a multiple of 4 (rows of `in` are K floats, 16-byte aligned).
// Persistent blocks: W transposed into shared memory once per block, [k][104];
// then 64-row tiles of `in`, double-buffered with cp.async so the next tile
// lands while this one is multiplied.  208 threads: thread (rg, cg) owns rows
// rg + 8 i (i < 8) and columns 4 cg .. 4 cg + 3 (26 column groups cover the
// 100 / 101 outputs of these layers with 4 % padding); a warp's threads share
// at most two row groups one row apart (different banks) and read each k's
// weights with one 16-byte load: 32 FMAs per three 16-byte shared loads.
// ---------------------------------------------------------------------------
constexpr int kTileRows = 64;
constexpr int kCG = 26;             // column groups of 4
constexpr int kNC = 4 * kCG;        // output columns per tile (N padded to 104)
constexpr int kDenseThreads = 8 * kCG;
constexpr int kXS = 108;  // activation row stride (floats): 16-byte multiple, consecutive rows 12 banks apart

__device__ __forceinline__ void cp_async16_zfill(float *dst, const float *src, bool valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

// What a dense launch reads and writes besides in / W / b / out.
struct DenseIO {
  // IN_H1: input row c is ReLU(P[c / A] + W1a[c % A] + b1) (layer 1 of child c)
  const float *P = nullptr, *w1a = nullptr, *b1 = nullptr;
  int A = 1;
  // EPI_STATE: columns 0..99 -> s_next = tanh, column 100 -> R_child = R_parent[c / A] + gp r
  float *s_next = nullptr, *R_child = nullptr;
  const float *Rp = nullptr;
  float gp = 1.f;
};
enum { IN_ROWS = 0, IN_H1 = 1 };
enum { EPI_LINEAR = 0, EPI_RELU = 1, EPI_STATE = 2 };

template <int IN, int EPI>
__global__ void __launch_bounds__(kDenseThreads) dense_kernel(const float *__restrict__ in, int64_t M, int K,
                                                    const float *__restrict__ W, const float *__restrict__ b, int N,
                                                    float *__restrict__ out, int ldo, const DenseIO io) {
  extern __shared__ __align__(16) float sm[];
  float *Wt = sm;                     // [K][kNC]
  float *Xs = sm + K * kNC;           // [2][kTileRows][kXS]
  const int rg = threadIdx.x / kCG, cg = threadIdx.x - rg * kCG;
  const int64_t ntiles = (M + kTileRows - 1) / kTileRows;
  const int kq = K / 4;  // 16-byte chunks per row
  // rows of a tile: copied with cp.async (IN_ROWS), or formed from the parent's
  // layer-1 product and the action column (IN_H1, synchronous)
  auto issue = [&](int64_t tile, int buf) {
    float *dst = Xs + buf * (kTileRows * kXS);
    const int64_t m0 = tile * kTileRows;
    for (int i = threadIdx.x; i < kTileRows * kq; i += blockDim.x) {
      const int r = i / kq, q = i - r * kq;
      const bool ok = m0 + r < M;
      if (IN == IN_ROWS) {
        cp_async16_zfill(dst + r * kXS + 4 * q, in + (ok ? (m0 + r) * K + 4 * q : 0), ok);
      } else {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ok) {
          const int64_t c = m0 + r, par = c / io.A;
          const int a = int(c - par * io.A);
          const float4 p = *reinterpret_cast<const float4 *>(io.P + par * K + 4 * q);
          const float4 w = *reinterpret_cast<const float4 *>(io.w1a + a * K + 4 * q);
          const float4 bb = *reinterpret_cast<const float4 *>(io.b1 + 4 * q);
          v = make_float4(fmaxf(p.x + w.x + bb.x, 0.f), fmaxf(p.y + w.y + bb.y, 0.f), fmaxf(p.z + w.z + bb.z, 0.f),
                          fmaxf(p.w + w.w + bb.w, 0.f));
        }
        *reinterpret_cast<float4 *>(dst + r * kXS + 4 * q) = v;
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  int64_t tile = blockIdx.x;
  if (tile < ntiles) issue(tile, 0);
  // W, read in its own row order (coalesced), stored transposed; ten loads of a
  // thread in flight at once (one at a time costs an L2 round trip per element)
  for (int i0 = threadIdx.x; i0 < kNC * K; i0 += 10 * blockDim.x) {
    float v[10];
#pragma unroll
    for (int u = 0; u < 10; ++u) {
      const int i = i0 + u * blockDim.x;
      v[u] = (i < kNC * K && i / K < N) ? __ldg(W + i) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 10; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < kNC * K) {
        const int n = i / K, k = i - n * K;
        Wt[k * kNC + n] = v[u];
      }
    }
  }
  float bias[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) bias[c] = (b && 4 * cg + c < N) ? b[4 * cg + c] : 0.f;
  for (int it = 0; tile < ntiles; tile += gridDim.x, ++it) {
    const int64_t next = tile + gridDim.x;
    if (next < ntiles)
      issue(next, (it + 1) & 1);
    else
      asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();  // this tile (and W) visible to every warp
    const float *xs = Xs + (it & 1) * (kTileRows * kXS) + rg * kXS;
    float acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = bias[c];
    for (int k0 = 0; k0 < K; k0 += 4) {
      float4 x[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) x[r] = *reinterpret_cast<const float4 *>(xs + 8 * r * kXS + k0);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float4 w = *reinterpret_cast<const float4 *>(Wt + (k0 + kk) * kNC + 4 * cg);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const float xv = kk == 0 ? x[r].x : (kk == 1 ? x[r].y : (kk == 2 ? x[r].z : x[r].w));
          acc[r][0] = fmaf(xv, w.x, acc[r][0]);
          acc[r][1] = fmaf(xv, w.y, acc[r][1]);
          acc[r][2] = fmaf(xv, w.z, acc[r][2]);
          acc[r][3] = fmaf(xv, w.w, acc[r][3]);
        }
      }
    }
    const int64_t m0 = tile * kTileRows + rg;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int64_t m = m0 + 8 * r;
      if (m >= M) break;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int n = 4 * cg + c;
        if (n >= N) continue;
        if (EPI == EPI_STATE) {
          if (n < kD)
            io.s_next[m * kD + n] = tanhf(acc[r][c]);
          else
            io.R_child[m] = (io.Rp ? io.Rp[m / io.A] : 0.f) + io.gp * acc[r][c];
        } else {
          out[m * ldo + n] = EPI == EPI_RELU ? fmaxf(acc[r][c], 0.f) : acc[r][c];
        }
      }
    }
    __syncthreads();  // every warp is done with this buffer before it is refilled
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Q(s) = W_q s + b_q per node (one warp per node, lane l holds s[l + 32 m]); a
// reduce-scatter butterfly leaves q[a] in lane a; max over the A actions.
__global__ void __launch_bounds__(256) dnn_q_kernel(const float *__restrict__ s, int64_t n, const float *__restrict__ wq,
                                                    const float *__restrict__ bq, int A, float *__restrict__ q,
                                                    float *__restrict__ maxq) {
  __shared__ float w[kMaxDnnA * 128];
#pragma unroll
  for (int i = threadIdx.x; i < kMaxDnnA * 128; i += 256) {  // all of a thread's loads in flight together
    const int a = i >> 7, k = i & 127;
    w[i] = (a < A && k < kD) ? __ldg(wq + a * kD + k) : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const float bias = lane < A ? bq[lane] : 0.f;
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x / 32);
  for (int64_t node = int64_t(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5); node < n; node += nwarps) {
    float x[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int k = lane + 32 * m;
      x[m] = k < kD ? s[node * kD + k] : 0.f;
    }
    float v[32];
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      float acc = 0.f;
      if (a < A) {
#pragma unroll
        for (int m = 0; m < 4; ++m) acc = fmaf(x[m], w[a * 128 + lane + 32 * m], acc);
      }
      v[a] = acc;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < o; ++i) {
        const float send = up ? v[i] : v[i + o];
        const float keep = up ? v[i + o] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    const float qa = v[0] + bias;
    if (q && lane < A) q[node * A + lane] = qa;
    float best = lane < A ? qa : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (maxq && lane == 0) maxq[node] = best;
  }
}

int sm_count() {
  static int sms = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 148;
  });
  return sms;
}


}  // namespace

struct DnnCtx {
  int device = 0, A = 0, d = 0;
  float gamma = 0.99f, corr = 1.f;
  bool exact_gev = false;
  cudaStream_t stream = nullptr;
  std::string err;
  Profiler *prof = nullptr;
  // weights: W1s [H][D], W1a [A][H], b1, W2, b2, W3, b3, Wo [D+1][H], bo, Wq [A][D], bq
  float *wbuf = nullptr;
  const float *w1s, *w1a, *b1, *w2, *b2, *w3, *b3, *wo, *bo, *wq, *bq;
  DevBuf lvl[2], Rl[2], q0, maxq1, r1, V, leafmax, P, hA, hB, io_roots, io_act, io_val;
  void *host = nullptr;
  size_t host_cap = 0;

  int fail(int code, const std::string &msg) {
    err = msg;
    set_thread_error(msg);
    return code;
  }
  int ensure(DevBuf &b, size_t bytes) {
    if (bytes <= b.cap) return BCTS_OK;
    if (b.p) {
      cudaStreamSynchronize(stream);
      cudaFree(b.p);
      b.p = nullptr;
      b.cap = 0;
    }
    const size_t want = (std::max(bytes, b.cap + b.cap / 2) + 255) & ~size_t(255);
    if (cudaMalloc(&b.p, want) != cudaSuccess) {
      cudaGetLastError();
      return fail(BCTS_ENOMEM, "DNN workload: device allocation of " + std::to_string(want) + " bytes failed");
    }
    b.cap = want;
    return BCTS_OK;
  }
  ~DnnCtx() {
    DevBuf *bufs[] = {&lvl[0], &lvl[1], &Rl[0], &Rl[1], &q0,  &maxq1, &r1,      &V,      &leafmax,
                      &P,      &hA,     &hB,     &io_roots, &io_act, &io_val};
    for (DevBuf *b : bufs)
      if (b->p) cudaFree(b->p);
    if (wbuf) cudaFree(wbuf);
    if (host) cudaFreeHost(host);
    if (stream) cudaStreamDestroy(stream);
    if (prof) profiler_destroy(prof);
  }

  template <int IN, int EPI>
  int dense(const float *in, int64_t M, int K, const float *W, const float *b, int N, float *out, int ldo,
            const DenseIO &io, cudaStream_t st) {
    if (M <= 0) return BCTS_OK;
    const size_t smem = size_t(K * kNC + 2 * kTileRows * kXS) * sizeof(float);
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [smem] {
      attr_err = cudaFuncSetAttribute(dense_kernel<IN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    });
    if (attr_err != cudaSuccess) return fail(BCTS_ECUDA, "DNN dense layer: shared-memory attribute refused");
    const int64_t tiles = (M + kTileRows - 1) / kTileRows;
    const unsigned grid = unsigned(tiles < int64_t(2) * sm_count() ? tiles : int64_t(2) * sm_count());
    ProfScope ps(K_DNN_MLP, st);
    dense_kernel<IN, EPI><<<grid, kDenseThreads, smem, st>>>(in, M, K, W, b, N, out, ldo, io);
    return cudaGetLastError() == cudaSuccess ? BCTS_OK : fail(BCTS_ECUDA, "DNN dense layer launch failed");
  }

  int qhead(const float *s, int64_t n, float *q, float *maxq, cudaStream_t st) {
    if (n <= 0) return BCTS_OK;
    const int64_t groups = (n + 7) / 8;
    const unsigned grid = unsigned(groups < int64_t(4) * sm_count() ? groups : int64_t(4) * sm_count());
    ProfScope ps(K_DNN_Q, st);
    dnn_q_kernel<<<grid, 256, 0, st>>>(s, n, wq, bq, A, q, maxq);
    return cudaGetLastError() == cudaSuccess ? BCTS_OK : fail(BCTS_ECUDA, "DNN Q head launch failed");
  }

  // Alg. 1's expansion of np parents: children states and accumulated rewards.
  int expand(const float *parents, const float *Rp, int64_t np, float gp, float *child, float *Rc, cudaStream_t st) {
    const int64_t chunk_p = kChunkRows / A > 0 ? kChunkRows / A : 1;
    int rc;
    const int64_t cp = np < chunk_p ? np : chunk_p, cc = cp * A;
    if ((rc = ensure(P, size_t(cp) * kH * 4)) != BCTS_OK) return rc;
    if ((rc = ensure(hA, size_t(cc) * kH * 4)) != BCTS_OK) return rc;
    if ((rc = ensure(hB, size_t(cc) * kH * 4)) != BCTS_OK) return rc;
    float *Pp = static_cast<float *>(P.p), *ha = static_cast<float *>(hA.p), *hb = static_cast<float *>(hB.p);
    for (int64_t off = 0; off < np; off += chunk_p) {
      const int64_t cnt = np - off < chunk_p ? np - off : chunk_p, nc = cnt * A;
      const DenseIO none;
      if ((rc = dense<IN_ROWS, EPI_LINEAR>(parents + off * kD, cnt, kD, w1s, nullptr, kH, Pp, kH, none, st)) !=
          BCTS_OK)
        return rc;
      DenseIO l2;  // layer 2 reads each child's layer-1 activations straight from P
      l2.P = Pp;
      l2.w1a = w1a;
      l2.b1 = b1;
      l2.A = A;
      if ((rc = dense<IN_H1, EPI_RELU>(nullptr, nc, kH, w2, b2, kH, hb, kH, l2, st)) != BCTS_OK) return rc;
      if ((rc = dense<IN_ROWS, EPI_RELU>(hb, nc, kH, w3, b3, kH, ha, kH, none, st)) != BCTS_OK) return rc;
      DenseIO so;  // the output layer writes the child's state and accumulated reward
      so.s_next = child + off * A * kD;
      so.R_child = Rc + off * A;
      so.Rp = Rp ? Rp + off : nullptr;
      so.gp = gp;
      so.A = A;
      if ((rc = dense<IN_ROWS, EPI_STATE>(ha, nc, kH, wo, bo, kD + 1, nullptr, 0, so, st)) != BCTS_OK) return rc;
    }
    return BCTS_OK;
  }

  int run(const float *d_roots, int n, int32_t *d_action, float *d_values, cudaStream_t st) {
    if (n <= 0) return BCTS_OK;
    ProfilerGuard pg(prof);
    std::vector<int64_t> N(d + 1);
    N[0] = n;
    for (int i = 1; i <= d; ++i) {
      N[i] = N[i - 1] * A;
      if (N[i] > 0x7FFFFFFFLL) return fail(BCTS_EINVAL, "DNN workload: n * A^d exceeds 2^31 - 1");
    }
    int rc;
    if ((rc = ensure(q0, size_t(n) * A * 4)) != BCTS_OK) return rc;
    float *q0p = static_cast<float *>(q0.p);
    if ((rc = qhead(d_roots, n, q0p, nullptr, st)) != BCTS_OK) return rc;
    if (d == 0) {
      rc = launch_finalize(q0p, nullptr, nullptr, nullptr, n, A, 0, A, gamma, 1.f, corr, d_action, d_values, st);
      return rc == BCTS_OK ? BCTS_OK : fail(rc, "DNN finalize launch failed");
    }
    if ((rc = ensure(maxq1, size_t(N[1]) * 4)) != BCTS_OK) return rc;
    if ((rc = ensure(r1, size_t(N[1]) * 4)) != BCTS_OK) return rc;
    if ((rc = ensure(V, size_t(N[1]) * 4)) != BCTS_OK) return rc;
    for (int b = 0; b < 2; ++b) {
      if ((rc = ensure(lvl[b], size_t(N[d]) * kD * 4)) != BCTS_OK) return rc;
      if ((rc = ensure(Rl[b], size_t(N[d]) * 4)) != BCTS_OK) return rc;
    }
    float *r1p = static_cast<float *>(r1.p), *m1 = static_cast<float *>(maxq1.p);
    // level 1 (R_1 = r(s_0, a), kept for the Bellman errors), its Q for Prop. 1
    float *cur = static_cast<float *>(lvl[1].p);
    if ((rc = expand(d_roots, nullptr, n, 1.f, cur, r1p, st)) != BCTS_OK) return rc;
    if ((rc = qhead(cur, N[1], nullptr, m1, st)) != BCTS_OK) return rc;
    const float *curR = r1p, *leafMax = m1;
    double gp = 1.0;
    for (int i = 1; i < d; ++i) {
      gp *= double(gamma);
      float *nxt = static_cast<float *>(lvl[(i + 1) & 1].p), *nxtR = static_cast<float *>(Rl[(i + 1) & 1].p);
      if ((rc = expand(cur, curR, N[i], float(gp), nxt, nxtR, st)) != BCTS_OK) return rc;
      cur = nxt;
      curR = nxtR;
    }
    if (d >= 2) {
      if ((rc = ensure(leafmax, size_t(N[d]) * 4)) != BCTS_OK) return rc;
      if ((rc = qhead(cur, N[d], nullptr, static_cast<float *>(leafmax.p), st)) != BCTS_OK) return rc;
      leafMax = static_cast<float *>(leafmax.p);
    }
    double gd = 1.0;
    for (int i = 0; i < d; ++i) gd *= double(gamma);
    int64_t seg = 1;
    for (int i = 1; i < d; ++i) seg *= A;
    float *Vp = static_cast<float *>(V.p);
    if ((rc = launch_segment_max(curR, leafMax, int64_t(n) * A, seg, float(gd), Vp, st)) != BCTS_OK)
      return fail(rc, "DNN backup launch failed");
    if ((rc = launch_finalize(q0p, m1, r1p, Vp, n, A, d, A, gamma, float(gd), corr, d_action, d_values, st, 0,
                              exact_gev ? 1 : 0)) != BCTS_OK)
      return fail(rc, "DNN finalize launch failed");
    return BCTS_OK;
  }
};

}  // namespace bcts

using bcts::DnnCtx;

extern "C" size_t bcts_dnn_numel(int A) {
  if (A < 1 || A > bcts::kMaxDnnA) return 0;
  const size_t D = bcts::kD, H = bcts::kH;
  return H * (D + A) + H + 2 * (H * H + H) + (D + 1) * H + (D + 1) + size_t(A) * D + size_t(A);
}

extern "C" int bcts_dnn_create(const float *weights, int A, int d, float gamma, float correction, int flags,
                               bcts_dnn_ctx **out) {
  using namespace bcts;
  if (!out || !weights || A < 1 || A > kMaxDnnA || d < 0 || d > kMaxDnnDepth || !(gamma > 0.f && gamma <= 1.f) ||
      !std::isfinite(correction)) {
    set_thread_error("bcts_dnn_create: invalid argument");
    return BCTS_EINVAL;
  }
  *out = nullptr;
  DnnCtx *c = new DnnCtx();
  c->A = A;
  c->d = d;
  c->gamma = gamma;
  c->corr = correction;
  c->exact_gev = (flags & BCTS_FLAG_EXACT_GEV) != 0;
  c->prof = profiler_create();
  if (cudaGetDevice(&c->device) != cudaSuccess || cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) !=
                                                      cudaSuccess) {
    cudaGetLastError();
    delete c;
    set_thread_error("bcts_dnn_create: no usable CUDA device");
    return BCTS_ECUDA;
  }
  // kernel layouts: W1 split into its state columns [H][D] and its action
  // columns transposed [A][H]; the other layers keep [out][in]
  const size_t D = kD, H = kH;
  const float *src = weights;
  const float *f1w = src, *f1b = f1w + H * (D + A), *f2w = f1b + H, *f2b = f2w + H * H, *f3w = f2b + H,
              *f3b = f3w + H * H, *fow = f3b + H, *fob = fow + (D + 1) * H, *fqw = fob + D + 1, *fqb = fqw + A * D;
  std::vector<float> hw;
  hw.reserve(bcts_dnn_numel(A));
  auto put = [&](const float *p, size_t n) {
    const size_t at = hw.size();
    hw.insert(hw.end(), p, p + n);
    return at;
  };
  std::vector<float> w1s(H * D), w1a(size_t(A) * H);
  for (size_t j = 0; j < H; ++j) {
    for (size_t k = 0; k < D; ++k) w1s[j * D + k] = f1w[j * (D + A) + k];
    for (int a = 0; a < A; ++a) w1a[size_t(a) * H + j] = f1w[j * (D + A) + D + a];
  }
  const size_t o_w1s = put(w1s.data(), w1s.size()), o_w1a = put(w1a.data(), w1a.size()), o_b1 = put(f1b, H),
               o_w2 = put(f2w, H * H), o_b2 = put(f2b, H), o_w3 = put(f3w, H * H), o_b3 = put(f3b, H),
               o_wo = put(fow, (D + 1) * H), o_bo = put(fob, D + 1), o_wq = put(fqw, size_t(A) * D),
               o_bq = put(fqb, A);
  if (cudaMalloc(&c->wbuf, hw.size() * sizeof(float)) != cudaSuccess ||
      cudaMemcpy(c->wbuf, hw.data(), hw.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    set_thread_error("bcts_dnn_create: weight upload failed");
    return BCTS_ENOMEM;
  }
  c->w1s = c->wbuf + o_w1s;
  c->w1a = c->wbuf + o_w1a;
  c->b1 = c->wbuf + o_b1;
  c->w2 = c->wbuf + o_w2;
  c->b2 = c->wbuf + o_b2;
  c->w3 = c->wbuf + o_w3;
  c->b3 = c->wbuf + o_b3;
  c->wo = c->wbuf + o_wo;
  c->bo = c->wbuf + o_bo;
  c->wq = c->wbuf + o_wq;
  c->bq = c->wbuf + o_bq;
  *out = reinterpret_cast<bcts_dnn_ctx *>(c);
  return BCTS_OK;
}

extern "C" void bcts_dnn_destroy(bcts_dnn_ctx *ctx) {
  if (!ctx) return;
  DnnCtx *c = reinterpret_cast<DnnCtx *>(ctx);
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  delete c;
}

extern "C" int bcts_dnn_search_device(bcts_dnn_ctx *ctx, const float *d_roots, int n, int32_t *d_action,
                                      float *d_values, void *stream) {
  if (!ctx) return BCTS_EINVAL;
  DnnCtx *c = reinterpret_cast<DnnCtx *>(ctx);
  if (n < 0 || (n > 0 && (!d_roots || !d_action || !d_values)))
    return c->fail(BCTS_EINVAL, "bcts_dnn_search_device: invalid argument");
  if (reinterpret_cast<uintptr_t>(d_roots) % 16 != 0)  // rows are copied to shared memory in 16-byte pieces
    return c->fail(BCTS_EINVAL, "bcts_dnn_search_device: d_roots must be 16-byte aligned");
  cudaSetDevice(c->device);
  return c->run(d_roots, n, d_action, d_values, stream ? (cudaStream_t)stream : c->stream);
}

extern "C" int bcts_dnn_search(bcts_dnn_ctx *ctx, const float *roots, int n, int32_t *out_action,
                               float *out_values) {
  using namespace bcts;
  if (!ctx) return BCTS_EINVAL;
  DnnCtx *c = reinterpret_cast<DnnCtx *>(ctx);
  if (n < 0 || (n > 0 && (!roots || !out_action || !out_values)))
    return c->fail(BCTS_EINVAL, "bcts_dnn_search: invalid argument");
  if (n == 0) return BCTS_OK;
  cudaSetDevice(c->device);
  const size_t in_b = size_t(n) * kD * 4, act_b = size_t(n) * 4, val_b = size_t(n) * c->A * 4;
  int rc;
  if ((rc = c->ensure(c->io_roots, in_b)) != BCTS_OK || (rc = c->ensure(c->io_act, act_b)) != BCTS_OK ||
      (rc = c->ensure(c->io_val, val_b)) != BCTS_OK)
    return rc;
  const size_t host_b = in_b + act_b + val_b;
  if (host_b > c->host_cap) {
    cudaStreamSynchronize(c->stream);
    if (c->host) cudaFreeHost(c->host);
    c->host = nullptr;
    c->host_cap = 0;
    if (cudaHostAlloc(&c->host, host_b, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return c->fail(BCTS_ENOMEM, "bcts_dnn_search: pinned host allocation failed");
    }
    c->host_cap = host_b;
  }
  char *hs = static_cast<char *>(c->host);
  std::memcpy(hs, roots, in_b);
  BCTS_CUDA_TRY(cudaMemcpyAsync(c->io_roots.p, hs, in_b, cudaMemcpyHostToDevice, c->stream), c->err);
  if ((rc = c->run(static_cast<const float *>(c->io_roots.p), n, static_cast<int32_t *>(c->io_act.p),
                   static_cast<float *>(c->io_val.p), c->stream)) != BCTS_OK)
    return rc;
  BCTS_CUDA_TRY(cudaMemcpyAsync(hs + in_b, c->io_act.p, act_b, cudaMemcpyDeviceToHost, c->stream), c->err);
  BCTS_CUDA_TRY(cudaMemcpyAsync(hs + in_b + act_b, c->io_val.p, val_b, cudaMemcpyDeviceToHost, c->stream), c->err);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return c->fail(BCTS_ECUDA, "bcts_dnn_search: CUDA error");
  }
  std::memcpy(out_action, hs + in_b, act_b);
  std::memcpy(out_values, hs + in_b + act_b, val_b);
  return BCTS_OK;
}

extern "C" int bcts_dnn_profile(bcts_dnn_ctx *ctx, int enable, double *out_ms, int64_t *out_launches,
                                int64_t *out_total) {
  if (!ctx) return BCTS_EINVAL;
  DnnCtx *c = reinterpret_cast<DnnCtx *>(ctx);
  return bcts::profiler_read(c->prof, c->stream, enable, out_ms, out_launches, out_total);
}

extern "C" const char *bcts_dnn_last_error(const bcts_dnn_ctx *ctx) {
  if (!ctx) return bcts_last_error(nullptr);
  return reinterpret_cast<const DnnCtx *>(ctx)->err.c_str();
}
