// search.cu -- the search context, the level-synchronous Batch-BFS driver
// (Alg. 1), the backup kernels (Eq. 1 max over each root action's sub-tree,
// Prop. 1 Bellman errors, Eq. 7 penalty, Eq. 3 correction, Eq. 4 argmax) and the
// C-ABI entry points that run them.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "search.cuh"

namespace bcts {

namespace {
thread_local std::string g_thread_err;
}

void set_thread_error(const std::string &msg) { g_thread_err = msg; }
const char *thread_error() { return g_thread_err.c_str(); }

// ---------------------------------------------------------------------------
// Backup kernels
// ---------------------------------------------------------------------------
namespace {

// Segment maxima are kept as order-preserving 32-bit keys: for finite floats
// key(a) < key(b) exactly when a < b, and key 0 lies below every float, so a
// zero-filled array means "no value yet" and atomicMax on keys is a float max
// whose result does not depend on the order of the updates.
__device__ __forceinline__ uint32_t order_key(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_value(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// V[s] = max over the seg_len consecutive leaves of segment s of R + gamma^d maxq
// (Alg. 1's leaf term; Eq. 1's max over a_1..a_d for root action s mod A).
// Short segments: one warp per segment, eight coalesced loads of each array in
// flight per lane.
// One segment by one warp.
__device__ __forceinline__ void segment_max_warp(const float *__restrict__ r, const float *__restrict__ q,
                                                 int64_t seg_len, float gamma_pow, uint32_t *__restrict__ out,
                                                 int lane) {
  float best = -INFINITY;
  int64_t i = lane;
  for (; i + 224 < seg_len; i += 256) {  // eight loads of each array in flight per lane
    float rv[8], qv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      rv[k] = __ldg(r + i + 32 * k);
      qv[k] = __ldg(q + i + 32 * k);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) best = fmaxf(best, rv[k] + gamma_pow * qv[k]);
  }
  for (; i < seg_len; i += 32) best = fmaxf(best, __ldg(r + i) + gamma_pow * __ldg(q + i));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
  if (lane == 0) *out = order_key(best);
}

__global__ void __launch_bounds__(256) segment_max_warp_kernel(const float *__restrict__ R,
                                                               const float *__restrict__ maxq, int64_t n_seg,
                                                               int64_t seg_len, float gamma_pow,
                                                               uint32_t *__restrict__ V) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t s = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); s < n_seg; s += nwarps)
    segment_max_warp(R + s * seg_len, maxq + s * seg_len, seg_len, gamma_pow, V + s, lane);
}

// The segments of several independent searches (the batched form's (A, d)
// groups) in one launch: group k's segments are seg_end[k - 1] .. seg_end[k] - 1.
__global__ void __launch_bounds__(256) segment_max_list_kernel(const __grid_constant__ BackupList L) {
  const int lane = threadIdx.x & 31;
  const int64_t total = L.seg_end[L.n - 1];
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t s = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); s < total; s += nwarps) {
    int k = 0;
    while (k < L.n - 1 && s >= L.seg_end[k]) ++k;
    const int64_t ls = s - (k ? L.seg_end[k - 1] : 0), len = L.seg_len[k];
    segment_max_warp(L.R[k] + ls * len, L.maxq[k] + ls * len, len, L.gamma_d[k],
                     reinterpret_cast<uint32_t *>(L.V[k]) + ls, lane);
  }
}

// Segments of kSegPart leaves or more: each block reduces kSegPart consecutive
// leaves of one segment
// (eight loads of each array in flight per thread) and folds its maximum into the
// segment's key with atomicMax; V is zero-filled first.
constexpr int kSegThreads = 256, kSegPerThread = 16, kSegPart = kSegThreads * kSegPerThread;
__global__ void __launch_bounds__(kSegThreads) segment_max_split_kernel(const float *__restrict__ R,
                                                                       const float *__restrict__ maxq,
                                                                       int64_t seg_len, int64_t parts,
                                                                       float gamma_pow,
                                                                       uint32_t *__restrict__ V) {
  const int64_t s = blockIdx.x / parts, part = blockIdx.x - s * parts;
  const int64_t lo = part * kSegPart, hi = lo + kSegPart < seg_len ? lo + kSegPart : seg_len;
  const float *r = R + s * seg_len, *q = maxq + s * seg_len;
  float best = -INFINITY;
  if (hi - lo == kSegPart) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v[kSegPerThread / 2];
#pragma unroll
      for (int k = 0; k < kSegPerThread / 2; ++k) {
        const int64_t i = lo + threadIdx.x + int64_t(h * (kSegPerThread / 2) + k) * kSegThreads;
        v[k] = __ldg(r + i) + gamma_pow * __ldg(q + i);
      }
#pragma unroll
      for (int k = 0; k < kSegPerThread / 2; ++k) best = fmaxf(best, v[k]);
    }
  } else {
    for (int64_t i = lo + threadIdx.x; i < hi; i += kSegThreads)
      best = fmaxf(best, __ldg(r + i) + gamma_pow * __ldg(q + i));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
  __shared__ float part_max[kSegThreads / 32];
  if ((threadIdx.x & 31) == 0) part_max[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = part_max[0];
#pragma unroll
    for (int w = 1; w < kSegThreads / 32; ++w) b = fmaxf(b, part_max[w]);
    atomicMax(V + s, order_key(b));
  }
}

// Lowest-index argmax across the warp (lanes carry (value, index) pairs).
__device__ __forceinline__ void warp_argmax_lowest(float &v, int &idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
    }
  }
}

// One warp per root, lane a holding action a (A <= 32): pi_o = argmax Q_0
// (Sec. 3.3, lowest index on ties), delta(a) from depths 0 and 1 (Prop. 1),
// delta_o = |delta(pi_o)|, delta_e = mean |delta(a)| over a != pi_o, the penalty
// B (Eq. 7, or with exact_gev Lemma 2's gap from the GEV shifts gev_e, gev_o the
// host computed for A^d - A^(d-1) and A^(d-1) leaves), corrected values (Eq. 3,
// scaled by c) and the action (Eq. 4).  V holds the segment maxima as order
// keys; `values` may alias V (each lane reads its own key before it writes).
__device__ __forceinline__ void finalize_root(const float *__restrict__ q0, const float *__restrict__ maxq1,
                                              const float *__restrict__ r1, const uint32_t *V, int64_t i, int A,
                                              int depth, int A_stride, float gamma, float gamma_d, float corr,
                                              int32_t *__restrict__ action, float *values, int q_stride,
                                              int exact_gev, float gev_e, float gev_o, int lane) {
  const bool on = lane < A;
  const float q = on ? q0[size_t(i) * q_stride + lane] : -INFINITY;
  float bq = q;
  int pi_o = on ? lane : 64;
  warp_argmax_lowest(bq, pi_o);
  float *out = values + size_t(i) * A_stride;
  if (depth == 0) {
    if (on) out[lane] = q;
    else if (lane < A_stride) out[lane] = 0.f;
    if (lane == 0) action[i] = pi_o;
    return;
  }
  const float Vv = on ? key_value(V[size_t(i) * A + lane]) : -INFINITY;
  const float delta = on ? r1[size_t(i) * A + lane] + gamma * maxq1[size_t(i) * A + lane] - q : 0.f;
  const float d_o = __shfl_sync(0xffffffffu, fabsf(delta), pi_o);
  float d_e = (on && lane != pi_o) ? fabsf(delta) : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d_e += __shfl_xor_sync(0xffffffffu, d_e, o);
  if (A > 1) d_e /= float(A - 1);
  float B;
  if (exact_gev) {
    B = 0.70710678118654752f * (d_e * gev_e - d_o * gev_o);  // sigma = delta / sqrt(2) (Prop. 1)
  } else {
    B = sqrtf(logf(float(A))) * (d_e * sqrtf(float(depth)) - d_o * sqrtf(float(depth - 1))) -
        (d_e - d_o) * 0.35355339059327373f;  // Eq. 7; 1 / sqrt(8)
  }
  const float pen = gamma_d * corr * B;
  float v = on ? Vv - (lane == pi_o ? 0.f : pen) : -INFINITY;
  __syncwarp();
  if (on) out[lane] = v;
  else if (lane < A_stride) out[lane] = 0.f;
  int best = on ? lane : 64;
  warp_argmax_lowest(v, best);
  if (lane == 0) action[i] = best;
}

__global__ void __launch_bounds__(256) finalize_kernel(const float *__restrict__ q0, const float *__restrict__ maxq1,
                                                       const float *__restrict__ r1, const uint32_t *V, int n,
                                                       int A, int depth, int A_stride, float gamma, float gamma_d,
                                                       float corr, int32_t *__restrict__ action, float *values,
                                                       int q_stride, int exact_gev, float gev_e, float gev_o) {
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;  // whole warps leave together
  finalize_root(q0, maxq1, r1, V, i, A, depth, A_stride, gamma, gamma_d, corr, action, values, q_stride, exact_gev,
                gev_e, gev_o, threadIdx.x & 31);
}

// The roots of several groups in one launch: group k's roots are
// root_end[k - 1] .. root_end[k] - 1, each with its own A, d and arrays.
__global__ void __launch_bounds__(256) finalize_list_kernel(const __grid_constant__ BackupList L) {
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (i >= L.root_end[L.n - 1]) return;
  int k = 0;
  while (k < L.n - 1 && i >= L.root_end[k]) ++k;
  finalize_root(L.q0[k], L.maxq1[k], L.r1[k], reinterpret_cast<const uint32_t *>(L.V[k]),
                i - (k ? L.root_end[k - 1] : 0), L.A[k], L.depth[k], L.A_stride, L.gamma, L.gamma_d[k], L.corr,
                L.action[k], L.values[k], L.q_stride, L.exact_gev, L.gev_e[k], L.gev_o[k], threadIdx.x & 31);
}

}  // namespace

// Lemma 2: expected shift of the maximum of m iid standard normals, the mean of
// its GEV limit, Phi^-1(1 - 1/m) + gamma_EM (Phi^-1(1 - 1/(e m)) - Phi^-1(1 - 1/m));
// 0 for one element.  Computed on the host in double: it depends only on (A, d).
// The upper quantile x(p), Q(x) = erfc(x / sqrt 2) / 2 = p, is found by Newton's
// method on log Q(x) = log p, kept inside a bisection bracket.
static double upper_normal_quantile(double p) {
  if (!(p > 0.0 && p < 1.0)) return p >= 1.0 ? -INFINITY : INFINITY;
  const double kRt2 = 1.4142135623730951, kRt2Pi = 2.5066282746310002;
  double lo = -40.0, hi = 40.0;
  double x = p < 0.5 ? std::sqrt(-2.0 * std::log(p)) : 0.0;
  for (int it = 0; it < 200; ++it) {
    const double Q = 0.5 * std::erfc(x / kRt2);
    if (Q > p) lo = x; else hi = x;
    const double phi = std::exp(-0.5 * x * x) / kRt2Pi;
    // d/dx log Q = -phi / Q, so the Newton step is (log Q - log p) Q / phi
    double nx = (Q > 0.0 && phi > 0.0) ? x + (std::log(Q) - std::log(p)) * Q / phi : 0.5 * (lo + hi);
    if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
    if (std::fabs(nx - x) <= 1e-15 * std::max(1.0, std::fabs(x))) return nx;
    x = nx;
  }
  return x;
}

static double gev_shift_host(double m) {
  if (m <= 1.0) return 0.0;
  const double x1 = upper_normal_quantile(1.0 / m);
  const double xe = upper_normal_quantile(1.0 / (2.718281828459045 * m));
  return x1 + 0.5772156649015329 * (xe - x1);
}

static int num_sms_backup() {
  static int sms = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
  });
  return sms;
}

// V (n_seg floats of storage) receives the segment maxima as order keys.
int launch_segment_max(const float *R, const float *maxq, int64_t n_seg, int64_t seg_len, float gamma_pow,
                       float *V, cudaStream_t st) {
  if (n_seg <= 0) return BCTS_OK;
  ProfScope ps(K_BACKUP, st);
  uint32_t *key = reinterpret_cast<uint32_t *>(V);
  if (seg_len >= kSegPart) {
    const int64_t parts = (seg_len + kSegPart - 1) / kSegPart;
    if (n_seg * parts > 0x7FFFFFFFLL) return BCTS_EINVAL;
    if (cudaMemsetAsync(key, 0, size_t(n_seg) * sizeof(uint32_t), st) != cudaSuccess) return BCTS_ECUDA;
    segment_max_split_kernel<<<unsigned(n_seg * parts), kSegThreads, 0, st>>>(R, maxq, seg_len, parts, gamma_pow,
                                                                              key);
  } else {
    const int64_t blocks = (n_seg + 7) / 8;
    const int64_t cap = int64_t(num_sms_backup()) * 8;  // 8 resident 256-thread blocks per SM
    segment_max_warp_kernel<<<unsigned(blocks < cap ? blocks : cap), 256, 0, st>>>(R, maxq, n_seg, seg_len,
                                                                                   gamma_pow, key);
  }
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

// Per-node export.  U = R + gamma^i V is the best root-discounted return through a
// node: at the leaves R + gamma^d max_a Q, above them the max over the A children
// (Alg. 1 order: children of x are x*A .. x*A + A - 1), so the upward pass is a
// pure max.  V = (U - R) / gamma^i is formed level by level afterwards.
__global__ void tree_leaf_kernel(const float *__restrict__ R, const float *__restrict__ maxq, float gamma_d,
                                 float *__restrict__ U, int64_t n) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) U[i] = R[i] + gamma_d * maxq[i];
}
__global__ void tree_up_kernel(const float *__restrict__ Uc, int A, float *__restrict__ U, int64_t n) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  float m = Uc[i * A];
  for (int a = 1; a < A; ++a) m = fmaxf(m, Uc[i * A + a]);
  U[i] = m;
}
__global__ void tree_value_kernel(const float *__restrict__ R, float inv_gamma_i, float *__restrict__ UV,
                                  int64_t n) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) UV[i] = (UV[i] - R[i]) * inv_gamma_i;
}

int launch_finalize(const float *q0, const float *maxq1, const float *r1, const float *V, int n, int A, int depth,
                    int A_stride, float gamma, float gamma_d, float corr, int32_t *action, float *values,
                    cudaStream_t st, int q_stride, int exact_gev) {
  if (n <= 0) return BCTS_OK;
  if (A > 32 || A_stride > 32) return BCTS_EINVAL;  // one warp per root
  ProfScope ps(K_BACKUP, st);
  float gev_e = 0.f, gev_o = 0.f;
  if (exact_gev && depth >= 1) {
    // Eq. 3's gap B_e - B_o itself (Lemma 2): A^d - A^(d-1) leaves under a != pi_o
    // against A^(d-1) under pi_o
    const double n_o = std::pow(double(A), double(depth - 1)), n_e = std::pow(double(A), double(depth)) - n_o;
    gev_e = float(gev_shift_host(n_e));
    gev_o = float(gev_shift_host(n_o));
  }
  finalize_kernel<<<unsigned((int64_t(n) * 32 + 255) / 256), 256, 0, st>>>(
      q0, maxq1, r1, reinterpret_cast<const uint32_t *>(V), n, A, depth, A_stride, gamma, gamma_d, corr, action,
      values, q_stride > 0 ? q_stride : A, exact_gev, gev_e, gev_o);
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

int launch_backup_list(BackupList &L, cudaStream_t st) {
  if (L.n <= 0) return BCTS_OK;
  ProfScope ps(K_BACKUP, st);
  for (int k = 0; k < L.n; ++k) {
    if (L.A[k] > 32 || L.A_stride > 32 || (L.depth[k] >= 1 && L.seg_len[k] >= 2 * kSegPart)) return BCTS_EINVAL;
    L.gev_e[k] = L.gev_o[k] = 0.f;
    if (L.exact_gev && L.depth[k] >= 1) {
      const double n_o = std::pow(double(L.A[k]), double(L.depth[k] - 1));
      const double n_e = std::pow(double(L.A[k]), double(L.depth[k])) - n_o;
      L.gev_e[k] = float(gev_shift_host(n_e));
      L.gev_o[k] = float(gev_shift_host(n_o));
    }
  }
  const int64_t segs = L.seg_end[L.n - 1];
  if (segs > 0) {
    const int64_t blocks = (segs + 7) / 8, cap = int64_t(num_sms_backup()) * 8;
    segment_max_list_kernel<<<unsigned(blocks < cap ? blocks : cap), 256, 0, st>>>(L);
  }
  const int64_t roots = L.root_end[L.n - 1];
  finalize_list_kernel<<<unsigned((roots * 32 + 255) / 256), 256, 0, st>>>(L);
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

// ---------------------------------------------------------------------------
// Context helpers
// ---------------------------------------------------------------------------
int Ctx::fail(int code, const std::string &msg) {
  err = msg;
  set_thread_error(msg);
  return code;
}

int Ctx::ensure(DevBuf &b, size_t bytes) {
  if (bytes <= b.cap) return BCTS_OK;
  const size_t old_cap = b.cap;
  if (b.p) {
    cudaStreamSynchronize(stream);
    cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  // Grow by at least half of the old capacity, so that a slowly rising size
  // (a serving load ramping up) reallocates only O(log) times: every
  // reallocation synchronises the device and invalidates captured graphs.
  const size_t exact = (bytes + 255) & ~size_t(255);
  const size_t grown = (std::max(exact, old_cap + old_cap / 2) + 255) & ~size_t(255);
  ++buf_generation;
  size_t want = grown;
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    want = exact;
    if (want == grown || cudaMalloc(&b.p, want) != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return fail(BCTS_ENOMEM, "device allocation of " + std::to_string(want) + " bytes failed");
    }
  }
  b.cap = want;
  return BCTS_OK;
}

int Ctx::ensure_host(HostBuf &b, size_t bytes) {
  if (bytes <= b.cap) return BCTS_OK;
  if (b.p) {
    cudaStreamSynchronize(stream);
    cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  const size_t want = (bytes + 255) & ~size_t(255);
  if (cudaHostAlloc(&b.p, want, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return fail(BCTS_ENOMEM, "pinned host allocation failed");
  }
  b.cap = want;
  return BCTS_OK;
}

int64_t Ctx::chunk_nodes(int64_t count) const {
  if (opt.leaf_chunk > 0) return opt.leaf_chunk;
  if (chunk_override > 0) return chunk_override;
  if (precision == BCTS_PREC_FP32_SIMT) return 16384;
  // One pass over as many nodes as fit, with their activation maps, in 1/16 of the
  // device memory (at least 32,768): longer passes amortise fc1's weight reads and
  // the launches (measured at the Atari-scale workload: one pass over 186,624
  // leaves against passes of 32,768: +2 % FP32-class, +8 % BF16 and E4M3).  A
  // larger count is split into equal passes.
  const int64_t per = int64_t(tc_scratch_bytes(int64_t(1) << 16, precision) >> 16) + 1;
  int64_t cap = int64_t(dev_mem / 16) / per;
  if (cap < 32768) cap = 32768;
  if (count <= 0) return cap;
  if (count <= cap) return count;
  const int64_t k = (count + cap - 1) / cap;
  return (count + k - 1) / k;
}

// Score `count` nodes: render + Q-network, chunked.  q (count x A) and maxq
// (count) may each be NULL.
int Ctx::eval_nodes(const bcts_state *states, int64_t count, float *q, float *maxq, cudaStream_t st,
                    const uint8_t *node_A, const float *zmap, uint32_t zbranch, const uint32_t *zparent) {
  const int64_t chunk = chunk_nodes(count);
  int rc;
  for (int64_t off = 0; off < count; off += chunk) {
    const int64_t cnt = count - off < chunk ? count - off : chunk;
    const ZLeaf zl{zmap, uint32_t(off), zbranch, zparent};
    if ((rc = qnet_nodes(states + off, nullptr, cnt, q ? q + off * A : nullptr, maxq ? maxq + off : nullptr, st,
                         node_A ? node_A + off : nullptr, zmap ? &zl : nullptr)) != BCTS_OK)
      return rc;
  }
  return BCTS_OK;
}

int Ctx::eval_nodes_ref(const bcts_state *states, int64_t count, float *q, float *maxq, cudaStream_t st,
                        const uint8_t *node_A) {
  ref_eval = true;
  const int rc = eval_nodes(states, count, q, maxq, st, node_A);
  ref_eval = false;
  return rc;
}

int Ctx::eval_frames(const FrameSrc &f, int64_t count, float *q, float *maxq, cudaStream_t st, bool ref) {
  const bool r = ref && tc_ref;
  const int64_t chunk = chunk_nodes(count);
  int rc;
  for (int64_t off = 0; off < count; off += chunk) {
    const int64_t cnt = count - off < chunk ? count - off : chunk;
    if ((rc = ensure(scratch_buf, tc_scratch_bytes(cnt, r ? int(BCTS_PREC_FP32) : precision))) != BCTS_OK) return rc;
    FrameSrc fc = f;
    fc.node0 = f.node0 + uint32_t(off);
    if (f.zmap) fc.zleaf0 = f.zleaf0 + uint32_t(off);
    rc = tc_qnet_forward(r ? tc_ref : tc, A, nullptr, nullptr, cnt, q ? q + off * A : nullptr,
                         maxq ? maxq + off : nullptr, scratch_buf.p, st, d_err, nullptr, nullptr, r ? -1 : conv_mask,
                         &fc);
    if (rc != BCTS_OK) return fail(rc, "tensor-core Q-network launch failed");
  }
  return BCTS_OK;
}

// Q-network on at most one chunk of nodes, given either states (rendered here)
// or frames.
int Ctx::qnet_nodes(const bcts_state *states, const uint8_t *frames, int64_t cnt, float *q, float *maxq,
                    cudaStream_t st, const uint8_t *node_A, const ZLeaf *zl) {
  int rc;
  if (precision == BCTS_PREC_FP32_SIMT) {
    if (states) {
      if ((rc = ensure(frames_buf, size_t(cnt) * kFrameBytes)) != BCTS_OK) return rc;
      if ((rc = launch_render(states, cnt, static_cast<uint8_t *>(frames_buf.p), st)) != BCTS_OK)
        return fail(rc, "render launch failed");
      frames = static_cast<const uint8_t *>(frames_buf.p);
    }
    if ((rc = ensure(scratch_buf, simt_scratch_bytes(cnt))) != BCTS_OK) return rc;
    SimtWeights w = simt;
    w.A = A;  // FC2 rows 0..A-1
    if ((rc = simt_qnet_forward(w, frames, cnt, q, maxq, scratch_buf.p, st, node_A)) != BCTS_OK)
      return fail(rc, "Q-network launch failed");
    return BCTS_OK;
  }
  if (states && !tc_fused_render) {
    if ((rc = ensure(frames_buf, size_t(cnt) * kFrameBytes)) != BCTS_OK) return rc;
    if ((rc = launch_render(states, cnt, static_cast<uint8_t *>(frames_buf.p), st)) != BCTS_OK)
      return fail(rc, "render launch failed");
    frames = static_cast<const uint8_t *>(frames_buf.p);
    states = nullptr;
  }
  const bool ref = ref_eval && tc_ref;
  if ((rc = ensure(scratch_buf, tc_scratch_bytes(cnt, ref ? int(BCTS_PREC_FP32) : precision))) != BCTS_OK) return rc;
  rc = tc_qnet_forward(ref ? tc_ref : tc, A, frames, states, cnt, q, maxq, scratch_buf.p, st, d_err, node_A,
                       states ? zl : nullptr, ref ? -1 : conv_mask);
  if (rc != BCTS_OK) return fail(rc, "tensor-core Q-network launch failed");
  return BCTS_OK;
}

// Per-node export after the backup: U = R + gamma^d max Q at the leaves, a max over
// the children upwards, then V = (U - R) / gamma^i per level; the leaves' V is
// their max Q itself.
int Ctx::export_tree(const std::vector<int64_t> &N, int A_, int d_, const float *leafMax, cudaStream_t st) {
  if (d_ < 1) return BCTS_OK;
  ProfScope ps(K_BACKUP, st);
  std::vector<int64_t> off(d_ + 1, 0);  // first node of level i (off[1] = 0)
  for (int i = 2; i <= d_; ++i) off[i] = off[i - 1] + N[i - 1];
  std::vector<double> gpow(d_ + 1, 1.0);
  for (int i = 1; i <= d_; ++i) gpow[i] = gpow[i - 1] * double(gamma);
  auto blocks = [](int64_t n) { return unsigned((n + 255) / 256); };
  tree_leaf_kernel<<<blocks(N[d_]), 256, 0, st>>>(tree_R + off[d_], leafMax, float(gpow[d_]), tree_V + off[d_],
                                                  N[d_]);
  for (int i = d_ - 1; i >= 1; --i)
    tree_up_kernel<<<blocks(N[i]), 256, 0, st>>>(tree_V + off[i + 1], A_, tree_V + off[i], N[i]);
  for (int i = 1; i < d_; ++i)
    tree_value_kernel<<<blocks(N[i]), 256, 0, st>>>(tree_R + off[i], float(1.0 / gpow[i]), tree_V + off[i], N[i]);
  if (cudaGetLastError() != cudaSuccess) return fail(BCTS_ECUDA, "tree export launch failed");
  BCTS_CUDA_TRY(cudaMemcpyAsync(tree_V + off[d_], leafMax, size_t(N[d_]) * sizeof(float), cudaMemcpyDeviceToDevice,
                                st),
                err);
  return BCTS_OK;
}

// Alg. 1 for n roots sharing (A_, d_): level-synchronous expansion, root and
// depth-1 evaluation for the Bellman errors, leaf scoring, backup.
int Ctx::run_search(const bcts_state *d_roots, int n, int A_, int d_, int32_t *d_action, float *d_values,
                    int A_stride, cudaStream_t st) {
  if (n <= 0) return BCTS_OK;
  if (prune_keep > 0 && d_ >= 3 && A_ == A_create && d_ == d)
    return run_search_pruned(d_roots, n, prune_keep, d_action, d_values, A_stride, st);
  ProfilerGuard pg(prof);
  std::vector<int64_t> N(d_ + 1);
  N[0] = n;
  for (int i = 1; i <= d_; ++i) N[i] = N[i - 1] * A_;
  if (N[d_] > 0x7FFFFFFFLL) return fail(BCTS_EINVAL, "tree too large: n * A^d exceeds 2^31 - 1");
  const int saved_A = A;
  A = A_;  // eval_nodes writes q rows of A_ entries
  int rc = BCTS_OK;
  const size_t lvl_bytes = size_t(d_ >= 1 ? N[d_] : 1) * kStateBytes;
  const size_t r_bytes = size_t(d_ >= 1 ? N[d_] : 1) * sizeof(float);
  do {
    if ((rc = ensure(q0_buf, size_t(n) * A_ * sizeof(float))) != BCTS_OK) break;
    if ((rc = ensure(maxq1_buf, size_t(n) * A_ * sizeof(float))) != BCTS_OK) break;
    if ((rc = ensure(V_buf, size_t(n) * A_ * sizeof(float))) != BCTS_OK) break;
    float *q0 = static_cast<float *>(q0_buf.p);
    float *maxq1 = static_cast<float *>(maxq1_buf.p);
    float *V = static_cast<float *>(V_buf.p);
    // Frame path (a tensor-core context with BCTS_FLAG_FRAMES): every node's
    // newest frame is rendered into device memory when its level is expanded
    // (the roots' whole stacks up front), and conv1 reads the stacks those frames
    // form (frame stacking, Sec. 5: slot h of a node at level i is the newest
    // frame of its ancestor 3 - h levels up, Alg. 1's parent being x / A).
    const bool fpath = tc && !tc_fused_render;
    const uint8_t *rootfr = nullptr;
    // slot h of the nodes of level i as frame source s of f
    auto slot_src = [&](int i, int h, FrameSrc &f, int sidx) {
      const int j = 3 - h;
      uint32_t div = 1;
      for (int k = 0; k < (i - j >= 1 ? j : i); ++k) div *= uint32_t(A_);
      f.div[sidx] = div;
      f.sub[sidx] = 0;
      if (i - j >= 1) {
        f.src[sidx] = static_cast<const uint8_t *>(lvlfr_buf[i - j].p);
        f.stride[sidx] = kSlotBytes;
      } else {
        f.src[sidx] = rootfr + (h + i) * kSlotBytes;
        f.stride[sidx] = kFrameBytes;
      }
    };
    if (fpath) {
      if ((rc = ensure(rootfr_buf, size_t(n) * kFrameBytes)) != BCTS_OK) break;
      rootfr = static_cast<const uint8_t *>(rootfr_buf.p);
      if ((rc = launch_render(d_roots, n, static_cast<uint8_t *>(rootfr_buf.p), st)) != BCTS_OK) {
        rc = fail(rc, "render launch failed");
        break;
      }
      size_t need = 0;  // inner levels' frames
      for (int i = 1; i < d_; ++i) need += size_t(N[i]) * kSlotBytes;
      if (need > (size_t(24) << 30)) {
        rc = fail(BCTS_ENOMEM, "frame path: the inner levels' frames exceed 24 GiB for this tree");
        break;
      }
    }
    // a1: root evaluation, pi_o (FP32-class in every precision)
    if (fpath) {
      FrameSrc f0;
      for (int h = 0; h < kHist; ++h) slot_src(0, h, f0, h);
      if ((rc = eval_frames(f0, n, q0, nullptr, st, true)) != BCTS_OK) break;
    } else if ((rc = eval_nodes_ref(d_roots, n, q0, nullptr, st)) != BCTS_OK) {
      break;
    }
    if (d_ == 0) {
      rc = launch_finalize(q0, nullptr, nullptr, nullptr, n, A_, 0, A_stride, gamma, 1.f, corr, d_action,
                           d_values, st);
      break;
    }
    for (int b = 0; b < 2; ++b) {
      if ((rc = ensure(lvl_buf[b], lvl_bytes)) != BCTS_OK) break;
      if ((rc = ensure(R_buf[b], r_bytes)) != BCTS_OK) break;
    }
    if (rc != BCTS_OK) break;
    if ((rc = ensure(r1_buf, size_t(n) * A_ * sizeof(float))) != BCTS_OK) break;
    // a2 at depth 0 -> 1; R_1 = r(s_0, a) (kept for the Bellman errors)
    bcts_state *L1 = static_cast<bcts_state *>(lvl_buf[1].p);
    float *r1 = static_cast<float *>(r1_buf.p);
    if ((rc = launch_expand(d_roots, nullptr, n, A_, 1.f, L1, r1, nullptr, st)) != BCTS_OK) {
      rc = fail(rc, "expand launch failed");
      break;
    }
    if (tree_R)
      BCTS_CUDA_TRY(cudaMemcpyAsync(tree_R, r1, size_t(N[1]) * sizeof(float), cudaMemcpyDeviceToDevice, st), err);
    // a3: depth-1 evaluation (for d = 1 these are the leaves), FP32-class in every
    // precision: these Q-values enter the Bellman errors of Prop. 1
    if (fpath) {
      if ((rc = ensure(lvlfr_buf[1], size_t(N[1]) * kSlotBytes)) != BCTS_OK) break;
      if ((rc = launch_render_newest(L1, N[1], static_cast<uint8_t *>(lvlfr_buf[1].p), st)) != BCTS_OK) {
        rc = fail(rc, "render launch failed");
        break;
      }
      FrameSrc f1;
      for (int h = 0; h < kHist; ++h) slot_src(1, h, f1, h);
      if ((rc = eval_frames(f1, N[1], nullptr, maxq1, st, true)) != BCTS_OK) break;
    } else if ((rc = eval_nodes_ref(L1, N[1], nullptr, maxq1, st)) != BCTS_OK) {
      break;
    }
    const float *leafR = r1;
    const float *leafMax = maxq1;
    if (d_ >= 2) {
      // a2 for depths 1 .. d-1 (ping-pong level buffers; level 1 lives in buffer 1)
      const bcts_state *cur = L1;
      const float *curR = r1;
      double gp = 1.0;
      for (int i = 1; i < d_; ++i) {
        gp *= double(gamma);
        bcts_state *nxt = static_cast<bcts_state *>(lvl_buf[(i + 1) & 1].p);
        float *nxtR = static_cast<float *>(R_buf[(i + 1) & 1].p);
        if ((rc = launch_expand(cur, curR, N[i], A_, float(gp), nxt, nxtR, nullptr, st)) != BCTS_OK) {
          rc = fail(rc, "expand launch failed");
          break;
        }
        if (tree_R) {
          int64_t off = 0;  // first node of level i + 1 in the export
          for (int j = 1; j <= i; ++j) off += N[j];
          if (cudaMemcpyAsync(tree_R + off, nxtR, size_t(N[i + 1]) * sizeof(float), cudaMemcpyDeviceToDevice,
                              st) != cudaSuccess) {
            rc = fail(BCTS_ECUDA, "tree export copy failed");
            break;
          }
        }
        if (fpath && i + 1 < d_) {  // an inner level: its newest frames
          if ((rc = ensure(lvlfr_buf[i + 1], size_t(N[i + 1]) * kSlotBytes)) != BCTS_OK) break;
          if ((rc = launch_render_newest(nxt, N[i + 1], static_cast<uint8_t *>(lvlfr_buf[i + 1].p), st)) !=
              BCTS_OK) {
            rc = fail(rc, "render launch failed");
            break;
          }
        }
        cur = nxt;
        curR = nxtR;
      }
      if (rc != BCTS_OK) break;
      // a4 + a5: leaf render and Q-network, max over actions.  With a tensor-core
      // context the leaf conv1 needs only the newest frame: the parents' three
      // newer slots (the leaves' older three) enter as partial maps computed
      // once per parent (when they fit: 51.2 KB per parent).
      if ((rc = ensure(leafmax_buf, size_t(N[d_]) * sizeof(float))) != BCTS_OK) break;
      if (fpath) {
        // the parents' partial conv1 maps on the tensor cores (weight channels 0-2
        // over their slots 1-3) when they fit, then per chunk of leaves: render
        // the leaves' newest frames, conv1 of that slot plus the parent's map
        const size_t zb = size_t(N[d_ - 1]) * kP1 * kC1 * sizeof(float);
        float *z = nullptr;
        if (zb <= (size_t(8) << 30)) {
          if ((rc = ensure(z_buf, zb)) != BCTS_OK) break;
          z = static_cast<float *>(z_buf.p);
          FrameSrc fz;
          for (int h = 1; h < kHist; ++h) slot_src(d_ - 1, h, fz, h - 1);
          const int64_t chunk = chunk_nodes(N[d_ - 1]);
          for (int64_t off = 0; off < N[d_ - 1] && rc == BCTS_OK; off += chunk) {
            const int64_t cnt = N[d_ - 1] - off < chunk ? N[d_ - 1] - off : chunk;
            fz.node0 = uint32_t(off);
            rc = tc_conv1_zmap_frames(tc, fz, cnt, z + size_t(off) * kP1 * kC1, st, d_err);
          }
          if (rc != BCTS_OK) {
            rc = fail(rc, "conv1 partial launch failed");
            break;
          }
        }
        const int64_t chunk = chunk_nodes(N[d_]);
        if ((rc = ensure(frames_buf, size_t(std::min<int64_t>(chunk, N[d_])) * kSlotBytes)) != BCTS_OK) break;
        uint8_t *lf = static_cast<uint8_t *>(frames_buf.p);
        float *lm = static_cast<float *>(leafmax_buf.p);
        for (int64_t off = 0; off < N[d_] && rc == BCTS_OK; off += chunk) {
          const int64_t cnt = N[d_] - off < chunk ? N[d_] - off : chunk;
          if ((rc = launch_render_newest(cur + off, cnt, lf, st)) != BCTS_OK) {
            rc = fail(rc, "render launch failed");
            break;
          }
          FrameSrc fl;
          if (z) {  // slot 3 only, plus the parent's partial map
            fl.src[0] = lf;
            fl.stride[0] = kSlotBytes;
            fl.zmap = z;
            fl.zleaf0 = uint32_t(off);
            fl.zbranch = uint32_t(A_);
          } else {  // the whole stack: slot 3 from this chunk, slots 0-2 from the ancestors
            for (int h = 0; h < kHist - 1; ++h) slot_src(d_, h, fl, h);
            fl.src[3] = lf;
            fl.stride[3] = kSlotBytes;
            fl.div[3] = 1;
            fl.sub[3] = uint32_t(off);
            fl.node0 = uint32_t(off);
          }
          rc = eval_frames(fl, cnt, nullptr, lm + off, st, false);
        }
        if (rc != BCTS_OK) break;
        leafR = curR;
        leafMax = lm;
      } else {
      const float *zmap = nullptr;
      const size_t zbytes = size_t(N[d_ - 1]) * kP1 * kC1 * sizeof(float);
      if (tc && tc_fused_render && tc_has_partial(tc) && zbytes <= (size_t(8) << 30)) {
        if ((rc = ensure(z_buf, zbytes)) != BCTS_OK) break;
        const bcts_state *par = static_cast<const bcts_state *>(lvl_buf[(d_ - 1) & 1].p);
        if (d_ - 1 == 1) par = L1;
        const int64_t chunk = chunk_nodes(N[d_ - 1]);
        for (int64_t off = 0; off < N[d_ - 1] && rc == BCTS_OK; off += chunk) {
          const int64_t cnt = N[d_ - 1] - off < chunk ? N[d_ - 1] - off : chunk;
          rc = tc_conv1_partial(tc, par + off, cnt, static_cast<float *>(z_buf.p) + size_t(off) * kP1 * kC1, st,
                                d_err);
        }
        if (rc != BCTS_OK) {
          rc = fail(rc, "conv1 partial launch failed");
          break;
        }
        zmap = static_cast<const float *>(z_buf.p);
      }
      if ((rc = eval_nodes(cur, N[d_], nullptr, static_cast<float *>(leafmax_buf.p), st, nullptr, zmap,
                           uint32_t(A_))) != BCTS_OK)
        break;
      leafR = curR;
      leafMax = static_cast<float *>(leafmax_buf.p);
      }
    }
    // a6: backup
    double gd = 1.0;
    for (int i = 0; i < d_; ++i) gd *= double(gamma);
    int64_t seg = 1;
    for (int i = 1; i < d_; ++i) seg *= A_;
    if ((rc = launch_segment_max(leafR, leafMax, int64_t(n) * A_, seg, float(gd), V, st)) != BCTS_OK) {
      rc = fail(rc, "backup launch failed");
      break;
    }
    if ((rc = launch_finalize(q0, maxq1, r1, V, n, A_, d_, A_stride, gamma, float(gd), corr, d_action, d_values,
                              st, 0, exact_gev ? 1 : 0)) != BCTS_OK) {
      rc = fail(rc, "finalize launch failed");
      break;
    }
    if (tree_R && tree_V && (rc = export_tree(N, A_, d_, leafMax, st)) != BCTS_OK) break;
  } while (0);
  A = saved_A;
  return rc;
}

Ctx::~Ctx() {
  if (stream) cudaStreamSynchronize(stream);
  for (DevBuf &b : lvlfr_buf)
    if (b.p) cudaFree(b.p);
  DevBuf *bufs[] = {&rootfr_buf, &frames_buf, &scratch_buf, &q0_buf, &maxq1_buf, &V_buf, &r1_buf, &leafmax_buf,
                    &lvl_buf[0], &lvl_buf[1], &R_buf[0], &R_buf[1], &io_roots, &io_action, &io_values,
                    &simt_w, &mixed_buf, &z_buf, &pr_cand, &pr_candR, &pr_candQ, &pr_par, &pr_parR, &pr_idx};
  for (DevBuf *b : bufs)
    if (b->p) cudaFree(b->p);
  for (auto &kv : sgraphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  if (host_stage.p) cudaFreeHost(host_stage.p);
  if (d_err) cudaFree(d_err);
  if (mixed) mixed_destroy(mixed);
  if (tc && owns_weights) tc_weights_destroy(tc);
  if (tc_ref && owns_weights) tc_weights_destroy(tc_ref);
  if (prof) profiler_destroy(prof);
  if (stream) cudaStreamDestroy(stream);
}

}  // namespace bcts

using bcts::Ctx;

namespace bcts {
// FP8 activation scales: run the plain FP32 network on a fixed calibration set
// (512 states from an internal Knuth MMIX LCG, each advanced three ticks so the
// history slots differ) and map each output map's largest value to 448, the
// largest normal E4M3 number.
static int calibrate_fp8(Ctx *c, float act_scale[3], std::string &err) {
  const int n = 512;
  std::vector<bcts_state> hs(n);
  uint64_t x = 0x2545F4914F6CDD1Dull;
  auto next = [&]() {
    x = x * 6364136223846793005ull + 1442695040888963407ull;
    return uint32_t(x >> 33);
  };
  for (int i = 0; i < n; ++i) {
    bcts_state s{};
    for (int k = 0; k < kObj; ++k)
      for (int hh = 0; hh < kHist; ++hh) {
        if (hh == 0) {
          s.pos[0][k][0] = int16_t(next() % kGrid);
          s.pos[0][k][1] = int16_t(next() % kGrid);
        } else {
          s.pos[hh][k][0] = s.pos[0][k][0];
          s.pos[hh][k][1] = s.pos[0][k][1];
        }
      }
    for (int k = 1; k < kObj; ++k) {
      s.vel[k][0] = int8_t(int(next() % 3) - 1);
      s.vel[k][1] = int8_t(int(next() % 3) - 1);
    }
    s.tick = next() & 0xFFFF;
    for (int t = 0; t < 3; ++t) {
      bcts_state nx;
      bcts_env_step(&s, int(next() % kMaxA), &nx, nullptr);
      s = nx;
    }
    hs[i] = s;
  }
  void *d_states = nullptr, *d_frames = nullptr, *d_scratch = nullptr, *d_q = nullptr;
  const size_t scratch_b = simt_scratch_bytes(n);
  int rc = BCTS_OK;
  std::vector<float> maps(size_t(n) * (kP1 * kC1 + kP2 * kC2 + kP3 * kC3));
  if (cudaMalloc(&d_states, size_t(n) * kStateBytes) != cudaSuccess ||
      cudaMalloc(&d_frames, size_t(n) * kFrameBytes) != cudaSuccess || cudaMalloc(&d_scratch, scratch_b) != cudaSuccess ||
      cudaMalloc(&d_q, size_t(n) * c->A_create * 4) != cudaSuccess) {
    rc = BCTS_ENOMEM;
    err = "calibration allocation failed";
  }
  if (rc == BCTS_OK && (cudaMemcpy(d_states, hs.data(), size_t(n) * kStateBytes, cudaMemcpyHostToDevice) != cudaSuccess ||
                        launch_render(static_cast<bcts_state *>(d_states), n, static_cast<uint8_t *>(d_frames), 0) !=
                            BCTS_OK ||
                        simt_qnet_forward(c->simt, static_cast<uint8_t *>(d_frames), n, static_cast<float *>(d_q),
                                          nullptr, d_scratch, 0) != BCTS_OK ||
                        cudaMemcpy(maps.data(), d_scratch, maps.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)) {
    rc = BCTS_ECUDA;
    err = "calibration run failed";
  }
  cudaGetLastError();
  if (d_states) cudaFree(d_states);
  if (d_frames) cudaFree(d_frames);
  if (d_scratch) cudaFree(d_scratch);
  if (d_q) cudaFree(d_q);
  if (rc != BCTS_OK) return rc;
  const size_t len[3] = {size_t(n) * kP1 * kC1, size_t(n) * kP2 * kC2, size_t(n) * kP3 * kC3};
  size_t o = 0;
  for (int l = 0; l < 3; ++l) {
    float mx = 0.f;
    for (size_t i = 0; i < len[l]; ++i) mx = std::max(mx, maps[o + i]);
    o += len[l];
    act_scale[l] = mx > 0.f ? mx / 448.f : 1.f;
  }
  return BCTS_OK;
}
}  // namespace bcts

extern "C" size_t bcts_qnet_numel(int A) {
  if (A < 1) return 0;
  return size_t(32) * 256 + 32 + size_t(64) * 512 + 64 + size_t(64) * 576 + 64 + size_t(512) * 3136 + 512 +
         size_t(A) * 512 + A;
}

extern "C" int bcts_create(const bcts_env_desc *env, const float *w, int A, int d, float gamma, float correction,
                           const bcts_options *opt, bcts_ctx **out) {
  using namespace bcts;
  if (!out || !w || A < 1 || A > kMaxA || d < 0 || d > kMaxDepth || !(gamma > 0.f && gamma <= 1.f) ||
      !std::isfinite(correction) || (env && env->kind != 0)) {
    set_thread_error("bcts_create: invalid argument");
    return BCTS_EINVAL;
  }
  *out = nullptr;
  Ctx *c = new Ctx();
  c->prof = profiler_create();
  c->A = c->A_create = A;
  c->d = d;
  c->gamma = gamma;
  c->corr = correction;
  if (opt) c->opt = *opt;
  c->precision = c->opt.precision;
  c->tc_fused_render = (c->opt.flags & BCTS_FLAG_FRAMES) == 0;
  c->exact_gev = (c->opt.flags & BCTS_FLAG_EXACT_GEV) != 0;
  if (const char *cm = std::getenv("BCTS_CONV_KERNELS")) {  // conv2 / conv3 kernel variants, bits as conv_mask
    const int m = std::atoi(cm);
    if (m >= 0 && m <= 31) {
      c->conv_mask = m;
      c->conv_mask_fixed = true;
    }
  }
  if (c->precision < BCTS_PREC_FP32 || c->precision > BCTS_PREC_FP32_SIMT) {
    delete c;
    set_thread_error("bcts_create: unknown precision");
    return BCTS_EINVAL;
  }
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    set_thread_error("bcts_create: no usable CUDA device");
    return BCTS_ECUDA;
  }
  {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) c->dev_mem = tot;
    cudaGetLastError();
  }
  if (cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess || cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    set_thread_error("bcts_create: device allocation failed");
    return BCTS_ENOMEM;
  }
  // Plain FP32 weights in the CUDA-core kernels' layouts.
  const size_t nw = bcts_qnet_numel(A);
  std::vector<float> hw(nw);
  const float *c1w = w, *c1b = c1w + 32 * 256, *c2w = c1b + 32, *c2b = c2w + 64 * 512, *c3w = c2b + 64,
              *c3b = c3w + 64 * 576, *f1w = c3b + 64, *f1b = f1w + size_t(512) * 3136, *f2w = f1b + 512,
              *f2b = f2w + size_t(A) * 512;
  float *o = hw.data();
  for (int i = 0; i < 32 * 256; ++i) o[i] = float(double(c1w[i]) / 255.0);
  o += 32 * 256;
  std::memcpy(o, c1b, 32 * sizeof(float));
  o += 32;
  for (int oc = 0; oc < 64; ++oc)
    for (int c = 0; c < 32; ++c)
      for (int ky = 0; ky < 4; ++ky)
        for (int kx = 0; kx < 4; ++kx) o[oc * 512 + (ky * 4 + kx) * 32 + c] = c2w[((oc * 32 + c) * 4 + ky) * 4 + kx];
  o += 64 * 512;
  std::memcpy(o, c2b, 64 * sizeof(float));
  o += 64;
  for (int oc = 0; oc < 64; ++oc)
    for (int c = 0; c < 64; ++c)
      for (int ky = 0; ky < 3; ++ky)
        for (int kx = 0; kx < 3; ++kx) o[oc * 576 + (ky * 3 + kx) * 64 + c] = c3w[((oc * 64 + c) * 3 + ky) * 3 + kx];
  o += 64 * 576;
  std::memcpy(o, c3b, 64 * sizeof(float));
  o += 64;
  for (int oc = 0; oc < 512; ++oc)
    for (int c = 0; c < 64; ++c)
      for (int p = 0; p < 49; ++p) o[size_t(oc) * 3136 + p * 64 + c] = f1w[size_t(oc) * 3136 + c * 49 + p];
  o += size_t(512) * 3136;
  std::memcpy(o, f1b, 512 * sizeof(float));
  o += 512;
  std::memcpy(o, f2w, size_t(A) * 512 * sizeof(float));
  o += size_t(A) * 512;
  std::memcpy(o, f2b, A * sizeof(float));
  if (c->ensure(c->simt_w, nw * sizeof(float)) != BCTS_OK ||
      cudaMemcpy(c->simt_w.p, hw.data(), nw * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    set_thread_error("bcts_create: weight upload failed");
    return BCTS_ENOMEM;
  }
  const float *b = static_cast<const float *>(c->simt_w.p);
  c->simt.c1w = b;
  c->simt.c1b = b + 32 * 256;
  c->simt.c2w = c->simt.c1b + 32;
  c->simt.c2b = c->simt.c2w + 64 * 512;
  c->simt.c3w = c->simt.c2b + 64;
  c->simt.c3b = c->simt.c3w + 64 * 576;
  c->simt.f1w = c->simt.c3b + 64;
  c->simt.f1b = c->simt.f1w + size_t(512) * 3136;
  c->simt.f2w = c->simt.f1b + 512;
  c->simt.f2b = c->simt.f2w + size_t(A) * 512;
  c->simt.A = A;
  if (c->precision != BCTS_PREC_FP32_SIMT) {
    std::string e;
    float act_scale[3] = {1.f, 1.f, 1.f};
    int rc = BCTS_OK;
    if (c->precision == BCTS_PREC_FP8) rc = calibrate_fp8(c, act_scale, e);
    if (rc == BCTS_OK)
      rc = tc_weights_create(hw.data(), A, c->precision, c->precision == BCTS_PREC_FP8 ? act_scale : nullptr,
                             &c->tc, e);
    if (rc == BCTS_OK && c->precision != BCTS_PREC_FP32)
      rc = tc_weights_create(hw.data(), A, BCTS_PREC_FP32, nullptr, &c->tc_ref, e);
    if (rc != BCTS_OK) {
      delete c;
      set_thread_error("bcts_create: " + e);
      return rc;
    }
  }
  *out = reinterpret_cast<bcts_ctx *>(c);
  return BCTS_OK;
}

extern "C" void bcts_destroy(bcts_ctx *ctx) {
  if (!ctx) return;
  bcts::serve_shutdown(reinterpret_cast<Ctx *>(ctx));
  delete reinterpret_cast<Ctx *>(ctx);
}

extern "C" const char *bcts_last_error(const bcts_ctx *ctx) {
  if (!ctx) return bcts::thread_error();
  return reinterpret_cast<const Ctx *>(ctx)->err.c_str();
}

extern "C" int bcts_search_device(bcts_ctx *ctx, const bcts_state *d_roots, int n, int32_t *d_action,
                                  float *d_values, void *stream) {
  if (!ctx) return BCTS_EINVAL;
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (n < 0 || (n > 0 && (!d_roots || !d_action || !d_values)))
    return c->fail(BCTS_EINVAL, "bcts_search_device: invalid argument");
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  if (n == 0) return BCTS_OK;
  return c->run_graphed({uintptr_t(n), reinterpret_cast<uintptr_t>(d_roots), reinterpret_cast<uintptr_t>(d_action),
                         reinterpret_cast<uintptr_t>(d_values), reinterpret_cast<uintptr_t>(st)},
                        st, [&] { return c->run_search(d_roots, n, c->A_create, c->d, d_action, d_values, c->A_create, st); });
}

extern "C" int bcts_backup(const float *d_leaf_R, const float *d_leaf_maxq, const float *d_q0, const float *d_r1,
                           const float *d_maxq1, int n, int A, int d, float gamma, float correction, int flags,
                           int32_t *d_action, float *d_values, void *stream) {
  using namespace bcts;
  if (n < 0 || A < 1 || A > 32 || d < 0 || d > 16 || !(gamma > 0.f && gamma <= 1.f) || !std::isfinite(correction) ||
      (flags & ~BCTS_FLAG_EXACT_GEV) != 0) {
    set_thread_error("bcts_backup: invalid argument");
    return BCTS_EINVAL;
  }
  if (n == 0) return BCTS_OK;
  if (!d_q0 || !d_action || !d_values || (d >= 1 && (!d_leaf_R || !d_leaf_maxq || !d_r1 || !d_maxq1))) {
    set_thread_error("bcts_backup: missing pointer");
    return BCTS_EINVAL;
  }
  int64_t seg = 1;
  for (int i = 1; i < d; ++i) {
    if (seg > (int64_t(1) << 40) / A) {
      set_thread_error("bcts_backup: more than 2^40 leaves per root action");
      return BCTS_EINVAL;
    }
    seg *= A;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double gd = 1.0;
  for (int i = 0; i < d; ++i) gd *= double(gamma);
  int rc;
  if (d >= 1) {
    // the segment maxima go to d_values (n * A floats of storage), which finalize
    // then overwrites in place with the corrected values
    if ((rc = launch_segment_max(d_leaf_R, d_leaf_maxq, int64_t(n) * A, seg, float(gd), d_values, st)) != BCTS_OK) {
      set_thread_error("bcts_backup: segment max launch failed");
      return rc;
    }
  }
  if ((rc = launch_finalize(d_q0, d_maxq1, d_r1, d_values, n, A, d, A, gamma, float(gd), correction, d_action,
                            d_values, st, 0, (flags & BCTS_FLAG_EXACT_GEV) ? 1 : 0)) != BCTS_OK) {
    set_thread_error("bcts_backup: finalize launch failed");
    return rc;
  }
  return BCTS_OK;
}

extern "C" int64_t bcts_tree_nodes(int n, int A, int d) {
  if (n < 0 || A < 1 || d < 0) return -1;
  int64_t total = 0, level = n;
  for (int i = 1; i <= d; ++i) {
    if (level > (int64_t(1) << 40) / A) return -1;
    level *= A;
    total += level;
  }
  return total;
}

extern "C" int bcts_search_tree(bcts_ctx *ctx, const bcts_state *d_roots, int n, int32_t *d_action,
                                float *d_values, float *d_node_R, float *d_node_V, void *stream) {
  if (!ctx) return BCTS_EINVAL;
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (n < 0 || (n > 0 && (!d_roots || !d_action || !d_values || (c->d >= 1 && (!d_node_R || !d_node_V)))))
    return c->fail(BCTS_EINVAL, "bcts_search_tree: invalid argument");
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  c->tree_R = d_node_R;
  c->tree_V = d_node_V;
  const int rc = c->run_search(d_roots, n, c->A_create, c->d, d_action, d_values, c->A_create, st);
  c->tree_R = c->tree_V = nullptr;
  return rc;
}

extern "C" int bcts_search(bcts_ctx *ctx, const bcts_state *roots, int n, int32_t *out_action, float *out_values) {
  if (!ctx) return BCTS_EINVAL;
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (n < 0 || (n > 0 && (!roots || !out_action || !out_values)))
    return c->fail(BCTS_EINVAL, "bcts_search: invalid argument");
  if (n == 0) return BCTS_OK;
  return c->search_host(roots, n, nullptr, nullptr, out_action, out_values);
}

namespace bcts {

// Host-pointer search: stage through pinned memory, run, copy back, check the
// device error word, synchronise.  With depths/actions set, roots are grouped by
// (A, d) (the batched form); otherwise all use the context's A and d.
// A plain search that ran eagerly before under the same key, with unchanged
// buffers, is captured into a CUDA graph and replayed from then on: small
// searches are bound by their launches.  Profiling runs eagerly (it records
// events); a stream that cannot be captured (the legacy stream, or one the
// caller is capturing) runs eagerly too.
int Ctx::run_graphed(const GraphKey &key, cudaStream_t st, const std::function<int()> &enqueue) {
  if (profiler_on(prof)) return enqueue();
  {
    SearchGraph &g = sgraphs[key];
    if (g.exec && g.generation == buf_generation) {
      BCTS_CUDA_TRY(cudaGraphLaunch(g.exec, st), err);
      profiler_add(prof, g.launches);
      return BCTS_OK;
    }
    if (g.calls >= 1 && g.last_generation == buf_generation) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
      const int64_t before = profiler_total(prof);
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        cudaGraph_t graph = nullptr;
        const int rc = enqueue();
        const cudaError_t ce = cudaStreamEndCapture(st, &graph);
        const bool ok = rc == BCTS_OK && ce == cudaSuccess && graph &&
                        cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (rc != BCTS_OK) return rc;
        if (ok) {
          g.generation = buf_generation;
          g.launches = profiler_total(prof) - before;
          BCTS_CUDA_TRY(cudaGraphLaunch(g.exec, st), err);
          return BCTS_OK;
        }
        g.exec = nullptr;
      } else {
        cudaGetLastError();
      }
    }
  }
  const int rc = enqueue();
  if (rc != BCTS_OK) return rc;
  if (sgraphs.size() > 32) {  // keep a few keys only
    for (auto it = sgraphs.begin(); it != sgraphs.end();) {
      if (it->first != key) {
        if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
        it = sgraphs.erase(it);
      } else {
        ++it;
      }
    }
  }
  SearchGraph &g = sgraphs[key];
  ++g.calls;
  g.last_generation = buf_generation;
  return BCTS_OK;
}

int Ctx::search_host(const bcts_state *roots, int n, const int32_t *depths, const int32_t *actions,
                     int32_t *out_action, float *out_values) {
  const int As = A_create;
  int rc;
  const size_t in_b = size_t(n) * kStateBytes, act_b = size_t(n) * 4, val_b = size_t(n) * As * 4;
  if ((rc = ensure(io_roots, in_b)) != BCTS_OK) return rc;
  if ((rc = ensure(io_action, act_b)) != BCTS_OK) return rc;
  if ((rc = ensure(io_values, val_b)) != BCTS_OK) return rc;
  if ((rc = ensure_host(host_stage, in_b + act_b + val_b + 64)) != BCTS_OK) return rc;
  char *hs = static_cast<char *>(host_stage.p);
  std::memcpy(hs, roots, in_b);
  const bcts_state *dr = static_cast<const bcts_state *>(io_roots.p);
  int32_t *da = static_cast<int32_t *>(io_action.p);
  float *dv = static_cast<float *>(io_values.p);
  int *herr = reinterpret_cast<int *>(hs + in_b + act_b + val_b);
  (void)actions;
  // copies in, the whole search, copies out: one stream-ordered pass (capturable)
  auto enqueue = [&]() -> int {
    BCTS_CUDA_TRY(cudaMemcpyAsync(io_roots.p, hs, in_b, cudaMemcpyHostToDevice, stream), err);
    const int r = run_search(dr, n, As, d, da, dv, As, stream);
    if (r != BCTS_OK) return r;
    BCTS_CUDA_TRY(cudaMemcpyAsync(hs + in_b, da, act_b, cudaMemcpyDeviceToHost, stream), err);
    BCTS_CUDA_TRY(cudaMemcpyAsync(hs + in_b + act_b, dv, val_b, cudaMemcpyDeviceToHost, stream), err);
    BCTS_CUDA_TRY(cudaMemcpyAsync(herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, stream), err);
    return BCTS_OK;
  };
  if (!depths && prune_keep == 0 && !tree_R) {
    rc = run_graphed({uintptr_t(n), 0, 0, 0, reinterpret_cast<uintptr_t>(stream)}, stream, enqueue);
  } else {
    rc = enqueue();
  }
  if (rc != BCTS_OK) {
    cudaStreamSynchronize(stream);
    return rc;
  }
  BCTS_CUDA_TRY(cudaStreamSynchronize(stream), err);
  if (*herr != 0) {
    cudaMemsetAsync(d_err, 0, sizeof(int), stream);
    cudaStreamSynchronize(stream);
    return fail(BCTS_EDEVICE, "a kernel reported error code " + std::to_string(*herr));
  }
  std::memcpy(out_action, hs + in_b, act_b);
  std::memcpy(out_values, hs + in_b + act_b, val_b);
  return BCTS_OK;
}

}  // namespace bcts

extern "C" int bcts_qnet(bcts_ctx *ctx, const uint8_t *d_frames, int64_t n, float *d_q, void *stream) {
  if (!ctx) return BCTS_EINVAL;
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (n < 0 || (n > 0 && (!d_frames || !d_q))) return c->fail(BCTS_EINVAL, "bcts_qnet: invalid argument");
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  bcts::ProfilerGuard pg(c->prof);
  const int64_t chunk = c->chunk_nodes(n);
  for (int64_t off = 0; off < n; off += chunk) {
    const int64_t cnt = n - off < chunk ? n - off : chunk;
    const int rc =
        c->qnet_nodes(nullptr, d_frames + off * bcts::kFrameBytes, cnt, d_q + off * c->A_create, nullptr, st);
    if (rc != BCTS_OK) return rc;
  }
  return BCTS_OK;
}
