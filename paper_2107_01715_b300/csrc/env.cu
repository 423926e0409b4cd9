// env.cu -- the simulator and the renderer of Alg. 1 on the GPU.
//
//   expand_kernel : Alg. 1's loop body for one depth: every child c = p * A + a of
//                   every frontier parent p is produced at once (replicate state
//                   and reward A times, advance the simulator with action a,
//                   R += gamma^i r).  One thread per child; integer arithmetic only.
//   render_kernel : the 4 x 84 x 84 uint8 frame stack of a state (Sec. 5 frame
//                   stacking), one block per history slot, one thread per 16
//                   output bytes, 16-byte stores.
//
// The sprite environment (agent + reward + two hazards on a 21 x 21 grid) is the
// stand-in for the Atari emulator the paper runs on the GPU (Sec. 4).
#include <cstdio>

#include "common.cuh"
#include "kernels.cuh"
#include "render.cuh"

namespace bcts {

namespace {

// Action direction table (noop, up, right, left, down, up-right, up-left,
// down-right, down-left), packed 2 bits per entry as (delta + 1) so that a warp
// holding many different actions reads it from a register, not a table.
constexpr int kDX[9] = {0, 0, 1, -1, 0, 1, -1, 1, -1};
constexpr int kDY[9] = {0, -1, 0, 0, 1, -1, -1, 1, 1};
constexpr uint32_t pack_dirs(const int (&v)[9]) {
  uint32_t p = 0;
  for (int i = 0; i < 9; ++i) p |= uint32_t(v[i] + 1) << (2 * i);
  return p;
}
constexpr uint32_t kDXP = pack_dirs(kDX);
constexpr uint32_t kDYP = pack_dirs(kDY);

union StateRegs {
  uint4 v[5];
  bcts_state s;
};

__host__ __device__ __forceinline__ uint32_t lowbias32(uint32_t x) {
  // C. Wellons' lowbias32 integer hash.
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

__host__ __device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__host__ __device__ __forceinline__ void bounce(int &p, int &v) {
  int q = p + v;
  if (q < 0) {
    q = -q;
    v = -v;
  }
  if (q > kGrid - 1) {
    q = 2 * (kGrid - 1) - q;
    v = -v;
  }
  p = q;
}

// One tick: agent moves by the action and clamps, objects move and reflect,
// contact (same cell) pays +1 / -1 and respawns the object at a hashed cell;
// the history slots shift by one.  Returns the reward clipped to [-1, 1].
__host__ __device__ __forceinline__ int sprite_step(const bcts_state &s, int a, bcts_state &n) {
  const int dir = a % 9, speed = 1 + a / 9;
  const int dx = int((kDXP >> (2 * dir)) & 3u) - 1;
  const int dy = int((kDYP >> (2 * dir)) & 3u) - 1;
  const int ax = clampi(s.pos[3][0][0] + speed * dx, 0, kGrid - 1);
  const int ay = clampi(s.pos[3][0][1] + speed * dy, 0, kGrid - 1);
#pragma unroll
  for (int h = 0; h < kHist - 1; ++h)
#pragma unroll
    for (int k = 0; k < kObj; ++k) {
      n.pos[h][k][0] = s.pos[h + 1][k][0];
      n.pos[h][k][1] = s.pos[h + 1][k][1];
    }
  n.pos[3][0][0] = (int16_t)ax;
  n.pos[3][0][1] = (int16_t)ay;
  n.vel[0][0] = s.vel[0][0];
  n.vel[0][1] = s.vel[0][1];
  int reward = 0;
#pragma unroll
  for (int k = 1; k < kObj; ++k) {
    int x = s.pos[3][k][0], y = s.pos[3][k][1];
    int vx = s.vel[k][0], vy = s.vel[k][1];
    bounce(x, vx);
    bounce(y, vy);
    if (x == ax && y == ay) {
      reward += (k == 1) ? 1 : -1;
      const uint32_t key = s.tick * 0x9E3779B1u + uint32_t(k) * 0x85EBCA77u +
                           uint32_t(ax * kGrid + ay) * 0xC2B2AE3Du;
      const uint32_t hsh = lowbias32(key);
      x = int(hsh % kGrid);
      y = int((hsh >> 16) % kGrid);
    }
    n.pos[3][k][0] = (int16_t)x;
    n.pos[3][k][1] = (int16_t)y;
    n.vel[k][0] = (int8_t)vx;
    n.vel[k][1] = (int8_t)vy;
  }
  n.tick = s.tick + 1u;
  n.pad = 0u;
  return clampi(reward, -1, 1);
}

constexpr int kExpandThreads = 256;

// Children c0 .. c0 + 255 of one level (one block): the block's children pass
// through shared memory, so that their 80-byte states leave as whole consecutive
// 16-byte chunks (a thread's own five stores would each touch 32 scattered half
// sectors).
__device__ __forceinline__ void expand_block(const uint4 *__restrict__ parents, const float *__restrict__ parent_R,
                                             uint32_t n_child, int A, float gamma_pow, uint4 *__restrict__ children,
                                             float *__restrict__ child_R, int8_t *__restrict__ child_reward,
                                             uint32_t c0, uint4 *stage) {
  const uint32_t c = c0 + threadIdx.x;
  if (c < n_child) {
    const uint32_t p = c / uint32_t(A);
    const int a = int(c - p * uint32_t(A));
    StateRegs in, out;
#pragma unroll
    for (int i = 0; i < 5; ++i) in.v[i] = __ldg(parents + size_t(p) * 5 + i);
    const int r = sprite_step(in.s, a, out.s);
#pragma unroll
    for (int i = 0; i < 5; ++i) stage[threadIdx.x * 5 + i] = out.v[i];
    if (child_R) {
      const float base = parent_R ? __ldg(parent_R + p) : 0.0f;
      child_R[c] = base + gamma_pow * float(r);
    }
    if (child_reward) child_reward[c] = (int8_t)r;
  }
  __syncthreads();
  const uint32_t nb = n_child - c0 < uint32_t(kExpandThreads) ? n_child - c0 : uint32_t(kExpandThreads);
  for (uint32_t i = threadIdx.x; i < nb * 5; i += kExpandThreads) children[size_t(c0) * 5 + i] = stage[i];
}

__global__ void __launch_bounds__(kExpandThreads) expand_kernel(const uint4 *__restrict__ parents,
                                                                const float *__restrict__ parent_R, uint32_t n_child,
                                                                int A, float gamma_pow, uint4 *__restrict__ children,
                                                                float *__restrict__ child_R,
                                                                int8_t *__restrict__ child_reward) {
  __shared__ uint4 stage[kExpandThreads * 5];
  expand_block(parents, parent_R, n_child, A, gamma_pow, children, child_R, child_reward,
               blockIdx.x * kExpandThreads, stage);
}

// One level of several independent trees (the batched form's (A, d) groups) in
// one launch: group k owns blocks block_end[k - 1] .. block_end[k] - 1.
__global__ void __launch_bounds__(kExpandThreads) expand_list_kernel(const __grid_constant__ ExpandList L) {
  __shared__ uint4 stage[kExpandThreads * 5];
  int k = 0;
  while (k < L.n - 1 && blockIdx.x >= L.block_end[k]) ++k;
  const uint32_t b0 = k ? L.block_end[k - 1] : 0u;
  expand_block(reinterpret_cast<const uint4 *>(L.parents[k]), L.parent_R[k], L.n_child[k], L.A[k], L.gamma_pow[k],
               reinterpret_cast<uint4 *>(L.children[k]), L.child_R[k], nullptr, (blockIdx.x - b0) * kExpandThreads,
               stage);
}

// Frame layout per state: [4 slots][84 rows][21 words]; word (h, y, cx) holds the
// 4 pixels of cell cx in pixel row y.  A 16-byte chunk is 4 consecutive words,
// 441 chunks per slot.  One block per (state, slot): a thread's chunk position is
// the same in every slot it renders, and the slot's four object cells are one
// 16-byte load that all threads share.
constexpr uint32_t kChunksPerSlot = kPix * kPix / 16;  // 441
constexpr int kRenderThreads = 448;                    // >= 441, whole warps

// Frames are background except the sprite rows: each object is 4 rows of one
// 4-pixel word (word index = pixel row * 21 + cell column).  A block renders a
// group of kRenderGroup slots: every thread writes its 16-byte background chunk
// of each slot, then, after a barrier, one thread per (slot, object, sprite row)
// writes that word as the renderer paints it (render_word: all objects in the
// cell, in index order, so objects sharing a cell give every writer the same
// value).  The barrier orders the word stores after the block's chunk stores;
// the next group writes other slots.
constexpr int kRenderGroup = 8;

__device__ __forceinline__ void render_group(const uint4 *__restrict__ states, uint64_t b0, uint64_t step,
                                             uint64_t n, bool newest, uint4 *__restrict__ frames) {
  const uint32_t jc = threadIdx.x;
  // the word writers' object cells, loaded before the background stores so that the
  // load latency overlaps them
  const int k = int(jc >> 4), obj = int(jc >> 2) & 3, r = int(jc & 3);
  const uint64_t bw = b0 + k * step;
  const bool writer = jc < kRenderGroup * 16 && bw < n;  // (slot, object, sprite row)
  uint4 P = make_uint4(0u, 0u, 0u, 0u);
  if (writer) P = __ldg(newest ? states + bw * 5 + 3 : states + (bw >> 2) * 5 + (bw & 3));
  if (jc < kChunksPerSlot) {
#pragma unroll
    for (int g = 0; g < kRenderGroup; ++g) {
      const uint64_t b = b0 + g * step;
      if (b < n) frames[b * kChunksPerSlot + jc] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  __syncthreads();
  if (writer) {
    const uint64_t b = bw;
    {
      int ox[4], oy[4];
      unpack_slot(P, ox, oy);
      const int y = 4 * oy[obj] + r, cx = ox[obj];
      reinterpret_cast<uint32_t *>(frames + b * kChunksPerSlot)[y * kGrid + cx] = render_word(ox, oy, cx, y);
    }
  }
}

// All four history slots: block-strided over (state, slot) pairs b = state * 4 + slot.
__global__ void __launch_bounds__(kRenderThreads) render_kernel(const uint4 *__restrict__ states, uint64_t n_slots,
                                                                uint4 *__restrict__ frames) {
  const uint64_t step = gridDim.x;
  for (uint64_t b0 = blockIdx.x; b0 < n_slots; b0 += kRenderGroup * step)
    render_group(states, b0, step, n_slots, false, frames);
}

// The newest history slot of each state only: frames [n][84][84], one per
// state.  In a search every expanded node's stack is its own newest frame plus
// its ancestors' (frame stacking, Sec. 5; Alg. 1's parent of x is x / A), so
// each node's frame is rendered once, when its level is expanded.
__global__ void __launch_bounds__(kRenderThreads) render_newest_kernel(const uint4 *__restrict__ states, uint64_t n,
                                                                       uint4 *__restrict__ frames) {
  const uint64_t step = gridDim.x;
  for (uint64_t b0 = blockIdx.x; b0 < n; b0 += kRenderGroup * step)
    render_group(states, b0, step, n, true, frames);
}

}  // namespace

int launch_render_newest(const bcts_state *states, int64_t n, uint8_t *frames, cudaStream_t stream) {
  if (n <= 0) return BCTS_OK;
  int sms = 148;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t cap = uint64_t(sms) * 4 * 2;  // two waves of four blocks per SM, each striding over states
  const unsigned blocks = unsigned(uint64_t(n) < cap ? uint64_t(n) : cap);
  ProfScope ps(K_RENDER, stream);
  render_newest_kernel<<<blocks, kRenderThreads, 0, stream>>>(reinterpret_cast<const uint4 *>(states), uint64_t(n),
                                                              reinterpret_cast<uint4 *>(frames));
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

int launch_expand_list(const ExpandList &L, cudaStream_t stream) {
  if (L.n <= 0) return BCTS_OK;
  const uint32_t blocks = L.block_end[L.n - 1];
  if (blocks == 0) return BCTS_OK;
  ProfScope ps(K_EXPAND, stream);
  expand_list_kernel<<<blocks, kExpandThreads, 0, stream>>>(L);
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

int launch_expand(const bcts_state *parents, const float *parent_R, int64_t n_parents, int A, float gamma_pow,
                  bcts_state *children, float *child_R, int8_t *child_reward, cudaStream_t stream) {
  const int64_t n_child = n_parents * A;
  if (n_child <= 0) return BCTS_OK;
  if (n_child > 0x7FFFFFFFLL) return BCTS_EINVAL;
  const int threads = 256;
  const unsigned blocks = unsigned((n_child + threads - 1) / threads);
  ProfScope ps(K_EXPAND, stream);
  expand_kernel<<<blocks, threads, 0, stream>>>(reinterpret_cast<const uint4 *>(parents), parent_R,
                                                uint32_t(n_child), A, gamma_pow,
                                                reinterpret_cast<uint4 *>(children), child_R, child_reward);
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

int launch_render(const bcts_state *states, int64_t n, uint8_t *frames, cudaStream_t stream) {
  if (n <= 0) return BCTS_OK;
  const uint64_t n_slots = uint64_t(n) * kHist;
  int sms = 148;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t cap = uint64_t(sms) * 4 * 16;  // four blocks per SM, grid-stride beyond 16 waves
  const unsigned blocks = unsigned(n_slots < cap ? n_slots : cap);
  ProfScope ps(K_RENDER, stream);
  render_kernel<<<blocks, kRenderThreads, 0, stream>>>(reinterpret_cast<const uint4 *>(states), n_slots,
                                                       reinterpret_cast<uint4 *>(frames));
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

}  // namespace bcts

extern "C" int bcts_expand(const bcts_state *d_parents, const float *d_parent_R, int64_t n_parents, int A,
                           float gamma_pow, bcts_state *d_children, float *d_child_R, int8_t *d_child_reward,
                           void *stream) {
  if (!d_parents || !d_children || n_parents < 0 || A < 1 || A > bcts::kMaxA) {
    bcts::set_thread_error("bcts_expand: invalid argument");
    return BCTS_EINVAL;
  }
  const int rc = bcts::launch_expand(d_parents, d_parent_R, n_parents, A, gamma_pow, d_children, d_child_R,
                                     d_child_reward, (cudaStream_t)stream);
  if (rc != BCTS_OK) bcts::set_thread_error("bcts_expand: launch failed");
  return rc;
}

extern "C" int bcts_render(const bcts_state *d_states, int64_t n, uint8_t *d_frames, void *stream) {
  if (!d_states || !d_frames || n < 0) {
    bcts::set_thread_error("bcts_render: invalid argument");
    return BCTS_EINVAL;
  }
  const int rc = bcts::launch_render(d_states, n, d_frames, (cudaStream_t)stream);
  if (rc != BCTS_OK) bcts::set_thread_error("bcts_render: launch failed");
  return rc;
}

// The same step on the host (one state), for callers that advance an episode
// by the chosen action (the serving simulator, tests).
extern "C" int bcts_env_step(const bcts_state *s, int a, bcts_state *out, int *reward) {
  if (!s || !out || a < 0 || a >= bcts::kMaxA) {
    bcts::set_thread_error("bcts_env_step: invalid argument");
    return BCTS_EINVAL;
  }
  bcts_state n;
  const int r = bcts::sprite_step(*s, a, n);
  *out = n;
  if (reward) *reward = r;
  return BCTS_OK;
}
