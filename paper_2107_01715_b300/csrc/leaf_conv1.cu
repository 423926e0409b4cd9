// leaf_conv1.cu -- conv1 of the leaves from their parents' partial maps.
//
// Frame stacking (Sec. 5) makes a child's history slots 0-2 its parent's slots
// 1-3, and conv1 is linear in its input channels, so a leaf's pre-activation is
// its parent's partial map Z = W_0 * slot1 + W_1 * slot2 + W_2 * slot3 + b
// (computed once per parent, by the second pass below) plus the term W_3 * slot3
// of its own newest frame.  That frame holds nothing but the four 4 x 4 sprites, so
// the term is zero outside the (at most 16) 8 x 8 stride-4 patches that cover an
// object's cell, and inside one it is the sum, over the objects in the patch, of
// T[k][dy][dx] = palette_k x (W_3 summed over sprite k's set pixels placed at cell
// offset (dy, dx) of the patch), a 32-channel table built once per context.
// Two objects on one cell overlap (the later one paints over the earlier one's
// pixels, Sec. 5's renderer); such a cell's term is summed from its rendered pixels.
//
// The leaf level is therefore a streaming pass, not a contraction: every output
// row is ReLU(Z) except the few next to an object.  One block takes a 80-row
// slice of the 400 patch rows for 36 consecutive leaves: it reads the slice of
// each parent's map once (siblings are consecutive), writes ReLU(Z) for every
// leaf, then overwrites the rows next to the leaves' objects with ReLU(Z + term).
// Output formats as the tensor-core layers expect them: bf16 (BF16), bf16 hi + lo
// (FP32-class split) or E4M3 scaled by the conv1 map's activation scale (FP8).
//
// The parents' partial maps are formed the same way: Z is b on every row and,
// on the (at most 48) rows next to an object of the parent's slots 1-3, b plus
// those slots' terms with weight channels 0-2.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "pack.cuh"
#include "render.cuh"

namespace bcts {
namespace {

constexpr int kSliceRows = 80;                      // patch rows per block (5 slices of 400)
constexpr int kSlices = kP1 / kSliceRows;
constexpr int kThreads = 160;                       // one float4 of 4 channels x 4 per thread
constexpr int kSliceF4 = kSliceRows * kC1 / 4;      // 640 float4 per slice
constexpr int kF4PerThread = kSliceF4 / kThreads;   // 4
constexpr int kLeaves = 36;                         // leaves per block
constexpr int kCands = 16;                          // (object, dy, dx) per leaf
constexpr int kRowWords = (kSliceRows + 31) / 32;   // per-node bitmap of a slice's listed rows
constexpr int kSlotF4 = kObj * 2 * 2 * (kC1 / 4);   // one weight channel's table as float4s
constexpr int kSlotW = 64 * kC1;                    // one weight channel's [64][32] floats
static_assert(kP1 % kSliceRows == 0 && kSliceF4 % kThreads == 0, "slice geometry");

struct Args {
  const bcts_state *states;
  int64_t n;
  const float *zmap;
  uint32_t leaf0, branch;
  const uint32_t *parent;
  const float *T;
  const float *W3;
  float out_scale;
  void *out_hi, *out_lo;
};

__device__ __forceinline__ uint32_t bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

// Store ReLU(v) for float4 number f of the leaves' row-major maps (4 channels);
// the ReLU is folded into the rounding conversion where no remainder is kept.
template <int MODE>
__device__ __forceinline__ void store_relu(const Args &p, int64_t f, float4 v) {
  if constexpr (MODE == 2) {  // activation scale (positive) then E4M3
    const float2 s = make_float2(p.out_scale, p.out_scale);
    reinterpret_cast<uint32_t *>(p.out_hi)[f] =
        relu_e4m3x4(mul2(make_float2(v.x, v.y), s), mul2(make_float2(v.z, v.w), s));
  } else if constexpr (MODE == 0) {
    reinterpret_cast<uint2 *>(p.out_hi)[f] =
        make_uint2(relu_bf16x2(make_float2(v.x, v.y)), relu_bf16x2(make_float2(v.z, v.w)));
  } else {
    v.x = fmaxf(v.x, 0.f);
    v.y = fmaxf(v.y, 0.f);
    v.z = fmaxf(v.z, 0.f);
    v.w = fmaxf(v.w, 0.f);
    const uint32_t h0 = bf16x2(v.x, v.y), h1 = bf16x2(v.z, v.w);
    reinterpret_cast<uint2 *>(p.out_hi)[f] = make_uint2(h0, h1);
    // remainder below the bf16 rounding, exact in FP32
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&h0));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&h1));
    reinterpret_cast<uint2 *>(p.out_lo)[f] = make_uint2(bf16x2(v.x - a.x, v.y - a.y), bf16x2(v.z - b.x, v.w - b.y));
  }
}

__device__ __forceinline__ void add4(float4 &a, const float4 b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
  a.w += b.w;
}

// The newest frame's term for patch (ox, oy), channels 4 c4 .. 4 c4 + 3.
// cx/cy: the leaf's object cells in its newest slot.
__device__ float4 patch_term(const int (&cx)[kObj], const int (&cy)[kObj], int ox, int oy, int c4,
                             const float4 *Ts, const float *__restrict__ W3) {
  float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < kObj; ++k) {
    const int dx = cx[k] - ox, dy = cy[k] - oy;
    if (dx < 0 || dx > 1 || dy < 0 || dy > 1) continue;
    bool lower = false, other = false;  // another object on this cell (lower index / any)
#pragma unroll
    for (int j = 0; j < kObj; ++j) {
      const bool same = j != k && cx[j] == cx[k] && cy[j] == cy[k];
      other |= same;
      lower |= same && j < k;
    }
    if (!other) {
      add4(d, Ts[((k * 2 + dy) * 2 + dx) * 8 + c4]);
    } else if (!lower) {
      // shared cell, taken once by its lowest object: the rendered pixels in
      // paint order (a later object's set sprite bits overwrite)
      for (int sy = 0; sy < 4; ++sy)
        for (int sx = 0; sx < 4; ++sx) {
          uint32_t pix = 0;
#pragma unroll
          for (int j = 0; j < kObj; ++j)
            if (cx[j] == cx[k] && cy[j] == cy[k] && ((kSprites >> (16 * j + 4 * sy + sx)) & 1ull))
              pix = (kPalette >> (8 * j)) & 0xFFu;
          if (pix) {
            const float4 w = reinterpret_cast<const float4 *>(W3)[((4 * dy + sy) * 8 + 4 * dx + sx) * 8 + c4];
            const float pf = float(pix);
            d.x = fmaf(pf, w.x, d.x);
            d.y = fmaf(pf, w.y, d.y);
            d.z = fmaf(pf, w.z, d.z);
            d.w = fmaf(pf, w.w, d.w);
          }
        }
    }
  }
  return d;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) leaf_conv1_kernel(const Args p) {
  __shared__ float4 Ts[kObj * 2 * 2 * 8];
  __shared__ int16_t cells[kLeaves][kObj][2];
  __shared__ uint32_t par[kLeaves];
  __shared__ uint32_t hits[kLeaves * kCands];  // (leaf << 16) | patch row, rows next to an object
  __shared__ int nhits;
  const int t = threadIdx.x;
  const int slice = blockIdx.y;
  const int64_t l0 = int64_t(blockIdx.x) * kLeaves;
  const int nl = p.n - l0 < kLeaves ? int(p.n - l0) : kLeaves;
  for (int i = t; i < kObj * 2 * 2 * 8; i += kThreads) Ts[i] = reinterpret_cast<const float4 *>(p.T)[i];
  for (int i = t; i < nl; i += kThreads) {
    // newest slot's object cells: pos[3][k][x, y], bytes 48..63 of the state
    const uint4 c = reinterpret_cast<const uint4 *>(p.states + l0 + i)[3];
    *reinterpret_cast<uint4 *>(&cells[i][0][0]) = c;
    const uint32_t g = p.leaf0 + uint32_t(l0) + uint32_t(i);
    par[i] = p.parent ? p.parent[g] : g / p.branch;
  }
  if (t == 0) nhits = 0;
  __syncthreads();
  // rows of this slice next to an object of some leaf (duplicates are harmless:
  // they compute and write the same values)
  for (int i = t; i < nl * kCands; i += kThreads) {
    const int j = i / kCands, c = i % kCands, k = c >> 2;
    const int ox = cells[j][k][0] - (c & 1), oy = cells[j][k][1] - ((c >> 1) & 1);
    if (ox < 0 || ox > 19 || oy < 0 || oy > 19) continue;
    const int r = oy * 20 + ox;
    if (r / kSliceRows != slice) continue;
    hits[atomicAdd(&nhits, 1)] = (uint32_t(j) << 16) | uint32_t(r);
  }
  // every row: ReLU(Z), the slice of each parent's map read once
  const float4 *Z = reinterpret_cast<const float4 *>(p.zmap);
  float4 z[kF4PerThread];
  uint32_t cur = 0xFFFFFFFFu;
  for (int j = 0; j < nl; ++j) {
    if (par[j] != cur) {
      cur = par[j];
      const float4 *zs = Z + size_t(cur) * (kP1 * kC1 / 4) + slice * kSliceF4;
#pragma unroll
      for (int i = 0; i < kF4PerThread; ++i) z[i] = __ldg(zs + i * kThreads + t);
    }
    const int64_t fb = (l0 + j) * int64_t(kP1 * kC1 / 4) + slice * kSliceF4;
#pragma unroll
    for (int i = 0; i < kF4PerThread; ++i) store_relu<MODE>(p, fb + i * kThreads + t, z[i]);
  }
  __syncthreads();  // orders the overwrites below after every thread's first write
  const int nh = nhits;
  for (int i = t; i < nh * 8; i += kThreads) {
    const uint32_t h = hits[i >> 3];
    const int c4 = i & 7, j = int(h >> 16), r = int(h & 0xFFFFu);
    int cx[kObj], cy[kObj];
#pragma unroll
    for (int k = 0; k < kObj; ++k) {
      cx[k] = cells[j][k][0];
      cy[k] = cells[j][k][1];
    }
    float4 v = __ldg(Z + size_t(par[j]) * (kP1 * kC1 / 4) + r * 8 + c4);
    add4(v, patch_term(cx, cy, r % 20, r / 20, c4, Ts, p.W3));
    store_relu<MODE>(p, (l0 + j) * int64_t(kP1 * kC1 / 4) + r * 8 + c4, v);
  }
}

// A parent's partial map Z = W_0 * slot1 + W_1 * slot2 + W_2 * slot3 + b, FP32,
// no ReLU; same block layout as the leaves.  T and W hold weight channels 0-2
// first.
__global__ void __launch_bounds__(kThreads) partial_map_kernel(const bcts_state *__restrict__ states, int64_t n,
                                                               const float *__restrict__ T,
                                                               const float *__restrict__ W,
                                                               const float *__restrict__ bias, float *__restrict__ Z) {
  __shared__ float4 Ts[3 * kSlotF4];
  __shared__ __align__(16) int16_t cells[kLeaves][3][kObj][2];  // the parent's slots 1-3: bytes 16..63 of a state
  __shared__ uint32_t listed[kLeaves][kRowWords];
  __shared__ uint32_t hits[kLeaves * 3 * kCands];  // (node << 16) | patch row
  __shared__ int nhits;
  const int t = threadIdx.x;
  const int slice = blockIdx.y;
  const int64_t l0 = int64_t(blockIdx.x) * kLeaves;
  const int nl = n - l0 < kLeaves ? int(n - l0) : kLeaves;
  for (int i = t; i < 3 * kSlotF4; i += kThreads) Ts[i] = __ldg(reinterpret_cast<const float4 *>(T) + i);
  for (int i = t; i < nl * 3; i += kThreads)
    reinterpret_cast<uint4 *>(&cells[0][0][0][0])[i] =
        __ldg(reinterpret_cast<const uint4 *>(states + l0 + i / 3) + 1 + (i % 3));
  for (int i = t; i < kLeaves * kRowWords; i += kThreads) (&listed[0][0])[i] = 0u;
  if (t == 0) nhits = 0;
  __syncthreads();
  // the rows of this slice next to an object of slots 1-3, each listed once
  for (int i = t; i < nl * 3 * kCands; i += kThreads) {
    const int j = i / (3 * kCands), c = i % (3 * kCands), h = c >> 4, k = (c >> 2) & 3;
    const int ox = cells[j][h][k][0] - (c & 1), oy = cells[j][h][k][1] - ((c >> 1) & 1);
    if (ox < 0 || ox > 19 || oy < 0 || oy > 19) continue;
    const int r = oy * 20 + ox - slice * kSliceRows;
    if (r < 0 || r >= kSliceRows) continue;
    const uint32_t bit = 1u << (r & 31);
    if (atomicOr(&listed[j][r >> 5], bit) & bit) continue;
    hits[atomicAdd(&nhits, 1)] = (uint32_t(j) << 16) | uint32_t(r + slice * kSliceRows);
  }
  // every row: b (a thread's four float4s share one channel group)
  float4 *Z4 = reinterpret_cast<float4 *>(Z);
  const float4 b4 = __ldg(reinterpret_cast<const float4 *>(bias) + (t & 7));
  for (int j = 0; j < nl; ++j) {
    const int64_t fb = (l0 + j) * int64_t(kP1 * kC1 / 4) + slice * kSliceF4;
#pragma unroll
    for (int i = 0; i < kF4PerThread; ++i) Z4[fb + i * kThreads + t] = b4;
  }
  __syncthreads();  // orders the overwrites below after every thread's first write
  const int nh = nhits;
  for (int i = t; i < nh * 8; i += kThreads) {
    const uint32_t hv = hits[i >> 3];
    const int c4 = i & 7, j = int(hv >> 16), r = int(hv & 0xFFFFu);
    float4 v = __ldg(reinterpret_cast<const float4 *>(bias) + c4);
#pragma unroll
    for (int h = 0; h < 3; ++h) {
      int cx[kObj], cy[kObj];
#pragma unroll
      for (int k = 0; k < kObj; ++k) {
        cx[k] = cells[j][h][k][0];
        cy[k] = cells[j][h][k][1];
      }
      add4(v, patch_term(cx, cy, r % 20, r / 20, c4, Ts + h * kSlotF4, W + h * kSlotW));
    }
    Z4[(l0 + j) * int64_t(kP1 * kC1 / 4) + r * 8 + c4] = v;
  }
}

}  // namespace

int launch_partial_map(const bcts_state *states, int64_t n, const float *T, const float *W, const float *bias,
                       float *Z, cudaStream_t st) {
  if (n <= 0) return BCTS_OK;
  if (n > 0x7FFFFFFFLL * kLeaves) return BCTS_EINVAL;
  const dim3 grid(unsigned((n + kLeaves - 1) / kLeaves), kSlices);
  ProfScope ps(K_CONV1_PARTIAL, st);
  partial_map_kernel<<<grid, kThreads, 0, st>>>(states, n, T, W, bias, Z);
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

int launch_leaf_conv1(int mode, const bcts_state *states, int64_t n, const ZLeaf &zl, const float *T,
                      const float *W3, float out_scale, void *out_hi, void *out_lo, cudaStream_t st) {
  if (n <= 0) return BCTS_OK;
  if (n > 0x7FFFFFFFLL * kLeaves) return BCTS_EINVAL;
  Args p{states, n, zl.zmap, zl.leaf0, zl.branch, zl.parent, T, W3, out_scale, out_hi, out_lo};
  const dim3 grid(unsigned((n + kLeaves - 1) / kLeaves), kSlices);
  ProfScope ps(K_CONV1_LEAF, st);
  if (mode == 0)
    leaf_conv1_kernel<0><<<grid, kThreads, 0, st>>>(p);
  else if (mode == 1)
    leaf_conv1_kernel<1><<<grid, kThreads, 0, st>>>(p);
  else
    leaf_conv1_kernel<2><<<grid, kThreads, 0, st>>>(p);
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

}  // namespace bcts
