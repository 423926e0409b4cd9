// conv_pair.cu -- conv2 of the leaf Q-network (Nature-DQN) as an implicit GEMM on
// tcgen05 with the weights resident in tensor memory and the pixels as the MMA's
// N dimension: two filter taps per instruction.
//
// conv2 has 64 output channels.  With pixels as M (conv_win.cu, conv_tma.cu) an
// instruction is M = 128 pixels x N = 64 channels, and an N = 64 tcgen05.mma
// takes about 47 cycles where its FLOPs need 32 (measured on B300: M = 128 and
// N >= 128 runs at the full 8,192 FLOP per cycle and SM, N = 64 at two thirds,
// whether A comes from shared or tensor memory).  Here the instruction is
// M = 128 weight rows x N = 128 pixels, the 128 rows being the 64 channels of two
// taps of the 2 x 2 stride-1 filter on the space-to-depth view (conv_win.cuh):
//
//   rows 0-63    W(ky2, 0) . X[r + 10 ky2]      (tap (ky2, 0) of output row r)
//   rows 64-127  W(ky2, 1) . X[r + 10 ky2]      (tap (ky2, 1) of output row r - 1)
//
// for ky2 = 0, 1 into one accumulator.  A column r of the upper half holds tap
// (ky2, 1)'s contribution to output row r - 1 (its input row is r - 1 + 10 ky2 +
// 1), so output row c0 + c of a tile starting at padded row c0 is
//
//   D[co][c] + D[64 + co][c + 1],   c = 0 .. 126,
//
// and tiles advance by 127 rows.  The A operand (the [tap (ky2,0); tap (ky2,1)]
// weight rows, 128 K each) stays in tensor memory for the whole kernel, so shared
// memory holds only input windows and the split mode needs no weight stream; the
// B operand is 128 consecutive rows of the window at the pair's shift, addressed
// by a shared-memory descriptor exactly as the window kernels address their A.
//
// FP32-class split (bf16 hi + lo on both sides): three instructions per K step,
// A_hi.X_hi + A_hi.X_lo + A_lo.X_hi, all at N = 128 (192 cycles per pair and K
// step against 224 for the N = 128 + N = 64 pair of the pixel-major form).
//
// Roles (one CTA per SM, persistent over a contiguous range of tiles):
//   warp 0    one lane issues the TMA window loads (one window per tile);
//   warp 1    allocates all 512 TMEM columns (two 128-column accumulators,
//             the weight rows at columns 256-511) and issues the MMAs;
//   warps 2-5 load the weights into TMEM once (each warp its 32 lanes), then per
//             tile copy the accumulator into a shared-memory staging tile
//             [column][lane] (which frees it for the next tile's MMAs) and finish
//             the output rows from there: eight lanes per row, four channels of
//             each half per lane, bias, ReLU and rounding, and 8-byte stores that
//             eight consecutive lanes make into one NHWC row.  (Finishing the rows
//             straight from the accumulator, one channel per thread, measured 2.5x
//             slower than the conv2 kernels of the pixel-major form: one 2-byte
//             store and the row's index arithmetic per element, in code too large
//             for the instruction cache.)
// Every wait is bounded; on a time-out the kernel records an error code, stops
// issuing, waits for its own copies and MMAs and frees TMEM.
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "conv_win.cuh"
#include "kernels.cuh"
#include "pack.cuh"
#include "tc_ptx.cuh"
#include "tma_host.cuh"

namespace bcts {
namespace tc {
namespace {

__device__ __forceinline__ void mma_ts_bf16(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
      "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]),
      "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]),
      "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}

template <int MODE>
struct PairCfg {
  using G = WinGeo<2>;
  static constexpr bool SPLIT = MODE == 1;
  static constexpr int ROWB = 128;                     // bf16 window row of one slab
  static constexpr int NA = SPLIT ? 2 : 1;             // hi (and lo) maps
  static constexpr int SLAB = (G::WROWS * ROWB + 1023) / 1024 * 1024;
  static constexpr int WIN_BYTES = NA * G::NSLAB * SLAB;
  static constexpr int LOAD_BYTES = NA * G::NSLAB * G::WROWS * ROWB;
  static constexpr int TSTEP = 127;                    // output rows per tile
  static constexpr int SROW = 132;                     // staging row: 128 TMEM lanes + 4 floats to spread the banks
  static constexpr int STG_BYTES = 128 * SROW * 4;      // the accumulator, [128 columns][128 lanes] FP32
  static constexpr int META_BYTES = 1024;
  static constexpr int BUDGET = 232448 - 1024 - META_BYTES - 64 * 4 - STG_BYTES;
  static constexpr int STAGES_RAW = BUDGET / WIN_BYTES;
  static constexpr int STAGES = STAGES_RAW > 4 ? 4 : STAGES_RAW;
  static constexpr int NUM_ACC = 2;
  static constexpr uint32_t ACC_COLS = 128;
  static constexpr uint32_t W_HI_COL = 256, W_LO_COL = 384;  // pair ky2 at + 64 ky2
  static constexpr uint32_t TMEM_COLS = 512;
  static constexpr int THREADS = 32 * 6;
  static constexpr int SMEM = 1024 + STAGES * WIN_BYTES + META_BYTES + 64 * 4 + STG_BYTES;
  static_assert(STAGES >= 2, "window pipeline depth");
  static_assert(SLAB % 1024 == 0, "1024-byte boundaries");
  static_assert(8 * (2 * STAGES + 2 * NUM_ACC + 4) + 8 <= META_BYTES, "barrier area");
  static_assert(SMEM <= 232448, "shared memory");
  // the B operand of pair ky2 at row offset o < 10 of its line: rows o + 10 ky2 .. + 127 < WROWS
  static_assert(9 + 10 + 127 < G::WROWS, "window rows");
};

struct PairParams {
  const __nv_bfloat16 *w_hi, *w_lo;  // [64][kpad], K = (ky, kx, c)
  int kpad;
  const float *bias;
  __nv_bfloat16 *out_hi, *out_lo;    // NHWC [node][81][64]
  uint32_t n;                        // nodes
  int num_tiles;                     // ceil(n * 100 / 127)
  int *d_err;
};

template <int MODE>
__global__ void __launch_bounds__(PairCfg<MODE>::THREADS, 1)
    conv_pair(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapXlo,
              const PairParams p) {
  using C = PairCfg<MODE>;
  using G = WinGeo<2>;
  constexpr int S = C::STAGES, NACC = C::NUM_ACC;
  constexpr bool SPLIT = C::SPLIT;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = smem_raw + (base - raw);
  // layout: [windows][barriers + meta][bias][staging]
  const uint32_t win0 = base;
  const uint32_t bar0 = win0 + S * C::WIN_BYTES;
  auto wfull_bar = [&](int s) { return bar0 + 8u * s; };
  auto wempty_bar = [&](int s) { return bar0 + 8u * (S + s); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * S + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * S + NACC + a); };
  const uint32_t wready_bar = bar0 + 8u * (2 * S + 2 * NACC);
  const uint32_t drain_bar = wready_bar + 8u;
  const uint32_t xfull_bar = drain_bar + 8u;  // the staging tile written by all four epilogue warps
  const uint32_t xfree_bar = xfull_bar + 8u;  // the staging tile read by all four
  uint8_t *meta = gbase + S * C::WIN_BYTES + 8 * (2 * S + 2 * NACC + 4);
  volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(meta);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(meta + 4);
  float *bias_s = reinterpret_cast<float *>(gbase + S * C::WIN_BYTES + C::META_BYTES);
  float *stg = bias_s + 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (p.num_tiles + int(gridDim.x) - 1) / int(gridDim.x);
  const int T0 = int(blockIdx.x) * per;
  const int TE = T0 + per < p.num_tiles ? T0 + per : p.num_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(wfull_bar(s), 1);
      mbar_init(wempty_bar(s), 1);
    }
    for (int a = 0; a < NACC; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), 4);
    }
    mbar_init(wready_bar, 4);
    mbar_init(drain_bar, 1);
    mbar_init(xfull_bar, 4);
    mbar_init(xfree_bar, 4);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32((const void *)tmem_slot), C::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_map(&mapX);
      if (SPLIT) tma_prefetch_map(&mapXlo);
      int gw = 0;
      for (int t = T0; t < TE; ++t, ++gw) {
        const int s = gw % S;
        if (!wait_bar(wempty_bar(s), uint32_t((gw / S) & 1) ^ 1u, abort_flag, p.d_err, 1)) break;
        mbar_arrive_expect_tx(wfull_bar(s), uint32_t(C::LOAD_BYTES));
        const uint32_t w = win0 + uint32_t(s * C::WIN_BYTES);
        const int line = (t * C::TSTEP) / G::PW;  // the window starts at the tile's line of 10
#pragma unroll
        for (int a = 0; a < C::NA; ++a)
#pragma unroll
          for (int sl = 0; sl < G::NSLAB; ++sl)
            tma_load_4d(w + uint32_t((a * G::NSLAB + sl) * C::SLAB),
                        a ? static_cast<const void *>(&mapXlo) : static_cast<const void *>(&mapX), 0, 0, sl, line,
                        wfull_bar(s));
      }
      // teardown: the last fill of every stage has landed
      for (int k = gw - 1; k >= 0 && k >= gw - S; --k)
        wait_bar_drain(wfull_bar(k % S), uint32_t((k / S) & 1), p.d_err);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(128);
      constexpr uint64_t kLoOff = uint64_t(uint32_t(G::NSLAB * C::SLAB) >> 4);  // the lo slabs (split)
      bool ok = wait_bar(wready_bar, 0, abort_flag, p.d_err, 6);
      tc_fence_after();
      int gw = 0, it = 0;
      for (int t = T0; t < TE && ok; ++t, ++it, ++gw) {
        const int acc = it % NACC;
        if (!wait_bar(tempty_bar(acc), uint32_t((it / NACC) & 1) ^ 1u, abort_flag, p.d_err, 2)) break;
        const int s = gw % S;
        if (!wait_bar(wfull_bar(s), uint32_t((gw / S) & 1), abort_flag, p.d_err, 3)) break;
        tc_fence_after();
        const uint32_t d = tmem + uint32_t(acc) * C::ACC_COLS;
        const int row_off = (t * C::TSTEP) % G::PW;  // tile start within its window line
        // one descriptor base per tile; (pair, slab, K step) offsets are constants
        const uint64_t wdesc =
            swz_desc(win0 + uint32_t(s * C::WIN_BYTES), C::ROWB) + uint64_t(uint32_t(row_off * C::ROWB) >> 4);
#pragma unroll
        for (int ky2 = 0; ky2 < 2; ++ky2)
#pragma unroll
          for (int sl = 0; sl < G::NSLAB; ++sl)
#pragma unroll
            for (int kk = 0; kk < C::ROWB / 32; ++kk) {
              const uint64_t b =
                  wdesc + uint64_t(uint32_t(sl * C::SLAB + ky2 * G::PW * C::ROWB) >> 4) + uint64_t(2 * kk);
              const uint32_t kcol = uint32_t(64 * ky2 + 32 * sl + 8 * kk);
              const uint32_t first = (ky2 == 0 && sl == 0 && kk == 0) ? 0u : 1u;
              mma_ts_bf16(d, tmem + C::W_HI_COL + kcol, b, idesc, first);
              if constexpr (SPLIT) {
                mma_ts_bf16(d, tmem + C::W_HI_COL + kcol, b + kLoOff, idesc, 1u);  // A_hi . X_lo
                mma_ts_bf16(d, tmem + C::W_LO_COL + kcol, b, idesc, 1u);           // A_lo . X_hi
              }
            }
        mma_commit(wempty_bar(s));
        mma_commit(tfull_bar(acc));
      }
      // drain: completes once every MMA issued above has finished
      mma_commit(drain_bar);
      wait_bar_drain(drain_bar, 0, p.d_err);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    // Warp w owns TMEM lanes 32 (w % 4) .. + 31: quarters 0-1 are tap (ky2, 0)'s
    // rows, 2-3 tap (ky2, 1)'s; output channel co = lane + 32 (q % 2) in both.
    const int q = warp & 3;
    const int co = (q & 1) * 32 + lane;
    const uint32_t lanes = uint32_t(q * 32) << 16;
    {
      // the weight rows of this warp's lanes into TMEM: row = (tap, co), for pair
      // ky2 the tap (ky2, q / 2), 128 K = two slabs of 64 (packed two per column)
      const int tx = q >> 1;
#pragma unroll
      for (int part = 0; part < (SPLIT ? 2 : 1); ++part) {
        const __nv_bfloat16 *wsrc = (part ? p.w_lo : p.w_hi) + size_t(co) * p.kpad;
#pragma unroll
        for (int ky2 = 0; ky2 < 2; ++ky2)
#pragma unroll
          for (int sl = 0; sl < G::NSLAB; ++sl) {
            const uint4 *src = reinterpret_cast<const uint4 *>(wsrc + G::wx(2 * ky2 + tx, sl));
            uint32_t v[32];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const uint4 u = __ldg(src + i);
              v[4 * i] = u.x;
              v[4 * i + 1] = u.y;
              v[4 * i + 2] = u.z;
              v[4 * i + 3] = u.w;
            }
            tmem_st32(tmem + lanes + (part ? C::W_LO_COL : C::W_HI_COL) + uint32_t(64 * ky2 + 32 * sl), v);
          }
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(wready_bar);
    }
    const int et = threadIdx.x - 64;  // 0..127
    if (et < 64) bias_s[et] = p.bias[et];
    named_bar_sync(1, 128);
    // phase 2 takes, in lane l of a warp, row l / 8 of the warp's four and the
    // output channels 4 (l % 8) .. + 3 and 32 + 4 (l % 8) .. + 3
    const int ch4 = lane & 7;
    const float4 ba = *reinterpret_cast<const float4 *>(bias_s + 4 * ch4);
    const float4 bb = *reinterpret_cast<const float4 *>(bias_s + 32 + 4 * ch4);
    const int scol = q * 32 + lane;  // this thread's staging column: its TMEM lane
    // hi (and lo) of ReLU(a + b + bias) for four channels: two packed bf16 pairs each
    auto finish = [&](float4 a, float4 u, float4 bias4, uint2 &hi, uint2 &lo) {
      const float2 x0 = add2(add2(make_float2(a.x, a.y), make_float2(u.x, u.y)), make_float2(bias4.x, bias4.y));
      const float2 x1 = add2(add2(make_float2(a.z, a.w), make_float2(u.z, u.w)), make_float2(bias4.z, bias4.w));
      if constexpr (SPLIT) {
        const float2 r0 = make_float2(fmaxf(x0.x, 0.f), fmaxf(x0.y, 0.f));
        const float2 r1 = make_float2(fmaxf(x1.x, 0.f), fmaxf(x1.y, 0.f));
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(r0.x, r0.y), h1 = __floats2bfloat162_rn(r1.x, r1.y);
        // lo = bf16(relu - hi): the difference is exact, one rounding
        const float2 d0 = fma2(__bfloat1622float2(h0), make_float2(-1.f, -1.f), r0);
        const float2 d1 = fma2(__bfloat1622float2(h1), make_float2(-1.f, -1.f), r1);
        const __nv_bfloat162 l0 = __floats2bfloat162_rn(d0.x, d0.y), l1 = __floats2bfloat162_rn(d1.x, d1.y);
        hi = make_uint2(*reinterpret_cast<const uint32_t *>(&h0), *reinterpret_cast<const uint32_t *>(&h1));
        lo = make_uint2(*reinterpret_cast<const uint32_t *>(&l0), *reinterpret_cast<const uint32_t *>(&l1));
      } else {
        hi = make_uint2(relu_bf16x2(x0), relu_bf16x2(x1));
        lo = hi;
      }
    };
    int it = 0;
    for (int t = T0; t < TE; ++t, ++it) {
      const int acc = it % NACC;
      if (!wait_bar(tfull_bar(acc), uint32_t((it / NACC) & 1), abort_flag, p.d_err, 4)) break;
      tc_fence_after();
      // the previous tile's staging has been read by all four warps
      if (it > 0 && !wait_bar(xfree_bar, uint32_t((it - 1) & 1), abort_flag, p.d_err, 4)) break;
      const uint32_t tb = tmem + lanes + uint32_t(acc) * C::ACC_COLS;
      // phase 1: the accumulator into the staging tile, stg[column][TMEM lane]
#pragma unroll 1
      for (int j = 0; j < 8; ++j) {
        uint32_t r[16];
        tmem_ld16(tb + uint32_t(16 * j), r);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 16; ++e) stg[(16 * j + e) * C::SROW + scol] = __uint_as_float(r[e]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(tempty_bar(acc));  // the accumulator is free for the next tile's MMAs
        mbar_arrive(xfull_bar);
      }
      if (!wait_bar(xfull_bar, uint32_t(it & 1), abort_flag, p.d_err, 4)) break;
      // phase 2: output row c0 + r = stg[r][co] + stg[r + 1][64 + co] + bias
      const uint32_t c0 = uint32_t(t) * uint32_t(C::TSTEP);
#pragma unroll 1
      for (int i = 0; i < 8; ++i) {
        const int r = 16 * i + 4 * (warp - 2) + (lane >> 3);
        if (r >= C::TSTEP) continue;
        const uint32_t pr = c0 + uint32_t(r);
        const uint32_t node = pr / uint32_t(G::PP), px = pr - node * uint32_t(G::PP);
        const uint32_t oy = px / uint32_t(G::PW), ox = px - oy * uint32_t(G::PW);
        if (node >= p.n || oy >= uint32_t(G::OW) || ox >= uint32_t(G::OW)) continue;
        const float *s0 = stg + r * C::SROW, *s1 = stg + (r + 1) * C::SROW + 64;
        const float4 la = *reinterpret_cast<const float4 *>(s0 + 4 * ch4);
        const float4 lb = *reinterpret_cast<const float4 *>(s0 + 32 + 4 * ch4);
        const float4 ua = *reinterpret_cast<const float4 *>(s1 + 4 * ch4);
        const float4 ub = *reinterpret_cast<const float4 *>(s1 + 32 + 4 * ch4);
        uint2 ha, la2, hb, lb2;
        finish(la, ua, ba, ha, la2);
        finish(lb, ub, bb, hb, lb2);
        const size_t o = (size_t(node) * G::P + oy * G::OW + ox) * 64 + 4 * ch4;
        *reinterpret_cast<uint2 *>(p.out_hi + o) = ha;
        *reinterpret_cast<uint2 *>(p.out_hi + o + 32) = hb;
        if constexpr (SPLIT) {
          *reinterpret_cast<uint2 *>(p.out_lo + o) = la2;
          *reinterpret_cast<uint2 *>(p.out_lo + o + 32) = lb2;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(xfree_bar);
    }
  }
  // teardown: every role has left its loop (all waits are bounded)
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

template <int MODE>
int launch_pair(const ConvTmaArgs &a, cudaStream_t st) {
  using C = PairCfg<MODE>;
  if (a.n <= 0) return BCTS_OK;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(conv_pair<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  });
  if (attr_err != cudaSuccess) return BCTS_ECUDA;
  const long long M = (long long)a.n * WinGeo<2>::PP;
  if (M > 0x7FFFFFFFLL) return BCTS_EINVAL;
  // the weight rows (K = 4 x 4 x 32 = 512) are read as 16-byte vectors from K
  // offsets that are multiples of 64
  if (a.kpad < 512 || a.kpad % 8 != 0 || (reinterpret_cast<uintptr_t>(a.w_hi) & 15) != 0 ||
      (C::SPLIT && (reinterpret_cast<uintptr_t>(a.w_lo) & 15) != 0))
    return BCTS_EINVAL;
  CUtensorMap mX, mXlo;
  int rc;
  if ((rc = encode_window_map<2>(&mX, a.in_hi, a.n, false)) != BCTS_OK) return rc;
  if (C::SPLIT) {
    if ((rc = encode_window_map<2>(&mXlo, a.in_lo, a.n, false)) != BCTS_OK) return rc;
  } else {
    mXlo = mX;
  }
  PairParams p{};
  p.w_hi = static_cast<const __nv_bfloat16 *>(a.w_hi);
  p.w_lo = static_cast<const __nv_bfloat16 *>(C::SPLIT ? a.w_lo : a.w_hi);
  p.kpad = a.kpad;
  p.bias = a.bias;
  p.out_hi = static_cast<__nv_bfloat16 *>(a.out_hi);
  p.out_lo = static_cast<__nv_bfloat16 *>(a.out_lo);
  p.n = uint32_t(a.n);
  const long long tiles = (M + C::TSTEP - 1) / C::TSTEP;
  p.num_tiles = int(tiles);
  p.d_err = a.d_err;
  const int grid = int(tiles < num_sms_tma() ? tiles : num_sms_tma());
  ProfScope ps(K_CONV2, st);
  conv_pair<MODE><<<grid, C::THREADS, C::SMEM, st>>>(mX, mXlo, p);
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

}  // namespace
}  // namespace tc

int launch_conv_pair(int mode, const ConvTmaArgs &a, cudaStream_t st) {
  if (mode == 0) return tc::launch_pair<0>(a, st);
  if (mode == 1) return tc::launch_pair<1>(a, st);
  return BCTS_EINVAL;
}

}  // namespace bcts
