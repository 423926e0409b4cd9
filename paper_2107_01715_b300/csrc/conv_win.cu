// conv_win.cu -- conv2 and conv3 of the leaf Q-network (Nature-DQN) as implicit
// GEMMs on tcgen05 whose A operand is read in place from a window of the input
// map held in shared memory.
//
// Stride-1 form.  Number the rows (pixels) of an NHWC map r = node*H*W + y*W + x.
// Output (y, x) of a stride-1 K x K convolution reads, at filter tap (ky, kx),
// input row r + ky*W + kx: the same shift for every output row once the output
// grid is padded to the input's width and height (outputs with x > W - K or
// y > H - K are computed and discarded).  So the A operand of a 128-row tile at
// one tap is 128 consecutive input rows starting at that shift, which a tcgen05
// shared-memory descriptor addresses directly.  One TMA box per tile brings the
// tile's rows plus the halo of the largest shift; each input row crosses from
// L2 into the SM once per tile instead of once per tap (the im2col re-reads of
// a gather: 3.2x the map for conv2, 5.4x for conv3).
//
// conv3 (64 @ 3x3 / 1 on [9][9][64]) has this form as it is: W = 9, shifts
// ky*9 + kx, 49 of every 81 padded rows kept.  conv2 (64 @ 4x4 / 2 on
// [20][20][32]) has it on the space-to-depth view of its input: [10][10]
// super-pixels of 2 x 2 pixels and 128 channels (dy, dx, c), a 2 x 2 stride-1
// filter, shifts ky2*10 + kx2, 81 of every 100 padded rows kept.  In the NHWC
// map the 64 channels (dx, c) of super-pixel row dy are 64 contiguous elements,
// so a 4D tiled TMA box (channels, x2, dy, node*10 + y2) reads the view as it is
// stored: window slab dy holds rows (y2, x2), and its weights are 64 consecutive
// K of the (ky, kx, c) order.  No layer writes a different layout for this.
//
// A window row is one slab's 64 channels: 128 bytes (bf16, 128-byte swizzle) or
// 64 bytes (E4M3, 64-byte swizzle).  A tap's operand starts at a row that is in
// general not a multiple of 8.  The swizzle (written by TMA, read by the MMA) is
// a function of the shared-memory address bits, so a descriptor whose start
// address is that row's address, with the matrix base offset left 0, reads
// rows that TMA stored from a 1024-byte aligned window base (measured on B300:
// setting the base offset to the row's phase instead gives wrong products).
//
// Roles (one CTA per SM, persistent over a contiguous range of tiles):
//   warp 0    one lane issues the TMA loads: resident weights once (BF16, FP8),
//             one window per tile (a stage), and in the FP32-class split mode
//             the [hi; lo] weight sub-tiles per (tap, slab), one tile behind;
//   warp 1    allocates TMEM and, from one lane, issues tcgen05.mma (M = 128,
//             32 bytes of K per instruction) into rotating FP32 accumulators;
//   warps 2-5 epilogue: tcgen05.ld, bias (FP8: per-column scale), ReLU, round to
//             bf16 (split: plus the remainder) or E4M3, and the kept rows to the
//             NHWC output (BF16 / E4M3 straight from registers, the split mode's
//             hi and lo rows through shared-memory staging).
// Precision modes as elsewhere: 0 BF16, 1 FP32-class split (A_hi B_hi + A_hi
// B_lo + A_lo B_hi), 2 FP8 E4M3 with per-channel scales.  Every wait is bounded;
// on a time-out the kernel records an error code, stops issuing, waits for its
// own copies and MMAs and frees TMEM.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "pack.cuh"
#include "conv_win.cuh"
#include "tc_ptx.cuh"
#include "tma_host.cuh"

namespace bcts {
namespace tc {

constexpr int kStgRowW = 144;  // epilogue staging row (128 output bytes + 16 to spread the banks)

template <int LAYER, int MODE>
struct WinCfg {
  using G = WinGeo<LAYER>;
  static constexpr bool SPLIT = MODE == 1, FP8 = MODE == 2;
  static constexpr int EB = FP8 ? 1 : 2;
  static constexpr int ROWB = 64 * EB;                // bytes of a window row of one slab
  static constexpr int NA = SPLIT ? 2 : 1;            // hi (and lo) maps
  static constexpr int NSUB = G::NTAP * G::NSLAB;     // K sub-blocks of 64 elements: (tap, slab)
  static constexpr int SLAB = (G::WROWS * ROWB + 1023) / 1024 * 1024;
  static constexpr int WIN_BYTES = NA * G::NSLAB * SLAB;
  static constexpr int LOAD_BYTES = NA * G::NSLAB * G::WROWS * ROWB;  // what the TMA boxes deliver
  static constexpr int BN = 64;                       // output channels
  static constexpr int BROWS = SPLIT ? 2 * BN : BN;   // weight rows per sub-tile ([hi; lo] in split mode)
  static constexpr int B_SUB = BROWS * ROWB;
  static constexpr bool B_RES = !SPLIT;               // BF16 / FP8 weights stay resident (32-72 KB)
  static constexpr int RES_BYTES = B_RES ? NSUB * B_SUB : 0;
  static constexpr int BST = B_RES ? 0 : 3;           // streamed weight stages (split mode)
  static constexpr int STG_BYTES = 4 * 32 * kStgRowW;
  static constexpr int META_BYTES = 1024;
  static constexpr int BUDGET = 232448 - 1024 - META_BYTES - 2 * BN * 4 - STG_BYTES;
  static constexpr int STAGES_RAW = (BUDGET - RES_BYTES - BST * B_SUB) / WIN_BYTES;
  static constexpr int STAGES = STAGES_RAW > 6 ? 6 : STAGES_RAW;
  static constexpr int ACC_N = SPLIT ? 2 * BN : BN;   // split: [A_hi B_hi | A_hi B_lo] side by side
  static constexpr int NUM_ACC = (512 / ACC_N) > 8 ? 8 : 512 / ACC_N;
  static constexpr uint32_t TMEM_COLS = NUM_ACC * ACC_N;
  static constexpr int THREADS = 32 * 6;
  static constexpr int SMEM =
      1024 + RES_BYTES + STAGES * WIN_BYTES + BST * B_SUB + META_BYTES + 2 * BN * 4 + STG_BYTES;
  static_assert(STAGES >= 2, "window pipeline depth (the split mode's weight stream runs a tile behind)");
  static_assert(SLAB % 1024 == 0 && B_SUB % 1024 == 0 && RES_BYTES % 1024 == 0, "1024-byte boundaries");
  static_assert(TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0, "TMEM columns");
  static_assert(8 * (2 * STAGES + 2 * BST + 2 * NUM_ACC + 2) + 8 <= META_BYTES, "barrier area");
  static_assert(SMEM <= 232448, "shared memory");
};

struct ConvWinParams {
  const float *bias;
  const float *colscale;  // FP8: per-output-channel weight scale x input activation scale
  float out_inv_scale;    // FP8: 1 / activation scale of the output map
  void *out_hi;           // NHWC [node][P][64]: bf16, or E4M3
  void *out_lo;           // split mode: bf16 remainders
  uint32_t n;             // nodes
  int num_tiles;          // ceil(n * PP / 128)
  int *d_err;
};

template <int LAYER, int MODE>
__global__ void __launch_bounds__(WinCfg<LAYER, MODE>::THREADS, 1)
    conv_win(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapAlo,
             const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapBlo,
             const ConvWinParams p) {
  using C = WinCfg<LAYER, MODE>;
  using G = WinGeo<LAYER>;
  constexpr int S = C::STAGES, NACC = C::NUM_ACC, BN = C::BN, BST = C::BST;
  constexpr int BSTM = BST > 0 ? BST : 1;  // modulus for the weight-stage counters (unused when resident)
  constexpr bool SPLIT = C::SPLIT, FP8 = C::FP8;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = smem_raw + (base - raw);
  // layout: [resident weights][windows][streamed weights][barriers + meta][bias, scale][staging]
  const uint32_t res = base;
  const uint32_t win0 = base + C::RES_BYTES;
  const uint32_t bring = win0 + S * C::WIN_BYTES;
  const uint32_t bar0 = bring + BST * C::B_SUB;
  auto wfull_bar = [&](int s) { return bar0 + 8u * s; };
  auto wempty_bar = [&](int s) { return bar0 + 8u * (S + s); };
  auto bfull_bar = [&](int b) { return bar0 + 8u * (2 * S + b); };
  auto bempty_bar = [&](int b) { return bar0 + 8u * (2 * S + BST + b); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * S + 2 * BST + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * S + 2 * BST + NACC + a); };
  const uint32_t wready_bar = bar0 + 8u * (2 * S + 2 * BST + 2 * NACC);
  const uint32_t drain_bar = wready_bar + 8u;
  const uint32_t meta_off = C::RES_BYTES + S * C::WIN_BYTES + BST * C::B_SUB;
  uint8_t *meta = gbase + meta_off + 8 * (2 * S + 2 * BST + 2 * NACC + 2);
  volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(meta);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(meta + 4);
  float *bias_s = reinterpret_cast<float *>(gbase + meta_off + C::META_BYTES);
  float *scale_s = bias_s + BN;
  uint8_t *stg_all = reinterpret_cast<uint8_t *>(scale_s + BN);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (p.num_tiles + int(gridDim.x) - 1) / int(gridDim.x);
  const int T0 = int(blockIdx.x) * per;
  const int TE = T0 + per < p.num_tiles ? T0 + per : p.num_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(wfull_bar(s), 1);
      mbar_init(wempty_bar(s), 1);
    }
    for (int b = 0; b < BST; ++b) {
      mbar_init(bfull_bar(b), 1);
      mbar_init(bempty_bar(b), 1);
    }
    for (int a = 0; a < NACC; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), 4);
    }
    mbar_init(wready_bar, 1);
    mbar_init(drain_bar, 1);
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
      tma_prefetch_map(&mapA);
      if (SPLIT) tma_prefetch_map(&mapAlo);
      tma_prefetch_map(&mapB);
      if (SPLIT) tma_prefetch_map(&mapBlo);
      if (C::B_RES) {
        mbar_arrive_expect_tx(wready_bar, uint32_t(C::RES_BYTES));
        for (int sb = 0; sb < C::NSUB; ++sb)
          tma_load_2d(res + uint32_t(sb * C::B_SUB), &mapB, G::wx(sb / G::NSLAB, sb % G::NSLAB), 0, wready_bar);
      }
      int gw = 0, gb = 0;
      // one tile's window: rows from the tile's first padded row on (conv2: from
      // the start of its line of 10), every slab, hi (and lo)
      auto load_win = [&](int t) -> bool {
        const int s = gw % S;
        if (!wait_bar(wempty_bar(s), uint32_t((gw / S) & 1) ^ 1u, abort_flag, p.d_err, 1)) return false;
        mbar_arrive_expect_tx(wfull_bar(s), uint32_t(C::LOAD_BYTES));
        const uint32_t w = win0 + uint32_t(s * C::WIN_BYTES);
        const int m0 = t * 128;
#pragma unroll
        for (int a = 0; a < C::NA; ++a)
#pragma unroll
          for (int sl = 0; sl < G::NSLAB; ++sl) {
            const uint32_t dst = w + uint32_t((a * G::NSLAB + sl) * C::SLAB);
            const void *map = a ? static_cast<const void *>(&mapAlo) : static_cast<const void *>(&mapA);
            if constexpr (LAYER == 2)
              tma_load_4d(dst, map, 0, 0, sl, m0 / G::PW, wfull_bar(s));
            else
              tma_load_2d(dst, map, 0, m0, wfull_bar(s));
          }
        ++gw;
        return true;
      };
      // the [hi; lo] weight sub-tiles of one tile, streamed (split mode)
      auto load_b = [&]() -> bool {
        for (int sb = 0; sb < C::NSUB; ++sb, ++gb) {
          const int b = gb % BSTM;
          if (!wait_bar(bempty_bar(b), uint32_t((gb / BSTM) & 1) ^ 1u, abort_flag, p.d_err, 1)) return false;
          mbar_arrive_expect_tx(bfull_bar(b), uint32_t(C::B_SUB));
          const uint32_t dst = bring + uint32_t(b * C::B_SUB);
          const int x = G::wx(sb / G::NSLAB, sb % G::NSLAB);
          tma_load_2d(dst, &mapB, x, 0, bfull_bar(b));
          tma_load_2d(dst + uint32_t(C::B_SUB / 2), &mapBlo, x, 0, bfull_bar(b));
        }
        return true;
      };
      bool ok = true;
      if constexpr (C::B_RES) {
        for (int t = T0; t < TE && ok; ++t) ok = load_win(t);
      } else {
        // the window of tile t + 1 is requested before the weights of tile t
        if (T0 < TE) ok = load_win(T0);
        for (int t = T0; t < TE && ok; ++t) {
          if (t + 1 < TE && !(ok = load_win(t + 1))) break;
          if (!(ok = load_b())) break;
        }
      }
      // teardown: the last fill of every stage (and the resident weights) has landed
      for (int k = gw - 1; k >= 0 && k >= gw - S; --k)
        wait_bar_drain(wfull_bar(k % S), uint32_t((k / S) & 1), p.d_err);
      for (int k = gb - 1; k >= 0 && k >= gb - BST; --k)
        wait_bar_drain(bfull_bar(k % BSTM), uint32_t((k / BSTM) & 1), p.d_err);
      if (C::B_RES) wait_bar_drain(wready_bar, 0, p.d_err);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc_n = FP8 ? idesc_e4m3(BN) : idesc_bf16(BN);
      constexpr uint32_t idesc_wide = idesc_bf16(2 * BN);  // [hi; lo] weight rows side by side
      bool ok = true;
      if (C::B_RES) ok = wait_bar(wready_bar, 0, abort_flag, p.d_err, 6);
      int gw = 0, gb = 0, it = 0;
      for (int t = T0; t < TE && ok; ++t, ++it) {
        const int acc = it % NACC;
        if (!wait_bar(tempty_bar(acc), uint32_t((it / NACC) & 1) ^ 1u, abort_flag, p.d_err, 2)) break;
        const int s = gw % S;
        if (!wait_bar(wfull_bar(s), uint32_t((gw / S) & 1), abort_flag, p.d_err, 3)) break;
        tc_fence_after();
        const uint32_t d = tmem + uint32_t(acc * C::ACC_N);
        const uint32_t w = win0 + uint32_t(s * C::WIN_BYTES);
        const int row_off = LAYER == 2 ? (t * 128) % G::PW : 0;  // tile start within its window line
        // The descriptors of one tile differ only in their start-address field
        // (bits 0-13: address / 16): one base for the window (at the tile's first
        // row) and one for the weights, plus offsets that are constants once the
        // loops are unrolled, so the issuing thread spends a few instructions per MMA.
        // Any 32-byte step of a window row takes the start address only (see the top
        // of the file).
        const uint64_t wdesc = swz_desc(w, C::ROWB) + uint64_t(uint32_t(row_off * C::ROWB) >> 4);
        auto a_off = [&](int sb) {  // window offset (in 16 bytes) of sub-block sb's first row
          const int tap = sb / G::NSLAB, sl = sb % G::NSLAB;
          return uint64_t(uint32_t(sl * C::SLAB + ((tap / G::TW) * G::PW + tap % G::TW) * C::ROWB) >> 4);
        };
        constexpr uint64_t kLoOff = uint64_t(uint32_t(G::NSLAB * C::SLAB) >> 4);  // the lo slabs (split)
        if constexpr (C::B_RES) {
          const uint64_t bdesc = swz_desc(res, C::ROWB);
#pragma unroll
          for (int sb = 0; sb < C::NSUB; ++sb) {
#pragma unroll
            for (int kk = 0; kk < C::ROWB / 32; ++kk) {  // 32 bytes of K per instruction
              const uint32_t acc_flag = (sb != 0 || kk != 0) ? 1u : 0u;
              const uint64_t a = wdesc + a_off(sb) + uint64_t(2 * kk);
              const uint64_t bd = bdesc + uint64_t(uint32_t(sb * C::B_SUB) >> 4) + uint64_t(2 * kk);
              if (FP8)
                mma_f8(d, a, bd, idesc_n, acc_flag);
              else
                mma_bf16(d, a, bd, idesc_n, acc_flag);
            }
          }
        } else {
          for (int sb = 0; sb < C::NSUB; ++sb) {
            const int b = gb % BSTM;
            if (!wait_bar(bfull_bar(b), uint32_t((gb / BSTM) & 1), abort_flag, p.d_err, 3)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t bdesc = swz_desc(bring + uint32_t(b * C::B_SUB), C::ROWB);
            const uint64_t a0 = wdesc + a_off(sb);
#pragma unroll
            for (int kk = 0; kk < C::ROWB / 32; ++kk) {
              const uint32_t acc_flag = (sb != 0 || kk != 0) ? 1u : 0u;
              const uint64_t bd = bdesc + uint64_t(2 * kk);
              mma_bf16(d, a0 + uint64_t(2 * kk), bd, idesc_wide, acc_flag);          // [A_hi B_hi | A_hi B_lo]
              mma_bf16(d, a0 + kLoOff + uint64_t(2 * kk), bd, idesc_n, 1u);          // + A_lo B_hi
            }
            mma_commit(bempty_bar(b));  // the weight stage is free once these MMAs have read it
            ++gb;
          }
        }
        if (!ok) break;
        mma_commit(wempty_bar(s));
        ++gw;
        mma_commit(tfull_bar(acc));
      }
      // drain: completes once every MMA issued above has finished
      mma_commit(drain_bar);
      wait_bar_drain(drain_bar, 0, p.d_err);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    // Warp w owns accumulator rows 32 (w % 4) .. + 31 (its TMEM lane quarter).
    const int q = warp & 3;
    const int et = threadIdx.x - 64;  // 0..127
    for (int i = et; i < BN; i += 128) {
      bias_s[i] = p.bias[i];
      scale_s[i] = FP8 ? p.colscale[i] : 1.f;
    }
    named_bar_sync(2, 128);
    uint8_t *stg = stg_all + (warp - 2) * (32 * kStgRowW);
    constexpr int ROWB_OUT = FP8 ? BN : BN * 2;  // bytes of one output row (one of hi / lo)
    constexpr int SEGS = ROWB_OUT / 16;
    // the warp's 32 staged rows: padded rows pr0 .. pr0 + 31, of which the ones
    // inside the output grid go to their NHWC rows
    auto flush = [&](uint8_t *dst, uint32_t pr0) {
      __syncwarp();
#pragma unroll
      for (int i = 0; i < SEGS; ++i) {
        const int k = lane + 32 * i, r = k / SEGS, sgm = k - r * SEGS;
        const uint32_t pr = pr0 + uint32_t(r);
        const uint32_t node = pr / uint32_t(G::PP), px = pr - node * uint32_t(G::PP);
        const uint32_t oy = px / uint32_t(G::PW), ox = px - oy * uint32_t(G::PW);
        if (node < p.n && oy < uint32_t(G::OW) && ox < uint32_t(G::OW))
          *reinterpret_cast<uint4 *>(dst + (size_t(node) * G::P + oy * G::OW + ox) * ROWB_OUT + sgm * 16) =
              *reinterpret_cast<const uint4 *>(stg + r * kStgRowW + sgm * 16);
      }
      __syncwarp();
    };
    int it = 0;
    for (int t = T0; t < TE; ++t, ++it) {
      const int acc = it % NACC;
      if (!wait_bar(tfull_bar(acc), uint32_t((it / NACC) & 1), abort_flag, p.d_err, 4)) break;
      tc_fence_after();
      const uint32_t pr0 = uint32_t(t) * 128u + uint32_t(q * 32);
      const uint32_t tbase = tmem + (uint32_t(q * 32) << 16) + uint32_t(acc * C::ACC_N);
      // this thread's row (accumulator lane pr0 + lane): its NHWC output row, if it
      // is inside the output grid.  BF16 / E4M3: the row's bytes are written
      // straight from registers, so shared memory serves the MMAs' operand reads
      // (measured: conv3 E4M3 0.75 -> 0.63 ms); the split mode's hi and lo rows go
      // through the staging rows (direct stores measured slower there)
      size_t orow = ~size_t(0);
      {
        const uint32_t pr = pr0 + uint32_t(lane);
        const uint32_t node = pr / uint32_t(G::PP), px = pr - node * uint32_t(G::PP);
        const uint32_t oy = px / uint32_t(G::PW), ox = px - oy * uint32_t(G::PW);
        if (node < p.n && oy < uint32_t(G::OW) && ox < uint32_t(G::OW))
          orow = (size_t(node) * G::P + oy * G::OW + ox) * ROWB_OUT;
      }
      uint8_t *ohi = static_cast<uint8_t *>(p.out_hi) + (orow == ~size_t(0) ? 0 : orow);
      const bool live = orow != ~size_t(0);
      constexpr int OW32 = BN / 2;  // split: 32-bit words of this thread's lo row
      uint32_t olo[SPLIT ? OW32 : 1];
#pragma unroll
      for (int j = 0; j < BN / 16; ++j) {
        uint32_t r[16];
        tmem_ld16(tbase + uint32_t(j * 16), r);
        float2 v[8];  // columns 2e, 2e + 1 of this 16-column chunk
        if (SPLIT) {
          uint32_t r2[16];  // the A_hi * B_lo half
          tmem_ld16(tbase + uint32_t(BN + j * 16), r2);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 8; ++e)
            v[e] = add2(make_float2(__uint_as_float(r[2 * e]), __uint_as_float(r[2 * e + 1])),
                        make_float2(__uint_as_float(r2[2 * e]), __uint_as_float(r2[2 * e + 1])));
        } else {
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = make_float2(__uint_as_float(r[2 * e]), __uint_as_float(r[2 * e + 1]));
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int n = j * 16 + 4 * e;
          const float4 c4 = *reinterpret_cast<const float4 *>(bias_s + n);
          const float2 c0 = make_float2(c4.x, c4.y), c1 = make_float2(c4.z, c4.w);
          if (FP8) {
            const float4 s4 = *reinterpret_cast<const float4 *>(scale_s + n);
            v[2 * e] = fma2(v[2 * e], make_float2(s4.x, s4.y), c0);
            v[2 * e + 1] = fma2(v[2 * e + 1], make_float2(s4.z, s4.w), c1);
          } else {
            v[2 * e] = add2(v[2 * e], c0);
            v[2 * e + 1] = add2(v[2 * e + 1], c1);
          }
        }
        if constexpr (FP8) {
          // ReLU, then the output map's activation scale (positive, so the order is free)
          const float2 inv = make_float2(p.out_inv_scale, p.out_inv_scale);
          uint32_t w[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) w[h] = relu_e4m3x4(mul2(v[2 * h], inv), mul2(v[2 * h + 1], inv));
          if (live) *reinterpret_cast<uint4 *>(ohi + j * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
          uint32_t hh[8], ll[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            if constexpr (SPLIT) {
              // hi = bf16(relu(v)), lo = bf16(relu(v) - hi)
              const float2 x = make_float2(fmaxf(v[e].x, 0.f), fmaxf(v[e].y, 0.f));
              const __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
              hh[e] = *reinterpret_cast<const uint32_t *>(&h);
              const float2 dd = fma2(__bfloat1622float2(h), make_float2(-1.f, -1.f), x);  // exact, one rounding
              const __nv_bfloat162 l = __floats2bfloat162_rn(dd.x, dd.y);
              ll[e] = *reinterpret_cast<const uint32_t *>(&l);
            } else {
              hh[e] = relu_bf16x2(v[e]);
            }
          }
          if constexpr (SPLIT) {
            *reinterpret_cast<uint4 *>(stg + lane * kStgRowW + j * 32) = make_uint4(hh[0], hh[1], hh[2], hh[3]);
            *reinterpret_cast<uint4 *>(stg + lane * kStgRowW + j * 32 + 16) = make_uint4(hh[4], hh[5], hh[6], hh[7]);
#pragma unroll
            for (int e = 0; e < 8; ++e) olo[j * 8 + e] = ll[e];
          } else if (live) {
            *reinterpret_cast<uint4 *>(ohi + j * 32) = make_uint4(hh[0], hh[1], hh[2], hh[3]);
            *reinterpret_cast<uint4 *>(ohi + j * 32 + 16) = make_uint4(hh[4], hh[5], hh[6], hh[7]);
          }
        }
      }
      if constexpr (SPLIT) {
        flush(static_cast<uint8_t *>(p.out_hi), pr0);
#pragma unroll
        for (int i = 0; i < OW32 / 4; ++i)
          *reinterpret_cast<uint4 *>(stg + lane * kStgRowW + i * 16) =
              make_uint4(olo[4 * i], olo[4 * i + 1], olo[4 * i + 2], olo[4 * i + 3]);
        flush(static_cast<uint8_t *>(p.out_lo), pr0);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar(acc));
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

// ---------------------------------------------------------------------------
// Host side: tensor maps and launch
// ---------------------------------------------------------------------------
// The input window map (conv_win.cuh).
template <int LAYER, int MODE>
int encode_window(CUtensorMap *m, const void *base, int64_t n) {
  return encode_window_map<LAYER>(m, base, n, WinCfg<LAYER, MODE>::FP8);
}

// Weights [64][kpad] (K-major): one box = 64 rows x 64 consecutive K.
template <int LAYER, int MODE>
int encode_win_weights(CUtensorMap *m, const void *w, int kpad) {
  using C = WinCfg<LAYER, MODE>;
  const Encoders &e = encoders();
  if (!e.tiled) return BCTS_ECUDA;
  const cuuint64_t dims[2] = {cuuint64_t(kpad), cuuint64_t(C::BN)};
  const cuuint64_t strides[1] = {cuuint64_t(kpad) * C::EB};
  const cuuint32_t box[2] = {64, cuuint32_t(C::BN)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = e.tiled(m, C::FP8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                             const_cast<void *>(w), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             swizzle_for(C::ROWB), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? BCTS_OK : BCTS_ECUDA;
}

template <int LAYER, int MODE>
int launch_win(const ConvTmaArgs &a, cudaStream_t st) {
  using C = WinCfg<LAYER, MODE>;
  using G = WinGeo<LAYER>;
  if (a.n <= 0) return BCTS_OK;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(conv_win<LAYER, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  });
  if (attr_err != cudaSuccess) return BCTS_ECUDA;
  const long long M = (long long)a.n * G::PP;
  if (M > 0x7FFFFFFFLL) return BCTS_EINVAL;
  CUtensorMap mA, mAlo, mB, mBlo;
  int rc;
  if ((rc = encode_win_weights<LAYER, MODE>(&mB, a.w_hi, a.kpad)) != BCTS_OK) return rc;
  if (C::SPLIT) {
    if ((rc = encode_win_weights<LAYER, MODE>(&mBlo, a.w_lo, a.kpad)) != BCTS_OK) return rc;
  } else {
    mBlo = mB;
  }
  if ((rc = encode_window<LAYER, MODE>(&mA, a.in_hi, a.n)) != BCTS_OK) return rc;
  if (C::SPLIT) {
    if ((rc = encode_window<LAYER, MODE>(&mAlo, a.in_lo, a.n)) != BCTS_OK) return rc;
  } else {
    mAlo = mA;
  }
  ConvWinParams p{};
  p.bias = a.bias;
  p.colscale = a.colscale;
  p.out_inv_scale = a.out_inv_scale;
  p.out_hi = a.out_hi;
  p.out_lo = a.out_lo;
  p.n = uint32_t(a.n);
  const long long tiles = (M + 127) / 128;
  p.num_tiles = int(tiles);
  p.d_err = a.d_err;
  const int grid = int(tiles < num_sms_tma() ? tiles : num_sms_tma());
  ProfScope ps(LAYER == 2 ? K_CONV2 : K_CONV3, st);
  conv_win<LAYER, MODE><<<grid, C::THREADS, C::SMEM, st>>>(mA, mAlo, mB, mBlo, p);
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

}  // namespace tc

int launch_conv_win(int layer, int mode, const ConvTmaArgs &a, cudaStream_t st) {
  if (layer == 2) {
    if (mode == 0) return tc::launch_win<2, 0>(a, st);
    if (mode == 1) return tc::launch_win<2, 1>(a, st);
    return tc::launch_win<2, 2>(a, st);
  }
  if (mode == 0) return tc::launch_win<3, 0>(a, st);
  if (mode == 1) return tc::launch_win<3, 1>(a, st);
  return tc::launch_win<3, 2>(a, st);
}

}  // namespace bcts
