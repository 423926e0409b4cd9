// conv_tma.cu -- conv2 and conv3 of the leaf Q-network (Nature-DQN) as implicit
// GEMMs on tcgen05, fed by TMA im2col loads.
//
//   out[M][64] = relu(A[M][K] W[64][K]^T + b),  M = nodes x output pixels,
//   K = (ky, kx, c): one "position" per filter tap (ky, kx), c over the input
//   channels of the NHWC activation map.
// For one 128-row tile and one filter tap, the A sub-tile is 128 output pixels'
// input channels at that tap: exactly what one im2col-mode TMA load fetches from
// the NHWC map (the map's bounding box walks the output pixels with the conv's
// stride, across node boundaries, and the im2col offset is the tap).  So a
// single thread fills a pipeline stage with a few bulk copies and one
// expect-tx arrival, instead of eight producer warps gathering 16-byte chunks
// and fencing them for the async proxy.
//
// Roles (one CTA per SM, persistent over a contiguous range of tiles):
//   warp 0    one lane issues the TMA loads (weights once, when they stay
//             resident; per stage the A sub-tiles of PPS taps, and in the
//             FP32-class split mode the weight sub-tiles too);
//   warp 1    allocates TMEM and, from one lane, issues tcgen05.mma (M = 128,
//             32 bytes of K per instruction) into rotating FP32 accumulators;
//   warps 2-5 epilogue: tcgen05.ld, bias (FP8: per-column scale), ReLU, round to
//             bf16 (split: plus the bf16 remainder) or E4M3, NHWC stores through
//             shared-memory staging.
// A sub-tile row holds one tap's channels: 32, 64 or 128 bytes, stored with the
// swizzle of that width (TMA writes it, the MMA descriptor reads it).
// Precision modes as in qnet_tc.cu: 0 BF16, 1 FP32-class split (hi + lo bf16,
// A_hi*B_hi + A_hi*B_lo + A_lo*B_hi), 2 FP8 E4M3 with per-channel scales.
// Every wait is bounded; on a time-out the kernel records an error code,
// stops issuing, waits for its own copies and MMAs and frees TMEM.
#include <cuda.h>  // CUtensorMap and its enums; the encoders come from the runtime's driver entry point
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "pack.cuh"
#include "tc_ptx.cuh"
#include "tma_host.cuh"

namespace bcts {
namespace tc {

template <int LAYER>
struct ConvGeo;
template <>
struct ConvGeo<2> {  // 64@4x4/2 on [20][20][32]
  static constexpr int IC = 32, IW = 20, OW = 9, KS = 4, S = 2;
};
template <>
struct ConvGeo<3> {  // 64@3x3/1 on [9][9][64]
  static constexpr int IC = 64, IW = 9, OW = 7, KS = 3, S = 1;
};

constexpr int kStgRowT = 144;  // epilogue staging row (128 output bytes + 16 to spread the banks)

template <int LAYER, int MODE>
struct TmaCfg {
  using G = ConvGeo<LAYER>;
  static constexpr bool SPLIT = MODE == 1, FP8 = MODE == 2;
  static constexpr int EB = FP8 ? 1 : 2;
  static constexpr int NPOS = G::KS * G::KS;  // filter taps
  static constexpr int P = G::OW * G::OW;     // output pixels per node
  static constexpr int ROWB = G::IC * EB;     // bytes of one tap's channels: 32, 64 or 128
  static constexpr int BN = 64;               // output channels
  static constexpr int A_SUB = 128 * ROWB;    // A sub-tile: 128 rows x one tap
  static constexpr int B_SUB = BN * ROWB;     // weight sub-tile: 64 rows x one tap (one of hi / lo)
  static constexpr int NA_SUB = SPLIT ? 2 : 1;
  // outside the split mode all taps' weights stay in shared memory (32-72 KB)
  static constexpr bool B_RES = !SPLIT;
  static constexpr int RES_BYTES = B_RES ? NPOS * B_SUB : 0;
  static constexpr int POS_BYTES = NA_SUB * A_SUB + (B_RES ? 0 : 2 * B_SUB);
  // taps per pipeline stage (dividing NPOS): about 24-48 KB per stage
  static constexpr int PPS = LAYER == 2 ? (SPLIT ? 2 : 4) : (FP8 ? 3 : 1);
  static constexpr int NKS = NPOS / PPS;
  static constexpr int STAGE_BYTES = PPS * POS_BYTES;
  static constexpr int STG_BYTES = 4 * 32 * kStgRowT;
  static constexpr int META_BYTES = 1024;  // barriers, TMEM address, abort flag
  static constexpr int BUDGET = 232448 - 1024 - META_BYTES - STG_BYTES - 2 * BN * 4;
  static constexpr int STAGES_RAW = (BUDGET - RES_BYTES) / STAGE_BYTES;
  static constexpr int STAGES = STAGES_RAW > 8 ? 8 : STAGES_RAW;
  static constexpr int ACC_N = SPLIT ? 2 * BN : BN;  // split: [A_hi B_hi | A_hi B_lo] side by side
  static constexpr int NUM_ACC = (512 / ACC_N) > 8 ? 8 : 512 / ACC_N;
  static constexpr uint32_t TMEM_COLS = NUM_ACC * ACC_N;
  static constexpr int THREADS = 32 * 6;
  static constexpr int SMEM = 1024 + RES_BYTES + STAGES * STAGE_BYTES + META_BYTES + 2 * BN * 4 + STG_BYTES;
  static_assert(NPOS % PPS == 0, "whole taps per stage");
  static_assert(STAGES >= 2, "pipeline depth");
  static_assert(A_SUB % 1024 == 0 && B_SUB % 1024 == 0 && RES_BYTES % 1024 == 0 && POS_BYTES % 1024 == 0,
                "sub-tiles on 1024-byte boundaries");
  static_assert(TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0, "TMEM columns");
  static_assert(8 * (2 * STAGES + 2 * NUM_ACC + 2) + 8 <= META_BYTES, "barrier area");
  static_assert(SMEM <= 232448, "shared memory");
};

struct ConvTmaParams {
  const float *bias;
  const float *colscale;  // FP8: per-output-channel weight scale x input activation scale
  float out_inv_scale;    // FP8: 1 / activation scale of the output map
  void *out_hi;           // NHWC [node][P][64]: bf16, or E4M3
  void *out_lo;           // split mode: bf16 remainders
  uint32_t M;             // output rows = nodes x P
  int num_tiles;
  int *d_err;
};

template <int LAYER, int MODE>
__global__ void __launch_bounds__(TmaCfg<LAYER, MODE>::THREADS, 1)
    conv_tma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapAlo,
             const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapBlo,
             const ConvTmaParams p) {
  using C = TmaCfg<LAYER, MODE>;
  using G = ConvGeo<LAYER>;
  constexpr int S = C::STAGES, NA = C::NUM_ACC, BN = C::BN;
  constexpr bool SPLIT = C::SPLIT, FP8 = C::FP8;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = smem_raw + (base - raw);
  // layout: [resident weights][stages][barriers + meta][bias, scale][epilogue staging]
  const uint32_t res = base;
  const uint32_t stage0 = base + C::RES_BYTES;
  const uint32_t bar0 = stage0 + S * C::STAGE_BYTES;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (S + s); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * S + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * S + NA + a); };
  const uint32_t wready_bar = bar0 + 8u * (2 * S + 2 * NA);
  const uint32_t drain_bar = wready_bar + 8u;
  uint8_t *meta = gbase + C::RES_BYTES + S * C::STAGE_BYTES + 8 * (2 * S + 2 * NA + 2);
  volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(meta);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(meta + 4);
  float *bias_s = reinterpret_cast<float *>(gbase + C::RES_BYTES + S * C::STAGE_BYTES + C::META_BYTES);
  float *scale_s = bias_s + BN;
  uint8_t *stg_all = reinterpret_cast<uint8_t *>(scale_s + BN);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // contiguous tile range per CTA: neighbouring output rows share input rows in L2
  const int per = (p.num_tiles + int(gridDim.x) - 1) / int(gridDim.x);
  const int T0 = int(blockIdx.x) * per;
  const int TE = T0 + per < p.num_tiles ? T0 + per : p.num_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < NA; ++a) {
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
        for (int pos = 0; pos < C::NPOS; ++pos)
          tma_load_2d(res + uint32_t(pos * C::B_SUB), &mapB, pos * G::IC, 0, wready_bar);
      }
      int g = 0;
      bool ok = true;
      for (int t = T0; t < TE && ok; ++t) {
        const uint32_t m0 = uint32_t(t) * 128u;
        const uint32_t node0 = m0 / uint32_t(C::P), px0 = m0 - node0 * uint32_t(C::P);
        const int oy0 = int(px0) / G::OW, ox0 = int(px0) - (int(px0) / G::OW) * G::OW;
        // traversal start: the first output pixel's window corner in input coordinates
        const int w0 = G::S * ox0, h0 = G::S * oy0;
        for (int ks = 0; ks < C::NKS; ++ks, ++g) {
          const int s = g % S;
          if (!wait_bar(empty_bar(s), uint32_t((g / S) & 1) ^ 1u, abort_flag, p.d_err, 1)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full_bar(s), uint32_t(C::STAGE_BYTES));
#pragma unroll
          for (int j = 0; j < C::PPS; ++j) {
            const int pos = ks * C::PPS + j;
            const int ky = pos / G::KS, kx = pos - (pos / G::KS) * G::KS;
            const uint32_t sub = stage0 + uint32_t(s * C::STAGE_BYTES + j * C::POS_BYTES);
            tma_load_im2col_4d(sub, &mapA, 0, w0, h0, int(node0), uint16_t(kx), uint16_t(ky), full_bar(s));
            if (SPLIT)
              tma_load_im2col_4d(sub + C::A_SUB, &mapAlo, 0, w0, h0, int(node0), uint16_t(kx), uint16_t(ky),
                                 full_bar(s));
            if (!C::B_RES) {
              const uint32_t sB = sub + uint32_t(C::NA_SUB * C::A_SUB);
              tma_load_2d(sB, &mapB, pos * G::IC, 0, full_bar(s));
              tma_load_2d(sB + C::B_SUB, &mapBlo, pos * G::IC, 0, full_bar(s));
            }
          }
        }
      }
      // teardown: the last fill of every stage (and the resident weights) has landed
      for (int k = g - 1; k >= 0 && k >= g - S; --k) wait_bar_drain(full_bar(k % S), uint32_t((k / S) & 1), p.d_err);
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
      const uint64_t stage_desc = swz_desc(stage0, C::ROWB), res_desc = swz_desc(res, C::ROWB);
      int g = 0, it = 0;
      for (int t = T0; t < TE && ok; ++t, ++it) {
        const int acc = it % NA;
        if (!wait_bar(tempty_bar(acc), uint32_t((it / NA) & 1) ^ 1u, abort_flag, p.d_err, 2)) break;
        tc_fence_after();
        const uint32_t d = tmem + uint32_t(acc * C::ACC_N);
        for (int ks = 0; ks < C::NKS; ++ks, ++g) {
          const int s = g % S;
          if (!wait_bar(full_bar(s), uint32_t((g / S) & 1), abort_flag, p.d_err, 3)) {
            ok = false;
            break;
          }
          tc_fence_after();
          // the descriptors differ only in their start-address field (address / 16)
          const uint64_t sd = stage_desc + uint64_t(uint32_t(s * C::STAGE_BYTES) >> 4);
#pragma unroll
          for (int j = 0; j < C::PPS; ++j) {
            const int pos = ks * C::PPS + j;
            const uint64_t aj = sd + uint64_t(uint32_t(j * C::POS_BYTES) >> 4);
            const uint64_t bj = C::B_RES ? res_desc + uint64_t(uint32_t(pos * C::B_SUB) >> 4)
                                         : aj + uint64_t(uint32_t(C::NA_SUB * C::A_SUB) >> 4);
#pragma unroll
            for (int kk = 0; kk < C::ROWB / 32; ++kk) {  // 32 bytes of K per instruction
              const uint32_t acc_flag = (pos != 0 || kk != 0) ? 1u : 0u;
              const uint64_t a = aj + uint64_t(2 * kk);
              const uint64_t b = bj + uint64_t(2 * kk);
              if (FP8) {
                mma_f8(d, a, b, idesc_n, acc_flag);
              } else if (SPLIT) {
                mma_bf16(d, a, b, idesc_wide, acc_flag);  // [A_hi B_hi | A_hi B_lo]
                mma_bf16(d, a + uint64_t(uint32_t(C::A_SUB) >> 4), b, idesc_n, 1u);  // + A_lo B_hi
              } else {
                mma_bf16(d, a, b, idesc_n, acc_flag);
              }
            }
          }
          mma_commit(empty_bar(s));  // the stage is free once these MMAs have read it
        }
        if (!ok) break;
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
    uint8_t *stg = stg_all + (warp - 2) * (32 * kStgRowT);
    constexpr int ROWB_OUT = FP8 ? BN : BN * 2;  // bytes of one output row (one of hi / lo)
    constexpr int SEGS = ROWB_OUT / 16;
    // write the warp's 32 staged rows to consecutive NHWC rows from mw0 on
    auto flush = [&](uint8_t *dst, uint32_t mw0) {
      __syncwarp();
#pragma unroll
      for (int i = 0; i < SEGS; ++i) {
        const int k = lane + 32 * i, r = k / SEGS, sgm = k - r * SEGS;
        if (mw0 + uint32_t(r) < p.M)
          *reinterpret_cast<uint4 *>(dst + size_t(mw0 + r) * ROWB_OUT + sgm * 16) =
              *reinterpret_cast<const uint4 *>(stg + r * kStgRowT + sgm * 16);
      }
      __syncwarp();
    };
    int it = 0;
    for (int t = T0; t < TE; ++t, ++it) {
      const int acc = it % NA;
      if (!wait_bar(tfull_bar(acc), uint32_t((it / NA) & 1), abort_flag, p.d_err, 4)) break;
      tc_fence_after();
      const uint32_t mw0 = uint32_t(t) * 128u + uint32_t(q * 32);
      const uint32_t tbase = tmem + (uint32_t(q * 32) << 16) + uint32_t(acc * C::ACC_N);
      constexpr int OW32 = FP8 ? BN / 4 : BN / 2;  // 32-bit words of this thread's output row
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
          *reinterpret_cast<uint4 *>(stg + lane * kStgRowT + j * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
          uint32_t hh[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            if constexpr (SPLIT) {
              // hi = bf16(relu(v)), lo = bf16(relu(v) - hi)
              const float2 x = make_float2(fmaxf(v[e].x, 0.f), fmaxf(v[e].y, 0.f));
              const __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
              hh[e] = *reinterpret_cast<const uint32_t *>(&h);
              const float2 dd = fma2(__bfloat1622float2(h), make_float2(-1.f, -1.f), x);  // exact, one rounding
              const __nv_bfloat162 l = __floats2bfloat162_rn(dd.x, dd.y);
              olo[j * 8 + e] = *reinterpret_cast<const uint32_t *>(&l);
            } else {
              hh[e] = relu_bf16x2(v[e]);
            }
          }
          *reinterpret_cast<uint4 *>(stg + lane * kStgRowT + j * 32) = make_uint4(hh[0], hh[1], hh[2], hh[3]);
          *reinterpret_cast<uint4 *>(stg + lane * kStgRowT + j * 32 + 16) = make_uint4(hh[4], hh[5], hh[6], hh[7]);
        }
      }
      flush(static_cast<uint8_t *>(p.out_hi), mw0);
      if constexpr (SPLIT) {
#pragma unroll
        for (int i = 0; i < OW32 / 4; ++i)
          *reinterpret_cast<uint4 *>(stg + lane * kStgRowT + i * 16) =
              make_uint4(olo[4 * i], olo[4 * i + 1], olo[4 * i + 2], olo[4 * i + 3]);
        flush(static_cast<uint8_t *>(p.out_lo), mw0);
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
const Encoders &encoders() {
  static Encoders e;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1{}, q2{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeIm2col", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess)
      e.im2col = reinterpret_cast<EncodeIm2col>(f1);
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess)
      e.tiled = reinterpret_cast<EncodeTiled>(f2);
    cudaGetLastError();
  });
  return e;
}

CUtensorMapSwizzle swizzle_for(int rowb) {
  return rowb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : (rowb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
}

// im2col map of an NHWC input map [n][IW][IW][IC]: 128 output pixels per load,
// the conv's stride as traversal stride, window corners 0 .. IW - KS per side.
template <int LAYER, int MODE>
int encode_input(CUtensorMap *m, const void *base, int64_t n) {
  using C = TmaCfg<LAYER, MODE>;
  using G = ConvGeo<LAYER>;
  const Encoders &e = encoders();
  if (!e.im2col) return BCTS_ECUDA;
  const cuuint64_t dims[4] = {cuuint64_t(G::IC), cuuint64_t(G::IW), cuuint64_t(G::IW), cuuint64_t(n)};
  const cuuint64_t strides[3] = {cuuint64_t(G::IC) * C::EB, cuuint64_t(G::IW) * G::IC * C::EB,
                                 cuuint64_t(G::IW) * G::IW * G::IC * C::EB};
  const int lower[2] = {0, 0};
  const int upper[2] = {-(G::KS - 1), -(G::KS - 1)};
  const cuuint32_t estr[4] = {1, cuuint32_t(G::S), cuuint32_t(G::S), 1};
  const CUresult r = e.im2col(m, C::FP8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                              const_cast<void *>(base), dims, strides, lower, upper, cuuint32_t(G::IC), 128u, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(C::ROWB), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? BCTS_OK : BCTS_ECUDA;
}

// tiled map of the weights [64][kpad] (K-major): one box = 64 rows x one tap.
template <int LAYER, int MODE>
int encode_weights(CUtensorMap *m, const void *w, int kpad) {
  using C = TmaCfg<LAYER, MODE>;
  using G = ConvGeo<LAYER>;
  const Encoders &e = encoders();
  if (!e.tiled) return BCTS_ECUDA;
  const cuuint64_t dims[2] = {cuuint64_t(kpad), cuuint64_t(C::BN)};
  const cuuint64_t strides[1] = {cuuint64_t(kpad) * C::EB};
  const cuuint32_t box[2] = {cuuint32_t(G::IC), cuuint32_t(C::BN)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = e.tiled(m, C::FP8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                             const_cast<void *>(w), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             swizzle_for(C::ROWB), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? BCTS_OK : BCTS_ECUDA;
}

int num_sms_tma() {
  static int sms = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
  });
  return sms;
}

template <int LAYER, int MODE>
int launch_tma(const ConvTmaArgs &a, cudaStream_t st) {
  using C = TmaCfg<LAYER, MODE>;
  if (a.n <= 0) return BCTS_OK;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(conv_tma<LAYER, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  });
  if (attr_err != cudaSuccess) return BCTS_ECUDA;
  const long long M = (long long)a.n * C::P;
  if (M > 0x7FFFFFFFLL) return BCTS_EINVAL;
  CUtensorMap mA, mAlo, mB, mBlo;
  int rc;
  if ((rc = encode_input<LAYER, MODE>(&mA, a.in_hi, a.n)) != BCTS_OK) return rc;
  if ((rc = encode_weights<LAYER, MODE>(&mB, a.w_hi, a.kpad)) != BCTS_OK) return rc;
  if (C::SPLIT) {
    if ((rc = encode_input<LAYER, MODE>(&mAlo, a.in_lo, a.n)) != BCTS_OK) return rc;
    if ((rc = encode_weights<LAYER, MODE>(&mBlo, a.w_lo, a.kpad)) != BCTS_OK) return rc;
  } else {
    mAlo = mA;
    mBlo = mB;
  }
  ConvTmaParams p{};
  p.bias = a.bias;
  p.colscale = a.colscale;
  p.out_inv_scale = a.out_inv_scale;
  p.out_hi = a.out_hi;
  p.out_lo = a.out_lo;
  p.M = uint32_t(M);
  const long long tiles = (M + 127) / 128;
  p.num_tiles = int(tiles);
  p.d_err = a.d_err;
  const int grid = int(tiles < num_sms_tma() ? tiles : num_sms_tma());
  ProfScope ps(LAYER == 2 ? K_CONV2 : K_CONV3, st);
  conv_tma<LAYER, MODE><<<grid, C::THREADS, C::SMEM, st>>>(mA, mAlo, mB, mBlo, p);
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

}  // namespace tc

int launch_conv_tma(int layer, int mode, const ConvTmaArgs &a, cudaStream_t st) {
  if (layer == 2) {
    if (mode == 0) return tc::launch_tma<2, 0>(a, st);
    if (mode == 1) return tc::launch_tma<2, 1>(a, st);
    return tc::launch_tma<2, 2>(a, st);
  }
  if (mode == 0) return tc::launch_tma<3, 0>(a, st);
  if (mode == 1) return tc::launch_tma<3, 1>(a, st);
  return tc::launch_tma<3, 2>(a, st);
}

}  // namespace bcts
