// qnet_tc.cu -- the leaf Q-network (Nature-DQN) on B300's 5th-generation tensor
// cores: tcgen05.mma with FP32 accumulators in tensor memory (TMEM).
//
// Every layer (conv1, conv2, conv3, fc1) is one persistent, warp-specialised
// implicit GEMM  out[M][N] = relu(A[M][K] W[N][K]^T + b), M = nodes x output
// pixels, K = Cin x kh x kw:
//   warps 0-7  producers: gather the A tile (im2col rows of the NHWC activation
//              map, or for conv1 the frame pixels -- read from the frame stacks
//              or rendered on the fly from the node states) and the weight tile
//              into 128-byte-swizzled shared memory (cp.async, or st.shared
//              after the uint8 -> bf16 conversion), then signal a full barrier;
//   last warp  allocates TMEM and, from one lane, issues tcgen05.mma (M = 128,
//              K = 16 per instruction) over the K blocks, committing each stage
//              back to its producer barrier and each finished tile to the
//              epilogue;
//   warps 8-11 (conv1: 8-15) epilogue: tcgen05.ld the accumulator (one TMEM lane per thread),
//              add bias, ReLU, round to bf16 (and, in the FP32-class mode, the
//              bf16 remainder) or E4M3 and store NHWC; up to eight accumulators
//              rotate so the next tiles' MMAs overlap this tile's epilogue.
// Precision modes: BF16 (one MMA per K step), FP8 (E4M3 operands, K = 32 per
// instruction, per-output-channel weight scales and per-layer activation
// scales) and FP32-class "split" mode, where every operand x is carried as
// hi = bf16(x), lo = bf16(x - hi) and the product is hi*hi + hi*lo + lo*hi
// (three MMAs; two for conv1, whose integer pixels are exact in bf16),
// accumulated in FP32.  FC2 and the max over actions run in FP32 on CUDA cores
// (9,216 MACs per node, 0.1 % of the network).  The leaves' conv1 is, on the
// default path, the streaming pass of leaf_conv1.cu over the sprite tables; on
// the frame path it runs here as layers 5 (the parents' partial maps from their
// older frames) and 6 (each leaf's newest frame plus its parent's map).  conv2
// and conv3 may instead run in the TMA im2col kernel (conv_tma.cu) or the
// shared-memory window kernel (conv_win.cu), chosen per precision.
//
// Every wait is bounded: a wait that runs out sets the context's device error
// word and an abort flag, every role leaves its loop, in-flight copies and MMAs
// are drained and TMEM is freed before the kernel returns.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "pack.cuh"
#include "render.cuh"
#include "tc_ptx.cuh"

namespace bcts {
namespace tc {

// ---------------------------------------------------------------------------
// Layer geometry
// ---------------------------------------------------------------------------
// LAYER 1: conv1 32@8x8/4, K = c*64 + ky*8 + kx (the PyTorch order), one K block
//          per input channel; A from uint8 frames or rendered from states.
// LAYER 2: conv2 64@4x4/2 on [20][20][32], K = (ky*4 + kx)*32 + c.
// LAYER 3: conv3 64@3x3/1 on [9][9][64],  K = (ky*3 + kx)*64 + c.
// LAYER 4: fc1 512 on the NHWC-flattened [7][7][64] map, N tiled by 256.
template <int LAYER>
struct Geo;
template <>
struct Geo<1> {
  static constexpr int BN = 32, KB = 4, P = 400, NTOT = 32, K = 256;
};
template <>
struct Geo<2> {
  static constexpr int BN = 64, KB = 8, P = 81, NTOT = 64, K = 512;
};
template <>
struct Geo<3> {
  static constexpr int BN = 64, KB = 9, P = 49, NTOT = 64, K = 576;
};
template <>
struct Geo<4> {
  static constexpr int BN = 256, KB = 49, P = 1, NTOT = 512, K = 3136;
};
// LAYER 5: the parents' partial conv1 maps from rendered frames: weight channels
//          0-2 over the parent's history slots 1-3, FP32 out, no ReLU.
// LAYER 6: the leaves' conv1 from rendered frames: weight channel 3 over the
//          leaf's newest frame, plus its parent's partial map, then the ReLU.
template <>
struct Geo<5> {
  static constexpr int BN = 32, KB = 3, P = 400, NTOT = 32, K = 192;
};
template <>
struct Geo<6> {
  static constexpr int BN = 32, KB = 1, P = 400, NTOT = 32, K = 64;
};

// Epilogue staging: 32 rows of up to 128 bytes (+16 to spread the banks) per warp.
constexpr int kStgRow = 144;
constexpr int kBarBytes = 512;  // mbarriers, TMEM address, abort flag

// MODE 0: BF16 operands; 1: FP32-class split (bf16 hi + lo); 2: FP8 E4M3 operands
// with per-output-channel weight scales and per-layer activation scales.
// A K block is always 128 bytes: 64 bf16 or 128 E4M3 elements (FP8 pads K to a
// whole block with zero weights).
// conv1 here is the full 4-channel convolution, for the roots and depth-1 nodes
// (rendered from their states) and for materialised frame stacks.  The leaves'
// conv1 and the parents' partial maps it starts from are streaming passes over
// sprite tables (leaf_conv1.cu).  A 128-byte K block holds one history slot
// (bf16) or two (E4M3: slots 2j, 2j + 1).
template <int LAYER, int MODE>
struct Cfg {
  using G = Geo<LAYER>;
  static constexpr bool SPLIT = MODE == 1, FP8 = MODE == 2;
  static constexpr int EB = FP8 ? 1 : 2;              // bytes per element
  static constexpr int KB_FULL = FP8 ? (G::K + 127) / 128 : G::K / 64;
  static constexpr int KB = KB_FULL;  // K blocks per tile
  static constexpr int KPAD = KB_FULL * (128 / EB);  // stored weight row length in elements
  // conv1 family (A from uint8 frame pixels): layers 1, 5, 6
  static constexpr bool C1 = LAYER == 1 || LAYER == 5 || LAYER == 6;
  static constexpr int WROW = C1 ? 256 : KPAD;  // row length of the stored weights
  // first weight K block and first weight channel (history slot) the tile uses,
  // and the number of channels: layer 5 channels 0-2, layer 6 channel 3
  static constexpr int KB0 = LAYER == 6 ? (FP8 ? 1 : 3) : 0;
  static constexpr int CH0 = LAYER == 6 ? 3 : 0;
  static constexpr int NCH = LAYER == 5 ? 3 : (LAYER == 6 ? 1 : 4);
  static constexpr bool A_LO = SPLIT && !C1;  // conv1's integer pixels are exact in bf16
  // Weights resident in shared memory for the whole kernel: conv1 (8-32 KB) and,
  // outside split mode, conv2/conv3 (32-72 KB), instead of one weight tile per
  // K block of every output tile fetched again from L2.
  static constexpr bool B_RES = C1 || (!SPLIT && (LAYER == 2 || LAYER == 3));
  // Split mode stores the weight tile as [hi rows; lo rows] so that one MMA of
  // twice the width gives A_hi*B_hi and A_hi*B_lo side by side in TMEM (the
  // epilogue adds the halves); fc1's 256-wide tiles keep separate MMAs.
  static constexpr bool B_CAT = SPLIT && LAYER != 4;
  static constexpr int A_BYTES = 128 * 128;
  static constexpr int B_ROWS = G::BN * (SPLIT ? 2 : 1);
  static constexpr int B_BYTES = G::BN * 128;            // one of hi / lo
  static constexpr int ACC_N = B_CAT ? 2 * G::BN : G::BN;  // accumulator columns per tile
  static constexpr int RES_BYTES = B_RES ? KB * B_ROWS * 128 : 0;
  // K blocks per pipeline stage, and stages the MMA thread waits for (and
  // fences) as one group.  A stage's hand-off (barrier wait, arrivals, proxy
  // fence, commit) costs about as much as its copies for the short 64-column
  // conv2/conv3 tiles: two K blocks per stage there halve it.  Split conv2/conv3
  // (48 KB K blocks) measured faster with single K blocks waited for in pairs
  // (and E4M3 with its two-K-block stages in pairs), fc1 with single ones.
  static constexpr int KPS = ((LAYER == 2 || LAYER == 3) && !SPLIT) ? 2 : 1;
  static constexpr int FGROUP = ((LAYER == 2 || LAYER == 3) && (KPS == 1 || FP8)) ? 2 : 1;
  static constexpr int NKS = (KB + KPS - 1) / KPS;  // stages per tile
  static constexpr int SUB_BYTES = A_BYTES * (A_LO ? 2 : 1) + (B_RES ? 0 : B_ROWS * 128);  // one K block
  static constexpr int STAGE_BYTES = KPS * SUB_BYTES;
  static constexpr int STAGES_RAW = (192 * 1024 - RES_BYTES) / STAGE_BYTES;
  // fused conv1 fills all KB stages of a tile together: a ring of RING tiles
  static constexpr int RING = LAYER == 1 ? (8 / KB >= 2 ? 8 / KB : 2) : 1;
  static constexpr int STAGES = LAYER == 1 ? RING * KB : (STAGES_RAW > 8 / KPS ? 8 / KPS : STAGES_RAW);
  // fused conv1: re-zero lists (8 x 256 entries) + node-state ring (3 tiles x 2 nodes)
  static constexpr int DIRTY_BYTES = LAYER == 1 ? 2 * 4 * 256 * 4 + 3 * 2 * 80 : 0;
  // conv1 (32-column tiles, the lightest epilogue) runs two epilogue warpgroups
  // on alternating tiles so each has two tiles' time to hide its load latency
  static constexpr int EPI_WG = C1 ? 2 : 1;
  // contiguous tile range per CTA (see the tile schedule in the kernel):
  // conv2/conv3 gain from it (neighbouring output rows share input rows), and so
  // do the frame path's partial maps and leaf conv1 (siblings are consecutive:
  // they share ancestor frames and their parent's partial map, which then stays
  // in the SM's L1 across the siblings' tiles; measured 3-5 % on layer 6)
  static constexpr bool CONTIG = LAYER == 2 || LAYER == 3 || LAYER == 5 || LAYER == 6;
  static constexpr int MMA_WARP = 8 + 4 * EPI_WG;
  static constexpr int THREADS = 32 * (MMA_WARP + 1);
  static constexpr int SMEM = RES_BYTES + STAGES * STAGE_BYTES + 1024 + kBarBytes + DIRTY_BYTES + 2 * G::NTOT * 4 +
                              4 * EPI_WG * 32 * kStgRow;
  // as many accumulators (up to 4) as TMEM's 512 columns hold, so the MMAs run
  // ahead of the two epilogue warpgroups
  static constexpr int NUM_ACC = (8 * ACC_N <= 512) ? 8 : ((4 * ACC_N <= 512) ? 4 : 2);
  static constexpr uint32_t TMEM_COLS = NUM_ACC * ACC_N < 32 ? 32 : NUM_ACC * ACC_N;
  static_assert(STAGES >= 2, "pipeline depth");
  static_assert(RES_BYTES % 1024 == 0 && SUB_BYTES % 1024 == 0, "1024-byte aligned tiles");
  static_assert(ACC_N <= 256 && TMEM_COLS <= 512, "accumulator");
  static_assert(SMEM <= 232448, "shared memory");
};

struct GemmParams {
  const void *a_hi;  // bf16 activations, uint8 frames or node states
  const void *a_lo;  // bf16 activation remainders (split mode, layers 2-4)
  const void *b_hi;  // weights [NTOT][KPAD], bf16 or E4M3
  const void *b_lo;
  const float *bias;
  const float *colscale;  // FP8: per-output-channel weight scale x input activation scale
  float out_inv_scale;    // FP8: 1 / activation scale of this layer's output map
  void *out_hi;  // bf16 NHWC (layers 1-3) or FP32 [M][512] (layer 4)
  void *out_lo;  // bf16 remainders (split mode, layers 1-3)
  uint32_t M;  // rows, < 2^31 (checked by the launcher)
  // conv1 family over frames: the A operand's history slot s (weight channel
  // CH0 + s) of node i of this launch is the 84 x 84 frame at
  // fsrc[s] + ((node0 + i) / fdiv[s] - fsub[s]) * fstride[s]
  const uint8_t *fsrc[4];
  uint32_t fdiv[4], fsub[4], fstride[4];
  uint32_t node0;
  // layer 6: partial map of the parent (FP32 [parent][400][32]) of node i: parent
  // = zparent[zleaf0 + i] if zparent is set, else (zleaf0 + i) / zbranch
  const float *zmap;
  const uint32_t *zparent;
  uint32_t zleaf0, zbranch;
  // layer 4 (fc1) with fc2 folded into its epilogue: fc2 weights [fA][512] FP32;
  // partial Q-values of each row's 256-column half, qpart[row][half][kMaxA]
  const float *w2;
  int fA;
  float *qpart;
  int num_tiles;
  int *d_err;
};

// warps 0-7 producers, 8 .. 8 + 4 EPI_WG - 1 epilogue, then the MMA warp
constexpr int kProdWarps = 8;
constexpr int kProd = 32 * kProdWarps;  // producer threads
constexpr int kEpiWarp0 = 8;

template <int LAYER, int MODE, bool FUSED>
__global__ void __launch_bounds__(Cfg<LAYER, MODE>::THREADS, 1) tc_gemm(const GemmParams p) {
  using C = Cfg<LAYER, MODE>;
  constexpr int kMmaWarp = C::MMA_WARP;
  using G = Geo<LAYER>;
  constexpr bool SPLIT = C::SPLIT, FP8 = C::FP8;
  constexpr int EB = C::EB;
  constexpr int BN = G::BN, KB = C::KB, S = C::STAGES;
  constexpr int NT = G::NTOT / BN;  // N tiles per M tile
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = smem_raw + (base - raw);
  // layout: [resident weights][stages][barriers + meta (256 B)][re-zero lists]
  const uint32_t res = base;
  const uint32_t stage0 = base + C::RES_BYTES;
  const uint32_t bar0 = stage0 + S * C::STAGE_BYTES;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (S + s); };
  constexpr int NA = C::NUM_ACC;
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * S + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * S + NA + a); };
  const uint32_t drain_bar = bar0 + 8u * (2 * S + 2 * NA);
  const uint32_t wready_bar = bar0 + 8u * (2 * S + 2 * NA + 1);
  uint8_t *meta = gbase + C::RES_BYTES + S * C::STAGE_BYTES + 8 * (2 * S + 2 * NA + 2);
  volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(meta);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(meta + 4);
  uint32_t *dirty = reinterpret_cast<uint32_t *>(gbase + C::RES_BYTES + S * C::STAGE_BYTES + kBarBytes);
  float *bias_s = reinterpret_cast<float *>(gbase + C::RES_BYTES + S * C::STAGE_BYTES + kBarBytes + C::DIRTY_BYTES);
  static_assert(8 * (2 * S + 2 * C::NUM_ACC + 2) + 8 <= kBarBytes, "barrier area");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto sA_of = [&](int s) { return stage0 + uint32_t(s) * C::STAGE_BYTES; };
  // Tile schedule, the same for every role: CTA b takes tiles T0, T0 + TS, ...
  // below TE.  Grid-stride, or one contiguous range per CTA (CONTIG): then
  // consecutive conv2/conv3 tiles re-read each other's input rows while they
  // are still in L2.
  int T0 = blockIdx.x, TS = gridDim.x, TE = p.num_tiles;
  if (C::CONTIG) {
    const int per = (p.num_tiles + int(gridDim.x) - 1) / int(gridDim.x);
    T0 = int(blockIdx.x) * per;
    TS = 1;
    TE = T0 + per < p.num_tiles ? T0 + per : p.num_tiles;
  }
  // K block kk of stage s: A (hi, then lo in split mode), then the weight tile unless resident
  auto sub_of = [&](int s, int kk) { return sA_of(s) + uint32_t(kk) * C::SUB_BYTES; };
  auto sB_of = [&](int s, int kk) { return sub_of(s, kk) + C::A_BYTES * (C::A_LO ? 2 : 1); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_bar(s), kProd);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < NA; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), 4);
    }
    mbar_init(drain_bar, 1);
    mbar_init(wready_bar, kProd);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) tmem_alloc(smem_u32((const void *)tmem_slot), C::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < kProdWarps) {
    // ------------------------------------------------------------ producers
    const int pt = threadIdx.x;  // 0..255
    const int ch = pt & 7, r0 = pt >> 3;  // 16-byte chunk ch of rows r0 + 32 i
    if (C::B_RES) {
      // resident weights: KB k-blocks of [B_ROWS x 64] (hi rows, then lo rows)
      for (int idx = pt; idx < KB * C::B_ROWS * 8; idx += kProd) {
        const int kb = idx / (C::B_ROWS * 8), rem = idx - kb * (C::B_ROWS * 8), r = rem >> 3, c = rem & 7;
        const uint32_t off = uint32_t(kb) * (C::B_ROWS * 128) + sw128_off(r, c);
        const uint8_t *src = static_cast<const uint8_t *>(r < BN ? p.b_hi : p.b_lo);
        cp_async16(res + off, src + ((long long)(r % BN) * C::WROW) * EB + (kb + C::KB0) * 128 + c * 16);
      }
      cp_commit();
      cp_wait<0>();
      fence_proxy_async();
      mbar_arrive(wready_bar);
    }
    if constexpr (LAYER == 1 && FUSED) {
      // conv1 operand rendered from node states (channel kb = history slot kb),
      // all KB stages of a tile at once.  An im2col row is zero unless one of
      // the 2 x 2 cells its 8 x 8 patch covers holds an object, so the tiles
      // stay zero and only the rows next to the <= 4 objects of the <= 2 nodes
      // a tile's 128 rows touch are rendered.  Candidate = (slot kb, node li,
      // object k, patch offset dy dx, 16-byte chunk cc): this thread owns
      // (li, k, dy, dx, cc) = its index and the 4 slots; duplicates write
      // identical bytes.  What a thread wrote into a stage is re-zeroed when
      // the stage next comes round (S = RING x KB: every RING-th tile).
      static_assert(!(LAYER == 1 && FUSED) || (S == C::RING * KB && C::RING * KB * kProd <= 8 * 256),
                    "ring of RING tiles");
      for (int idx = pt; idx < S * (C::STAGE_BYTES / 16); idx += kProd)
        st_shared16(stage0 + uint32_t(idx) * 16u, make_uint4(0u, 0u, 0u, 0u));
      for (int j = 0; j < 8; ++j) dirty[j * kProd + pt] = 0u;
      const int li = pt >> 7, k = (pt >> 5) & 3, dy = (pt >> 4) & 1, dx = (pt >> 3) & 1, cc = pt & 7;
      // node states of a tile's <= 2 nodes, fetched two tiles ahead into a ring of
      // three; every tile commits one cp.async group (possibly empty), so at the
      // start of a tile exactly its own group and the next one are outstanding.
      // The fetch is issued after the tile's proxy fence so the fence never waits
      // for it.
      const uint32_t ring = smem_u32(dirty + 8 * kProd);
      auto prefetch_states = [&](int t, int slot) {
        if (pt < 10) {
          const uint32_t m0 = uint32_t(t) * 128u;
          const uint32_t mlast = (m0 + 127u < p.M - 1u) ? m0 + 127u : p.M - 1u;
          const uint32_t leaf0 = m0 / uint32_t(kP1), leaf_last = mlast / uint32_t(kP1);
          const uint32_t l = (leaf0 + uint32_t(pt / 5) <= leaf_last) ? leaf0 + uint32_t(pt / 5) : leaf_last;
          cp_async16(ring + uint32_t(slot * 160 + pt * 16),
                     reinterpret_cast<const uint4 *>(p.a_hi) + size_t(l) * 5 + (pt % 5));
        }
        cp_commit();
      };
      if (T0 < TE) prefetch_states(T0, 0);
      else cp_commit();
      if (T0 + TS < TE) prefetch_states(T0 + TS, 1);
      else cp_commit();
      int c = 0;  // tiles so far
      for (int t = T0; t < TE; t += TS, ++c) {
        {
          // the MMA thread commits once per tile, to the tile's last stage: its
          // completion frees all KB stages (and those of every earlier tile)
          const int gl = c * KB + KB - 1;
          const int s = gl % S;
          const uint32_t round = uint32_t(gl / S);
          wait_bar(empty_bar(s), (round & 1u) ^ 1u, abort_flag, p.d_err, 1);
        }
        named_bar_sync(1, kProd);  // every producer decides together
        if (*abort_flag) break;
        cp_wait<1>();  // this tile's node states (the next tile's may still be in flight)
        uint32_t *dj = dirty + (c % C::RING) * (KB * kProd);
#pragma unroll
        for (int j = 0; j < KB; ++j) {
          const uint32_t a = dj[j * kProd + pt];
          if (a) st_shared16(a, make_uint4(0u, 0u, 0u, 0u));
        }
        named_bar_sync(1, kProd);  // states visible, re-zeroing done
        uint4 P[4];
        const uint4 *Ps = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint8_t *>(dirty + 8 * kProd) +
                                                          (c % 3) * 160 + li * 80);
#pragma unroll
        for (int j = 0; j < 4; ++j) P[j] = Ps[j];
        const uint32_t m0 = uint32_t(t) * 128u;
        const uint32_t mlast = (m0 + 127u < p.M - 1u) ? m0 + 127u : p.M - 1u;
        const uint32_t leaf0 = m0 / uint32_t(kP1), leaf_last = mlast / uint32_t(kP1);
        // bf16: K block j = history slot j, chunk cc = kernel row cc (8 pixels);
        // E4M3: K block j = slots 2j, 2j+1, chunk cc = slot 2j + cc/4, kernel rows
        // 2(cc%4) and 2(cc%4)+1 (16 pixels)
#pragma unroll
        for (int j = 0; j < KB; ++j) {
          uint32_t wrote = 0u;
          const uint32_t leaf = leaf0 + uint32_t(li);
          const int slot = FP8 ? 2 * j + (cc >> 2) : j;
          // the slot depends on the chunk (E4M3): read it from the state ring, not
          // from a runtime-indexed register array (which would live in local memory)
          const uint4 Pv = FP8 ? Ps[slot & 3] : P[slot & 3];
          const uint32_t wk = (k & 2) ? ((k & 1) ? Pv.w : Pv.z) : ((k & 1) ? Pv.y : Pv.x);
          const int ox = int(int16_t(wk & 0xFFFFu)) - dx, oy = int(int16_t(wk >> 16)) - dy;
          const uint32_t m = leaf * uint32_t(kP1) + uint32_t(oy * 20 + ox);
          if (slot <= 3 && leaf <= leaf_last && ox >= 0 && ox <= 19 && oy >= 0 && oy <= 19 && m >= m0 &&
              m <= mlast) {
            int oxs[4], oys[4];
            unpack_slot(Pv, oxs, oys);
            uint4 v;
            if (FP8) {
              const int y = 4 * oy + 2 * (cc & 3);
              const uint32_t w[4] = {render_word(oxs, oys, ox, y), render_word(oxs, oys, ox + 1, y),
                                     render_word(oxs, oys, ox, y + 1), render_word(oxs, oys, ox + 1, y + 1)};
              v = pixels16_to_e4m3(w);
            } else {
              const int y = 4 * oy + cc;
              v = pixels8_to_bf16(render_word(oxs, oys, ox, y), render_word(oxs, oys, ox + 1, y));
            }
            wrote = sA_of((c * KB + j) % S) + sw128_off(int(m - m0), cc);
            st_shared16(wrote, v);
          }
          dj[j * kProd + pt] = wrote;
        }
        fence_proxy_async();
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) mbar_arrive(full_bar((c * KB + kb) % S));
        if (t + 2 * TS < TE) prefetch_states(t + 2 * TS, (c + 2) % 3);
        else cp_commit();
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
    } else if constexpr (C::C1) {
      // conv1 from rendered frames, one K block of one tile per stage.  Thread pt
      // fills row pt / 2 of the tile, chunks 4 (pt % 2) .. + 3: bf16, chunk ch =
      // 8 pixels of kernel row ch of weight channel CH0 + kb; E4M3, chunk ch = 16
      // pixels of kernel rows 2(ch%4), 2(ch%4)+1 of weight channel
      // 2 (KB0 + kb) + ch/4 (channels outside the tile's range stay zero).  The
      // row's frame address is computed once per stage, and neighbouring lanes
      // read neighbouring pixels.  The next stages' pixel words are loaded into
      // registers before this stage is converted and stored.
      constexpr int NW = FP8 ? 4 : 2;  // 32-bit pixel words per 16-byte chunk
      // E4M3 K blocks hold two slots; where only one is live (layer 6: channel 3
      // beside a zero channel 2; layer 5's second block: channel 2 beside a zero
      // channel 3) the row's two threads take two live chunks (kernel row pairs
      // 2 half, 2 half + 1) and two zero chunks each, not one slot each
      const int row = pt >> 1, half = pt & 1;
      // for K block kb: exactly one live slot? its slot index and first chunk
      auto bal_of = [&](int kb, int &lsl, int &lbase) {
        const int s0 = 2 * (C::KB0 + kb) - C::CH0, s1 = s0 + 1;
        const bool l0 = s0 >= 0 && s0 < C::NCH, l1 = s1 >= 0 && s1 < C::NCH;
        lsl = l0 ? s0 : s1;
        lbase = l0 ? 0 : 4;
        return FP8 && l0 != l1;
      };
      auto live_of = [&](int kb) {
        const int sl = FP8 ? 2 * (C::KB0 + kb) + half - C::CH0 : kb;
        return sl >= 0 && sl < C::NCH;
      };
      auto load_stage = [&](int t, int kb, uint32_t(&w)[4][NW]) {
        const uint32_t m0 = uint32_t(t / NT) * 128u;
        int lsl, lbase;
        const bool BAL = bal_of(kb, lsl, lbase);
        const int sl = BAL ? lsl : (FP8 ? 2 * (C::KB0 + kb) + half - C::CH0 : kb);  // A slot
        const bool live = sl >= 0 && sl < C::NCH;
        const int sc = live ? sl : 0;
        uint32_t m = m0 + uint32_t(row);
        if (m > p.M - 1u) m = p.M - 1u;
        const uint32_t node = m / uint32_t(kP1);
        const int px = int(m - node * uint32_t(kP1)), oy = px / 20, ox = px - oy * 20;
        const uint32_t nd = p.node0 + node, fd = p.fdiv[sc];
        const uint8_t *frame = p.fsrc[sc] + size_t((fd == 1u ? nd : nd / fd) - p.fsub[sc]) * p.fstride[sc] +
                               (4 * oy) * 84 + 4 * ox;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (FP8) {
            const uint8_t *src = frame + 2 * (BAL ? 2 * half + (j & 1) : j) * 84;
#pragma unroll
            for (int k = 0; k < NW; ++k) w[j][k] = 0u;
            if (BAL ? j < 2 : live) {
              w[j][0] = __ldg(reinterpret_cast<const uint32_t *>(src));
              w[j][1] = __ldg(reinterpret_cast<const uint32_t *>(src + 4));
              w[j][NW > 2 ? 2 : 0] = __ldg(reinterpret_cast<const uint32_t *>(src + 84));
              w[j][NW > 3 ? 3 : 0] = __ldg(reinterpret_cast<const uint32_t *>(src + 88));
            }
          } else {
            const uint8_t *src = frame + (4 * half + j) * 84;
            w[j][0] = __ldg(reinterpret_cast<const uint32_t *>(src));
            w[j][1] = __ldg(reinterpret_cast<const uint32_t *>(src + 4));
          }
        }
      };
      // stage positions (tile, K block) in issue order; two stages' loads stay in
      // flight ahead of the one being stored (three register buffers in rotation)
      struct Pos {
        int t, kb;
      };
      auto adv = [&](Pos q) {
        if (++q.kb == KB) {
          q.kb = 0;
          q.t += TS;
        }
        return q;
      };
      int g = 0;
      auto consume = [&](const Pos &q, const uint32_t(&w)[4][NW]) {
        const int s = g % S;
        if (!wait_bar(empty_bar(s), uint32_t((g / S) & 1) ^ 1u, abort_flag, p.d_err, 1)) return false;
        const uint32_t sA = sA_of(s);
        int lsl, lbase;
        const bool BAL = bal_of(q.kb, lsl, lbase);
        const bool live = BAL || live_of(q.kb);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          uint4 v = make_uint4(0u, 0u, 0u, 0u);
          if (FP8) {
            if (BAL ? j < 2 : live) {
              const uint32_t w4[4] = {w[j][0], w[j][1], w[j][NW > 2 ? 2 : 0], w[j][NW > 3 ? 3 : 0]};
              v = pixels16_to_e4m3(w4);
            }
          } else {
            v = pixels8_to_bf16(w[j][0], w[j][1]);
          }
          // BAL: live chunks lbase + 2 half + j (j < 2), zero chunks in the other half
          const int chunk = BAL ? (j < 2 ? lbase + 2 * half + j : (4 - lbase) + 2 * half + j - 2) : 4 * half + j;
          st_shared16(sA + sw128_off(row, chunk), v);
        }
        fence_proxy_async();
        mbar_arrive(full_bar(s));
        ++g;
        return true;
      };
      uint32_t b0[4][NW], b1[4][NW], b2[4][NW];
      Pos p0{T0, 0}, p1 = adv(p0), p2 = adv(p1);
      if (p0.t < TE) load_stage(p0.t, p0.kb, b0);
      if (p1.t < TE) load_stage(p1.t, p1.kb, b1);
      for (;;) {
        if (p0.t >= TE) break;
        if (p2.t < TE) load_stage(p2.t, p2.kb, b2);
        if (!consume(p0, b0)) break;
        p0 = p1, p1 = p2, p2 = adv(p2);
        if (p0.t >= TE) break;
        if (p2.t < TE) load_stage(p2.t, p2.kb, b0);
        if (!consume(p0, b1)) break;
        p0 = p1, p1 = p2, p2 = adv(p2);
        if (p0.t >= TE) break;
        if (p2.t < TE) load_stage(p2.t, p2.kb, b1);
        if (!consume(p0, b2)) break;
        p0 = p1, p1 = p2, p2 = adv(p2);
      }
    } else {
      // every stage's copies stay in flight until they land; the full barrier
      // counts one hardware arrival per producer thread at that moment
      int g = 0;
      bool ok = true;
      for (int t = T0; t < TE && ok; t += TS) {
        const uint32_t m0 = uint32_t(t / NT) * 128u;
        const int n0 = (t % NT) * BN;
        // per-row source offsets for this tile (rows r0 + 32 i)
        long long rowoff[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          uint32_t m = m0 + uint32_t(r0 + 32 * i);
          if (m > p.M - 1u) m = p.M - 1u;
          const uint32_t leaf = m / uint32_t(G::P);
          const int px = int(m - leaf * uint32_t(G::P));
          if (LAYER == 2) {
            const int oy = px / 9, ox = px - oy * 9;
            rowoff[i] = (long long)leaf * (kP1 * kC1) + (2 * oy * 20 + 2 * ox) * kC1;
          } else if (LAYER == 3) {
            const int oy = px / 7, ox = px - oy * 7;
            rowoff[i] = (long long)leaf * (kP2 * kC2) + (oy * 9 + ox) * kC2;
          } else {
            rowoff[i] = (long long)m * kKF;
          }
        }
        for (int ks = 0; ks < C::NKS; ++ks) {
          const int s = g % S;
          const uint32_t round = uint32_t(g / S);
          if (!wait_bar(empty_bar(s), (round & 1u) ^ 1u, abort_flag, p.d_err, 1)) {
            ok = false;
            break;
          }
#pragma unroll
          for (int kk = 0; kk < C::KPS; ++kk) {
          const int kb = ks * C::KPS + kk;
          if (kb >= KB) break;
          const uint32_t sA = sub_of(s, kk);
          const uint32_t sAlo = sA + C::A_BYTES;
          const uint32_t sB = sB_of(s, kk);
          const uint32_t sBlo = sB + C::B_BYTES;
          // A tile: im2col rows of the NHWC activation map
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint32_t off = sw128_off(r0 + 32 * i, ch);
            long long e;  // element offset; a 16-byte chunk is 8 bf16 or 16 E4M3 elements
            if (FP8) {
              if (LAYER == 2) {  // K block = 4 kernel positions x 32 channels
                const int pos = 4 * kb + (ch >> 1), ky = pos >> 2, kx = pos & 3;
                e = rowoff[i] + (ky * 20 + kx) * kC1 + (ch & 1) * 16;
              } else if (LAYER == 3) {  // 2 positions x 64 channels; position 9 is padding
                int pos = 2 * kb + (ch >> 2);
                pos = pos > 8 ? 8 : pos;  // any finite data: the padded weights are zero
                const int ky = pos / 3, kx = pos - 3 * (pos / 3);
                e = rowoff[i] + (ky * 9 + kx) * kC2 + (ch & 3) * 16;
              } else {  // fc1: K padded from 3136 to 3200
                int off = kb * 128 + ch * 16;
                off = off >= kKF ? off - 64 : off;
                e = rowoff[i] + off;
              }
            } else if (LAYER == 2) {
              const int pos = 2 * kb + (ch >> 2), ky = pos >> 2, kx = pos & 3;
              e = rowoff[i] + (ky * 20 + kx) * kC1 + (ch & 3) * 8;
            } else if (LAYER == 3) {
              const int ky = kb / 3, kx = kb - 3 * (kb / 3);
              e = rowoff[i] + (ky * 9 + kx) * kC2 + ch * 8;
            } else {
              e = rowoff[i] + kb * 64 + ch * 8;
            }
            cp_async16(sA + off, static_cast<const uint8_t *>(p.a_hi) + e * EB);
            if (C::A_LO) cp_async16(sAlo + off, static_cast<const uint8_t *>(p.a_lo) + e * EB);
          }
          // B tile (weights, [NTOT][K] K-major): hi rows, then lo rows
#pragma unroll
          for (int i = 0; i < (C::B_RES ? 0 : BN / 32); ++i) {
            const int r = r0 + 32 * i;
            const uint32_t off = sw128_off(r, ch);
            const long long eb = ((long long)(n0 + r) * C::KPAD) * EB + kb * 128 + ch * 16;  // bytes
            cp_async16(sB + off, static_cast<const uint8_t *>(p.b_hi) + eb);
            if (SPLIT) cp_async16(sBlo + off, static_cast<const uint8_t *>(p.b_lo) + eb);
          }
          }
          cp_async_arrive(full_bar(s));
          ++g;
        }
      }
      asm volatile("cp.async.wait_all;" ::: "memory");  // nothing may still be landing at teardown
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc_wide = idesc_bf16(C::B_CAT ? 2 * BN : BN);  // [hi; lo] weight rows
      constexpr uint32_t idesc_n = FP8 ? idesc_e4m3(BN) : idesc_bf16(BN);
      const uint64_t stage_desc = sw128_desc(stage0), res_desc = sw128_desc(res);
      int g = 0, it = 0;
      bool ok = true;
      if (C::B_RES) ok = wait_bar(wready_bar, 0, abort_flag, p.d_err, 6);
      for (int t = T0; t < TE && ok; t += TS, ++it) {
        const int acc = it % NA;
        if (!wait_bar(tempty_bar(acc), (uint32_t((it / NA) & 1)) ^ 1u, abort_flag, p.d_err, 2)) break;
        tc_fence_after();
        const uint32_t d = tmem + uint32_t(acc * C::ACC_N);
        // cp.async-fed stages were written through the generic proxy and the
        // hardware arrival carries no proxy fence: one fence per group of F
        // stages orders them before the tensor core's async-proxy reads.  conv1's
        // producers write with st.shared and fence themselves.
        constexpr bool kFence = !C::C1;
        constexpr int F = (kFence && S >= 4) ? C::FGROUP : 1;
        constexpr bool kTileCommit = LAYER == 1 && FUSED;  // one commit frees the tile's stages
        for (int ks0 = 0; ks0 < C::NKS && ok; ks0 += F) {
          const int nf = (C::NKS - ks0) < F ? (C::NKS - ks0) : F;
          for (int f = 0; f < nf; ++f) {
            const int sf = (g + f) % S;
            if (!wait_bar(full_bar(sf), uint32_t((g + f) / S) & 1u, abort_flag, p.d_err, 3)) {
              ok = false;
              break;
            }
          }
          if (!ok) break;
          if (kFence) fence_proxy_async();
          tc_fence_after();
          for (int f = 0; f < nf; ++f) {
          const int ks = ks0 + f;
          const int s = g % S;
#pragma unroll
          for (int kk = 0; kk < C::KPS; ++kk) {
          const int kb = ks * C::KPS + kk;
          if (kb >= KB) break;
          // descriptors differ only in their start-address field (address / 16):
          // offsets from the stage area's and the resident weights' descriptors
          const uint64_t ad = stage_desc + uint64_t((uint32_t(s) * C::STAGE_BYTES + uint32_t(kk) * C::SUB_BYTES) >> 4);
          const uint64_t bd = C::B_RES ? res_desc + uint64_t((uint32_t(kb) * (C::B_ROWS * 128)) >> 4)
                                       : ad + uint64_t(uint32_t(C::A_BYTES * (C::A_LO ? 2 : 1)) >> 4);
          constexpr uint64_t kAlo = uint64_t(uint32_t(C::A_BYTES) >> 4), kBlo = uint64_t(uint32_t(C::B_BYTES) >> 4);
#pragma unroll
          for (int j = 0; j < 4; ++j) {  // K = 16 bf16 / 32 E4M3 = 32 bytes per instruction
            const uint32_t first = (kb != 0 || j != 0) ? 1u : 0u;
            const uint64_t a = ad + uint64_t(2 * j);
            const uint64_t b = bd + uint64_t(2 * j);
            if (FP8) {
              mma_f8(d, a, b, idesc_n, first);
            } else if (C::B_CAT) {
              mma_bf16(d, a, b, idesc_wide, first);  // [A_hi B_hi | A_hi B_lo]
              if (C::A_LO) mma_bf16(d, a + kAlo, b, idesc_n, 1u);  // + A_lo B_hi
            } else {
              mma_bf16(d, a, b, idesc_n, first);
              if (SPLIT) {
                mma_bf16(d, a, b + kBlo, idesc_n, 1u);
                if (C::A_LO) mma_bf16(d, a + kAlo, b, idesc_n, 1u);
              }
            }
          }
          }
          if (!kTileCommit || ks == C::NKS - 1) mma_commit(empty_bar(s));  // stage(s) free once read
          ++g;
          }
        }
        if (!ok) break;
        mma_commit(tfull_bar(acc));
      }
      // drain: this commit completes once every MMA issued above has finished
      // (also after an abort), so TMEM and shared memory can be released
      mma_commit(drain_bar);
      const long long t0 = clock64();
      while (!mbar_try(drain_bar, 0)) {
        __nanosleep(64);
        if (clock64() - t0 > kWaitCycles) {
          if (p.d_err) atomicCAS(p.d_err, 0, 5);
          break;
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    // Each warp owns 32 accumulator rows (its TMEM lane quarter).  Results are
    // staged row by row in shared memory and written out as contiguous 16-byte
    // segments, so every global store instruction covers whole lines.
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    float *scale_s = bias_s + G::NTOT;
    const int eg = (warp - kEpiWarp0) >> 2;  // warpgroup: tiles it with it % EPI_WG == eg
    for (int i = threadIdx.x - 32 * kEpiWarp0; i < G::NTOT; i += 128 * C::EPI_WG) {
      bias_s[i] = LAYER == 6 ? 0.f : p.bias[i];  // layer 6: the parent's partial map carries the bias
      scale_s[i] = FP8 ? p.colscale[i] : 1.f;
    }
    named_bar_sync(2, 128 * C::EPI_WG);
    uint8_t *stg = reinterpret_cast<uint8_t *>(bias_s + 2 * G::NTOT) + (warp - kEpiWarp0) * (32 * kStgRow);
    // output row bytes of one array (conv layers: whole rows; fc1: one 16-column chunk)
    constexpr int ROWB = LAYER == 4 ? 64 : (LAYER == 5 ? BN * 4 : (FP8 ? BN : BN * 2));
    constexpr int SEGS = ROWB / 16;  // 16-byte segments per row
    static_assert(ROWB + 16 <= kStgRow && kC1 * 4 + 16 <= kStgRow, "staging row");
    // write the warp's 32 staged rows (ROWB bytes each) to dst rows of `stride` bytes
    auto flush = [&](uint8_t *dst, size_t stride, uint32_t mw0) {
      __syncwarp();
#pragma unroll
      for (int i = 0; i < SEGS; ++i) {
        const int k = lane + 32 * i, r = k / SEGS, sgm = k - r * SEGS;
        if (mw0 + uint32_t(r) < p.M)
          *reinterpret_cast<uint4 *>(dst + size_t(mw0 + r) * stride + sgm * 16) =
              *reinterpret_cast<const uint4 *>(stg + r * kStgRow + sgm * 16);
      }
      __syncwarp();
    };
    constexpr int EW = C::EPI_WG;
    int it = eg;
    for (int t = T0 + eg * TS; t < TE; t += EW * TS, it += EW) {
      const int acc = it % NA;
      // layer 6: the warp's 32 rows of their parents' partial maps (FP32, 32
      // columns = 128 bytes a row), loaded before the wait so that the latency
      // overlaps the MMAs, and coalesced: load i of lane l is the 16-byte piece
      // l % 8 of row l / 8 + 4 i
      float4 zr[LAYER == 6 ? 8 : 1];
      if constexpr (LAYER == 6) {
        uint32_t m = uint32_t(t / NT) * 128u + uint32_t(q * 32 + lane);
        if (m > p.M - 1u) m = p.M - 1u;
        const uint32_t node = m / uint32_t(kP1), px = m - node * uint32_t(kP1);
        const uint32_t par = p.zparent ? __ldg(p.zparent + p.zleaf0 + node) : (p.zleaf0 + node) / p.zbranch;
        const float4 *zrow = reinterpret_cast<const float4 *>(p.zmap + (size_t(par) * kP1 + px) * kC1);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float4 *src = reinterpret_cast<const float4 *>(
              __shfl_sync(0xffffffffu, reinterpret_cast<uintptr_t>(zrow), (lane >> 3) + 4 * i));
          zr[i] = __ldg(src + (lane & 7));
        }
      }
      if (!wait_bar(tfull_bar(acc), uint32_t((it / NA) & 1), abort_flag, p.d_err, 4)) break;
      tc_fence_after();
      if constexpr (LAYER == 6) {
        // The accumulator rows (FP32; split mode: the sum of its two halves) pass
        // through the staging rows once; lane l then takes columns 4 (l % 8) .. + 3
        // of rows l / 8 + 4 i, the layout its parent-map pieces were loaded in,
        // adds them (the map holds the bias), applies the ReLU, rounds and stores
        // to the NHWC map: consecutive lanes write consecutive bytes.
        const uint32_t mw0 = uint32_t(t / NT) * 128u + uint32_t(q * 32);
        const uint32_t tbase = tmem + (uint32_t(q * 32) << 16) + uint32_t(acc * C::ACC_N);
#pragma unroll
        for (int j = 0; j < BN / 16; ++j) {
          uint32_t r[16];
          tmem_ld16(tbase + uint32_t(j * 16), r);
          float v[16];
          if (C::B_CAT) {
            uint32_t r2[16];  // the A_hi * B_lo half
            tmem_ld16(tbase + uint32_t(BN + j * 16), r2);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const float2 x = add2(make_float2(__uint_as_float(r[2 * e]), __uint_as_float(r[2 * e + 1])),
                                    make_float2(__uint_as_float(r2[2 * e]), __uint_as_float(r2[2 * e + 1])));
              v[2 * e] = x.x;
              v[2 * e + 1] = x.y;
            }
          } else {
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
          }
#pragma unroll
          for (int e = 0; e < 4; ++e)
            *reinterpret_cast<float4 *>(stg + lane * kStgRow + j * 64 + e * 16) =
                make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty_bar(acc));  // the accumulator is in the staging rows
        const int pc = lane & 7;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int rr = (lane >> 3) + 4 * i;
          float4 a = *reinterpret_cast<const float4 *>(stg + rr * kStgRow + pc * 16);
          float2 lo2 = make_float2(a.x, a.y), hi2 = make_float2(a.z, a.w);
          if (FP8) {  // per-column weight x input scale of the E4M3 product
            const float4 s4 = *reinterpret_cast<const float4 *>(scale_s + 4 * pc);
            lo2 = mul2(lo2, make_float2(s4.x, s4.y));
            hi2 = mul2(hi2, make_float2(s4.z, s4.w));
          }
          lo2 = add2(lo2, make_float2(zr[i].x, zr[i].y));
          hi2 = add2(hi2, make_float2(zr[i].z, zr[i].w));
          const uint32_t m = mw0 + uint32_t(rr);
          if (m >= p.M) continue;
          if constexpr (FP8) {
            const float2 inv = make_float2(p.out_inv_scale, p.out_inv_scale);
            *reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(p.out_hi) + size_t(m) * BN + pc * 4) =
                relu_e4m3x4(mul2(lo2, inv), mul2(hi2, inv));
          } else if constexpr (SPLIT) {
            // hi = bf16(relu(v)), lo = bf16(relu(v) - hi)
            uint32_t hw[2], lw[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float2 y = h ? hi2 : lo2;
              const float2 x = make_float2(fmaxf(y.x, 0.f), fmaxf(y.y, 0.f));
              const __nv_bfloat162 hb = __floats2bfloat162_rn(x.x, x.y);
              hw[h] = *reinterpret_cast<const uint32_t *>(&hb);
              const float2 d = fma2(__bfloat1622float2(hb), make_float2(-1.f, -1.f), x);  // exact, one rounding
              const __nv_bfloat162 lb = __floats2bfloat162_rn(d.x, d.y);
              lw[h] = *reinterpret_cast<const uint32_t *>(&lb);
            }
            *reinterpret_cast<uint2 *>(static_cast<uint8_t *>(p.out_hi) + size_t(m) * BN * 2 + pc * 8) =
                make_uint2(hw[0], hw[1]);
            *reinterpret_cast<uint2 *>(static_cast<uint8_t *>(p.out_lo) + size_t(m) * BN * 2 + pc * 8) =
                make_uint2(lw[0], lw[1]);
          } else {
            *reinterpret_cast<uint2 *>(static_cast<uint8_t *>(p.out_hi) + size_t(m) * BN * 2 + pc * 8) =
                make_uint2(relu_bf16x2(lo2), relu_bf16x2(hi2));
          }
        }
        __syncwarp();  // the staging rows are read before the next tile writes them
        continue;
      }
      const uint32_t mw0 = uint32_t(t / NT) * 128u + uint32_t(q * 32);
      const int n0 = (t % NT) * BN;
      const uint32_t tbase = tmem + (uint32_t(q * 32) << 16) + uint32_t(acc * C::ACC_N);
      // this thread's output row: hi part staged as it is produced, lo part kept
      // in registers until the hi rows are written
      constexpr int OW = LAYER == 4 ? 1 : (FP8 ? BN / 4 : BN / 2);
      uint32_t olo[SPLIT && LAYER != 4 ? OW : 1];
      // fc1 in the split mode: this row's fc2 partial sums over the tile's 256
      // columns (BF16 / E4M3, whose fc1 MMAs are shorter than this arithmetic,
      // write the FP32 map for fc2_max_kernel instead)
      constexpr bool FOLD = LAYER == 4 && SPLIT;
      float qs[FOLD ? kMaxA : 1];
#pragma unroll
      for (int a = 0; a < (FOLD ? kMaxA : 1); ++a) qs[a] = 0.f;
      // then the 16 chunks stay a rolled loop: unrolled, the fc2 sums and the
      // chunks' loads overlapped beyond the 128 registers of this 13-warp CTA
#pragma unroll(FOLD ? 1 : BN / 16)
      for (int j = 0; j < BN / 16; ++j) {
        uint32_t r[16];
        tmem_ld16(tbase + uint32_t(j * 16), r);
        float2 v[8];  // columns 2e, 2e + 1 of this 16-column chunk
        if (C::B_CAT) {
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
        // per-column scale (E4M3 accumulators carry the weight and input scales)
        // plus bias
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int n = n0 + j * 16 + 4 * e;
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
        if constexpr (LAYER == 5) {  // partial map: FP32, no ReLU
#pragma unroll
          for (int e = 0; e < 4; ++e)
            *reinterpret_cast<float4 *>(stg + lane * kStgRow + j * 64 + e * 16) =
                make_float4(v[2 * e].x, v[2 * e].y, v[2 * e + 1].x, v[2 * e + 1].y);
        } else if constexpr (FOLD) {
          // h = ReLU(v) for these 16 columns, folded straight into fc2: qs[a] +=
          // h . W2[a][n0 + 16 j ..] (every lane reads the same weights: broadcast)
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = make_float2(fmaxf(v[e].x, 0.f), fmaxf(v[e].y, 0.f));
#pragma unroll
          for (int a = 0; a < kMaxA; ++a) {
            if (a < p.fA) {
              const float4 *wr = reinterpret_cast<const float4 *>(p.w2 + size_t(a) * G::NTOT + n0 + j * 16);
              float acc_a = qs[a];
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const float4 w4 = __ldg(wr + k);
                acc_a = fmaf(v[2 * k].x, w4.x, acc_a);
                acc_a = fmaf(v[2 * k].y, w4.y, acc_a);
                acc_a = fmaf(v[2 * k + 1].x, w4.z, acc_a);
                acc_a = fmaf(v[2 * k + 1].y, w4.w, acc_a);
              }
              qs[a] = acc_a;
            }
          }
        } else if constexpr (LAYER == 4) {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            *reinterpret_cast<float4 *>(stg + lane * kStgRow + e * 16) =
                make_float4(fmaxf(v[2 * e].x, 0.f), fmaxf(v[2 * e].y, 0.f), fmaxf(v[2 * e + 1].x, 0.f),
                            fmaxf(v[2 * e + 1].y, 0.f));
          flush(static_cast<uint8_t *>(p.out_hi) + (size_t(n0) + j * 16) * 4, size_t(G::NTOT) * 4, mw0);
        } else if constexpr (FP8) {
          // ReLU, then the output map's activation scale (positive, so the order is free)
          const float2 inv = make_float2(p.out_inv_scale, p.out_inv_scale);
          uint32_t w[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) w[h] = relu_e4m3x4(mul2(v[2 * h], inv), mul2(v[2 * h + 1], inv));
          *reinterpret_cast<uint4 *>(stg + lane * kStgRow + j * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
          uint32_t hh[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            if constexpr (SPLIT) {
              // hi = bf16(relu(v)), lo = bf16(relu(v) - hi)
              const float2 x = make_float2(fmaxf(v[e].x, 0.f), fmaxf(v[e].y, 0.f));
              const __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
              hh[e] = *reinterpret_cast<const uint32_t *>(&h);
              const float2 d = fma2(__bfloat1622float2(h), make_float2(-1.f, -1.f), x);  // exact product, one rounding
              const __nv_bfloat162 l = __floats2bfloat162_rn(d.x, d.y);
              olo[j * 8 + e] = *reinterpret_cast<const uint32_t *>(&l);
            } else {
              hh[e] = relu_bf16x2(v[e]);
            }
          }
          *reinterpret_cast<uint4 *>(stg + lane * kStgRow + j * 32) = make_uint4(hh[0], hh[1], hh[2], hh[3]);
          *reinterpret_cast<uint4 *>(stg + lane * kStgRow + j * 32 + 16) = make_uint4(hh[4], hh[5], hh[6], hh[7]);
        }
      }
      if constexpr (FOLD) {
        const uint32_t m = mw0 + uint32_t(lane);
        if (m < p.M) {
          float *dst = p.qpart + (size_t(m) * NT + size_t(t % NT)) * kMaxA;
#pragma unroll
          for (int a = 0; a < kMaxA; ++a)
            if (a < p.fA) dst[a] = qs[a];
        }
      }
      if constexpr (LAYER != 4) {
        flush(static_cast<uint8_t *>(p.out_hi), size_t(ROWB), mw0);
        if constexpr (SPLIT && LAYER != 5) {
#pragma unroll
          for (int i = 0; i < OW / 4; ++i)
            *reinterpret_cast<uint4 *>(stg + lane * kStgRow + i * 16) =
                make_uint4(olo[4 * i], olo[4 * i + 1], olo[4 * i + 2], olo[4 * i + 3]);
          flush(static_cast<uint8_t *>(p.out_lo), size_t(ROWB), mw0);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar(acc));
    }
  }
  // teardown: every role has left its loop (all waits are bounded)
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int num_sms() {
  static int sms = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 148;
  });
  return sms;
}

template <int LAYER, int MODE, bool FUSED>
int launch(const GemmParams &p0, long long M, int kind, cudaStream_t st) {
  using C = Cfg<LAYER, MODE>;
  if (M <= 0) return BCTS_OK;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(tc_gemm<LAYER, MODE, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    C::SMEM);
  });
  if (attr_err != cudaSuccess) return BCTS_ECUDA;
  if (M > 0x7FFFFFFFLL) return BCTS_EINVAL;
  GemmParams p = p0;
  p.M = uint32_t(M);
  const long long mt = (M + 127) / 128;
  const long long tiles = mt * (Geo<LAYER>::NTOT / Geo<LAYER>::BN);
  if (tiles > 0x7FFFFFFFLL) return BCTS_EINVAL;
  p.num_tiles = int(tiles);
  const int grid = int(tiles < num_sms() ? tiles : num_sms());
  ProfScope ps(kind, st);
  tc_gemm<LAYER, MODE, FUSED><<<grid, C::THREADS, C::SMEM, st>>>(p);
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

uint16_t f2bf(float f) {  // round to nearest even
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7FFFFFFFu) > 0x7F800000u) return 0x7FC0;
  const uint32_t r = 0x7FFFu + ((u >> 16) & 1u);
  return uint16_t((u + r) >> 16);
}
float bf2f(uint16_t h) {
  const uint32_t u = uint32_t(h) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

}  // namespace tc

struct TcWeights {
  int A = 0;
  int precision = 0;
  void *blob = nullptr;
  const void *w_hi[4] = {};  // conv1, conv2, conv3, fc1: bf16 hi (BF16 / split) or E4M3 (FP8), [rows][KPAD]
  const void *w_lo[4] = {};  // bf16 lo (split)
  const float *bias[4] = {};
  const float *colscale[4] = {};  // FP8: weight scale of each output channel x input activation scale
  float out_inv_scale[4] = {};    // FP8: 1 / activation scale of each layer's output map
  int kpad[4] = {};               // stored weight row length per layer (elements)
  const float *f2w = nullptr, *f2b = nullptr;
  // conv1 from the sprite tables (the weights as this precision multiplies them):
  const float *c1T = nullptr;  // [4 channels][4 objects][2 dy][2 dx][32] palette x W_c summed over the sprite
  const float *c1W = nullptr;  // [4 channels][64 patch pixels][32]
};

namespace {
constexpr int kWRows[4] = {32, 64, 64, 512};

// Value of an E4M3 code (1 sign, 4 exponent bits with bias 7, 3 mantissa bits;
// exponent 0 is subnormal; the saturated encoder never emits the NaN code).
float e4m3_value(uint8_t b) {
  const int e = (b >> 3) & 15, m = b & 7;
  const float mag = e == 0 ? std::ldexp(float(m), -9) : std::ldexp(float(8 + m), e - 10);
  return (b & 0x80) ? -mag : mag;
}
constexpr int kWK[4] = {256, 512, 576, 3136};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
}  // namespace

size_t tc_scratch_bytes(int64_t chunk, int precision) {
  const size_t maps = size_t(kP1) * kC1 + size_t(kP2) * kC2 + size_t(kP3) * kC3;  // elements per node
  const size_t bytes = precision == BCTS_PREC_FP32 ? 4 : (precision == BCTS_PREC_FP8 ? 1 : 2);
  return align256(size_t(chunk) * maps * bytes) + 3 * 256 + align256(size_t(chunk) * kF1 * 4) + 4096;
}

// `w` holds the weights in the CUDA-core layouts (conv1 pre-scaled by 1/255,
// conv2/conv3 K = (ky, kx, c), fc1 columns NHWC); the same orders serve here.
// act_scale (FP8 only): activation scales of the conv1, conv2, conv3 output maps.
int tc_weights_create(const float *w, int A, int precision, const float *act_scale, TcWeights **out,
                      std::string &err) {
  *out = nullptr;
  if (precision != BCTS_PREC_FP32 && precision != BCTS_PREC_BF16 && precision != BCTS_PREC_FP8) {
    err = "precision not available on the tensor-core path";
    return BCTS_ENOKERNEL;
  }
  const bool fp8 = precision == BCTS_PREC_FP8;
  if (fp8 && !act_scale) {
    err = "FP8 weights need activation scales";
    return BCTS_EINVAL;
  }
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) {
    cudaGetLastError();
    err = "tensor-core Q-network needs an sm_103 (B300) device";
    return BCTS_ENOKERNEL;
  }
  const float *src[4];
  const float *bsrc[4];
  src[0] = w;
  bsrc[0] = src[0] + 32 * 256;
  src[1] = bsrc[0] + 32;
  bsrc[1] = src[1] + 64 * 512;
  src[2] = bsrc[1] + 64;
  bsrc[2] = src[2] + 64 * 576;
  src[3] = bsrc[2] + 64;
  bsrc[3] = src[3] + size_t(512) * 3136;
  const float *f2w = bsrc[3] + 512;
  const float *f2b = f2w + size_t(A) * 512;
  int kpad[4];
  for (int l = 0; l < 4; ++l) kpad[l] = fp8 ? (kWK[l] + 127) / 128 * 128 : kWK[l];
  const size_t eb = fp8 ? 1 : 2;
  // blob: per layer [hi, lo] weights, then FP32 biases, column scales, fc2 weights and biases
  std::vector<size_t> off;
  size_t total = 0;
  for (int l = 0; l < 4; ++l) {
    off.push_back(total);
    total += align256(size_t(kWRows[l]) * kpad[l] * eb);
    off.push_back(total);
    total += align256(size_t(kWRows[l]) * kpad[l] * eb);
  }
  for (int l = 0; l < 8; ++l) {  // biases (0..3), column scales (4..7)
    off.push_back(total);
    total += align256(size_t(kWRows[l % 4]) * 4);
  }
  const size_t off_f2w = total;
  total += align256(size_t(A) * 512 * 4);
  const size_t off_f2b = total;
  total += align256(size_t(A) * 4);
  const size_t off_T = total;
  total += align256(size_t(kHist) * kObj * 4 * kC1 * 4);
  const size_t off_W3 = total;
  total += align256(size_t(kHist) * 64 * kC1 * 4);
  std::vector<uint8_t> h(total, 0);
  TcWeights *t = new TcWeights();
  for (int l = 0; l < 4; ++l) {
    const size_t R = kWRows[l], K = kWK[l], KP = kpad[l];
    if (fp8) {
      // per-output-channel scale: the row's max |w| maps to 448, E4M3's largest normal
      uint8_t *q = h.data() + off[2 * l];
      float *cs = reinterpret_cast<float *>(h.data() + off[12 + l]);
      const float s_in = l == 0 ? 1.f : act_scale[l - 1];  // conv1 reads raw pixel values
      for (size_t r = 0; r < R; ++r) {
        float mx = 0.f;
        for (size_t k = 0; k < K; ++k) mx = std::max(mx, std::fabs(src[l][r * K + k]));
        const float sw = mx > 0.f ? mx / 448.f : 1.f;
        for (size_t k = 0; k < K; ++k)
          q[r * KP + k] = uint8_t(__nv_cvt_float_to_fp8(src[l][r * K + k] / sw, __NV_SATFINITE, __NV_E4M3));
        cs[r] = sw * s_in;  // padded columns K..KP stay zero
      }
      t->out_inv_scale[l] = l < 3 ? 1.f / act_scale[l] : 1.f;
    } else {
      uint16_t *hi = reinterpret_cast<uint16_t *>(h.data() + off[2 * l]);
      uint16_t *lo = reinterpret_cast<uint16_t *>(h.data() + off[2 * l + 1]);
      for (size_t i = 0; i < R * K; ++i) {
        hi[i] = tc::f2bf(src[l][i]);
        lo[i] = tc::f2bf(src[l][i] - tc::bf2f(hi[i]));
      }
      float *cs = reinterpret_cast<float *>(h.data() + off[12 + l]);
      for (size_t r = 0; r < R; ++r) cs[r] = 1.f;
    }
    std::memcpy(h.data() + off[8 + l], bsrc[l], R * 4);
  }
  {
    // conv1's weights per input channel (K = channel * 64 + ky * 8 + kx) as this
    // precision multiplies them, and the per-object sprite sums
    float *Ws = reinterpret_cast<float *>(h.data() + off_W3);  // [channel][64][32]
    for (int hc = 0; hc < kHist; ++hc)
      for (int c = 0; c < kC1; ++c)
        for (int k = 0; k < 64; ++k) {
          const int kk = hc * 64 + k;
          float w;
          if (precision == BCTS_PREC_FP32) {
            w = src[0][c * 256 + kk];
          } else if (fp8) {
            const uint8_t code = h[off[0] + size_t(c) * kpad[0] + kk];
            w = e4m3_value(code) * reinterpret_cast<const float *>(h.data() + off[12])[c];
          } else {
            w = tc::bf2f(reinterpret_cast<const uint16_t *>(h.data() + off[0])[c * 256 + kk]);
          }
          Ws[(hc * 64 + k) * kC1 + c] = w;
        }
    float *T = reinterpret_cast<float *>(h.data() + off_T);  // [channel][object][dy][dx][32]
    for (int hc = 0; hc < kHist; ++hc)
      for (int o = 0; o < kObj; ++o)
        for (int dy = 0; dy < 2; ++dy)
          for (int dx = 0; dx < 2; ++dx)
            for (int c = 0; c < kC1; ++c) {
              double acc = 0.0;
              for (int sy = 0; sy < 4; ++sy)
                for (int sx = 0; sx < 4; ++sx)
                  if ((kSprites >> (16 * o + 4 * sy + sx)) & 1ull)
                    acc += double(Ws[(hc * 64 + (4 * dy + sy) * 8 + 4 * dx + sx) * kC1 + c]);
              T[(((hc * kObj + o) * 2 + dy) * 2 + dx) * kC1 + c] =
                  float(acc * double((kPalette >> (8 * o)) & 0xFFu));
            }
  }
  std::memcpy(h.data() + off_f2w, f2w, size_t(A) * 512 * 4);
  std::memcpy(h.data() + off_f2b, f2b, size_t(A) * 4);
  t->A = A;
  t->precision = precision;
  for (int l = 0; l < 4; ++l) t->kpad[l] = kpad[l];
  if (cudaMalloc(&t->blob, total) != cudaSuccess ||
      cudaMemcpy(t->blob, h.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    if (t->blob) cudaFree(t->blob);
    delete t;
    err = "tensor-core weight upload failed";
    return BCTS_ENOMEM;
  }
  uint8_t *b = static_cast<uint8_t *>(t->blob);
  for (int l = 0; l < 4; ++l) {
    t->w_hi[l] = b + off[2 * l];
    t->w_lo[l] = b + off[2 * l + 1];
    t->bias[l] = reinterpret_cast<const float *>(b + off[8 + l]);
    t->colscale[l] = reinterpret_cast<const float *>(b + off[12 + l]);
  }
  t->f2w = reinterpret_cast<const float *>(b + off_f2w);
  t->f2b = reinterpret_cast<const float *>(b + off_f2b);
  t->c1T = reinterpret_cast<const float *>(b + off_T);
  t->c1W = reinterpret_cast<const float *>(b + off_W3);
  *out = t;
  return BCTS_OK;
}

void tc_weights_destroy(TcWeights *w) {
  if (!w) return;
  if (w->blob) cudaFree(w->blob);
  delete w;
}

namespace {
void set_frames(tc::GemmParams &p, const FrameSrc &f) {
  for (int h = 0; h < kHist; ++h) {
    p.fsrc[h] = f.src[h];
    p.fdiv[h] = f.div[h] ? f.div[h] : 1u;
    p.fsub[h] = f.sub[h];
    p.fstride[h] = f.stride[h];
  }
  p.node0 = f.node0;
}

// fc2 after fc1's epilogue: q[node][a] = (partial of fc1 columns 0-255 +
// partial of columns 256-511) + b2[a], and the max over the node's first node_A
// actions (the batched form; else all A), the outputs launch_fc2_max gives.
__global__ void fc2_combine_kernel(const float *__restrict__ qpart, const float *__restrict__ b2, int A, int64_t n,
                                   float *__restrict__ q, float *__restrict__ maxq,
                                   const uint8_t *__restrict__ node_A) {
  const int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (node >= n) return;
  const float *p0 = qpart + node * (2 * kMaxA);
  const int An = node_A ? int(node_A[node]) : A;
  float best = -INFINITY;
  for (int a = 0; a < A; ++a) {
    const float v = (p0[a] + p0[kMaxA + a]) + __ldg(b2 + a);
    if (q) q[node * A + a] = v;
    if (a < An) best = fmaxf(best, v);
  }
  if (maxq) maxq[node] = best;
}

int launch_fc2_combine(const float *qpart, const float *b2, int A, int64_t n, float *q, float *maxq,
                       cudaStream_t st, const uint8_t *node_A) {
  if (n <= 0) return BCTS_OK;
  ProfScope ps(K_FC2, st);
  fc2_combine_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(qpart, b2, A, n, q, maxq, node_A);
  return cudaGetLastError() == cudaSuccess ? BCTS_OK : BCTS_ECUDA;
}

template <int MODE>
int tc_forward_impl(const TcWeights *w, int A, const uint8_t *frames, const bcts_state *states, int64_t n,
                    float *q, float *maxq, void *scratch, cudaStream_t st, int *d_err, const uint8_t *node_A,
                    const ZLeaf *zl, int conv_tma_mask, const FrameSrc *fs) {
  constexpr bool SPLIT = MODE == 1;
  const size_t eb = MODE == 2 ? 1 : 2;
  uint8_t *s = static_cast<uint8_t *>(scratch);
  auto take = [&](size_t bytes) {
    uint8_t *r = s;
    s += align256(bytes);
    return r;
  };
  const size_t m1 = size_t(n) * kP1 * kC1, m2 = size_t(n) * kP2 * kC2, m3 = size_t(n) * kP3 * kC3;
  void *a1 = take(m1 * eb), *a1l = SPLIT ? take(m1 * eb) : nullptr;
  void *a2 = take(m2 * eb), *a2l = SPLIT ? take(m2 * eb) : nullptr;
  void *a3 = take(m3 * eb), *a3l = SPLIT ? take(m3 * eb) : nullptr;
  float *h = reinterpret_cast<float *>(take(size_t(n) * kF1 * 4));
  int rc;
  tc::GemmParams p{};
  p.d_err = d_err;
  auto layer = [&](int l, const void *in, const void *in_lo, void *o, void *o_lo) {
    p.a_hi = in;
    p.a_lo = in_lo;
    p.b_hi = w->w_hi[l];
    p.b_lo = w->w_lo[l];
    p.bias = w->bias[l];
    p.colscale = w->colscale[l];
    p.out_inv_scale = w->out_inv_scale[l];
    p.out_hi = o;
    p.out_lo = o_lo;
  };
  layer(0, states ? static_cast<const void *>(states) : static_cast<const void *>(frames), nullptr, a1, a1l);
  // frame sources of the conv1 producers: the given ones, or contiguous stacks
  FrameSrc cont;
  if (!fs && frames) {
    for (int h = 0; h < kHist; ++h) {
      cont.src[h] = frames + h * kSlotBytes;
      cont.stride[h] = kFrameBytes;
    }
  }
  set_frames(p, fs ? *fs : cont);
  if (fs && fs->zmap) {
    // the leaves' conv1 from their newest frame plus the parent's partial map
    p.zmap = fs->zmap;
    p.zparent = fs->zparent;
    p.zleaf0 = fs->zleaf0;
    p.zbranch = fs->zbranch;
    rc = tc::launch<6, MODE, false>(p, (long long)n * kP1, K_CONV1_LEAF, st);
  } else if (zl && states) {
    // the newest slot: weight channel 3
    rc = launch_leaf_conv1(MODE, states, n, *zl, w->c1T + 3 * (kObj * 4 * kC1), w->c1W + 3 * (64 * kC1),
                           w->out_inv_scale[0], a1, a1l, st);
  } else {
    rc = states ? tc::launch<1, MODE, true>(p, (long long)n * kP1, K_CONV1, st)
                : tc::launch<1, MODE, false>(p, (long long)n * kP1, K_CONV1, st);
  }
  if (rc != BCTS_OK) return rc;
  // conv2 and conv3: TMA-fed implicit GEMMs (conv_tma.cu)
  const bool pair2 = (conv_tma_mask & 16) && MODE != 2;  // E4M3 has no tap-pair kernel
  auto conv = [&](int l, const void *in, const void *in_lo, void *o, void *o_lo) {
    ConvTmaArgs a{};
    a.in_hi = in;
    a.in_lo = in_lo;
    a.w_hi = w->w_hi[l];
    a.w_lo = w->w_lo[l];
    a.kpad = w->kpad[l];
    a.bias = w->bias[l];
    a.colscale = w->colscale[l];
    a.out_inv_scale = w->out_inv_scale[l];
    a.out_hi = o;
    a.out_lo = o_lo;
    a.n = n;
    a.d_err = d_err;
    if (l == 1 && pair2) return launch_conv_pair(MODE, a, st);
    return (conv_tma_mask >> (l + 1)) & 1 ? launch_conv_win(l + 1, MODE, a, st) : launch_conv_tma(l + 1, MODE, a, st);
  };
  // conv2 / conv3: tap-pair (conv_pair.cu, conv2 only), window-fed (conv_win.cu),
  // TMA im2col-fed (conv_tma.cu) or cp.async-gathered (tc_gemm), chosen per layer
  // by conv_tma_mask (bit 4 tap pair; bits 2 / 3 window, bits 0 / 1 im2col, for
  // conv2 / conv3)
  if ((conv_tma_mask & 5) || pair2) {
    rc = conv(1, a1, a1l, a2, a2l);
  } else {
    layer(1, a1, a1l, a2, a2l);
    rc = tc::launch<2, MODE, false>(p, (long long)n * kP2, K_CONV2, st);
  }
  if (rc != BCTS_OK) return rc;
  if (conv_tma_mask & 10) {
    rc = conv(2, a2, a2l, a3, a3l);
  } else {
    layer(2, a2, a2l, a3, a3l);
    rc = tc::launch<3, MODE, false>(p, (long long)n * kP3, K_CONV3, st);
  }
  if (rc != BCTS_OK) return rc;
  if constexpr (SPLIT) {
    // fc1 with fc2 folded into its epilogue: each row's partial Q-values per
    // 256-column half (in the space of the FP32 fc1 map, which is not written),
    // then bias + the two halves and the max (measured: fc1 + fc2 1.38 against
    // 1.48 ms per Atari-scale search; in BF16 / E4M3 the fold costs more than
    // the FP32 map it saves)
    layer(3, a3, a3l, nullptr, nullptr);
    p.w2 = w->f2w;
    p.fA = A;
    p.qpart = h;
    if ((rc = tc::launch<4, MODE, false>(p, (long long)n, K_FC1, st)) != BCTS_OK) return rc;
    return launch_fc2_combine(h, w->f2b, A, n, q, maxq, st, node_A);
  }
  layer(3, a3, a3l, h, nullptr);  // FP32 output for FC2
  if ((rc = tc::launch<4, MODE, false>(p, (long long)n, K_FC1, st)) != BCTS_OK) return rc;
  return launch_fc2_max(h, w->f2w, w->f2b, A, n, q, maxq, st, node_A);
}
}  // namespace

int tc_default_conv_mask(int precision) {
  // measured per layer on B300 at the Atari-scale workload (CUDA events, same
  // call): BF16 reads conv2 and conv3 from shared-memory windows (conv_win.cu);
  // E4M3 reads conv2 from windows and takes conv3 through TMA im2col; the
  // FP32-class split mode takes conv2 through tap pairs (conv_pair.cu: 2.30 ms
  // against 3.22 ms for the cp.async gather, the best of the pixel-major
  // kernels) and conv3 through TMA im2col (its window variant, whose padded rows
  // cost 65 % more MMAs, measured slower)
  return precision == BCTS_PREC_BF16 ? 12 : (precision == BCTS_PREC_FP8 ? 6 : 18);
}

int tc_qnet_forward(const TcWeights *w, int A, const uint8_t *frames, const bcts_state *states, int64_t n, float *q,
                    float *maxq, void *scratch, cudaStream_t st, int *d_err, const uint8_t *node_A,
                    const ZLeaf *zl, int conv_tma_mask, const FrameSrc *fs) {
  if (n <= 0) return BCTS_OK;
  if (conv_tma_mask < 0) conv_tma_mask = tc_default_conv_mask(w->precision);
  if (w->precision == BCTS_PREC_FP32)
    return tc_forward_impl<1>(w, A, frames, states, n, q, maxq, scratch, st, d_err, node_A, zl, conv_tma_mask, fs);
  if (w->precision == BCTS_PREC_FP8)
    return tc_forward_impl<2>(w, A, frames, states, n, q, maxq, scratch, st, d_err, node_A, zl, conv_tma_mask, fs);
  return tc_forward_impl<0>(w, A, frames, states, n, q, maxq, scratch, st, d_err, node_A, zl, conv_tma_mask, fs);
}

int tc_conv1_zmap_frames(const TcWeights *w, const FrameSrc &fs, int64_t n, float *z, cudaStream_t st, int *d_err) {
  if (n <= 0) return BCTS_OK;
  tc::GemmParams p{};
  p.d_err = d_err;
  p.b_hi = w->w_hi[0];
  p.b_lo = w->w_lo[0];
  p.bias = w->bias[0];
  p.colscale = w->colscale[0];
  p.out_hi = z;
  set_frames(p, fs);
  const long long M = (long long)n * kP1;
  if (w->precision == BCTS_PREC_FP32) return tc::launch<5, 1, false>(p, M, K_CONV1_PARTIAL, st);
  if (w->precision == BCTS_PREC_FP8) return tc::launch<5, 2, false>(p, M, K_CONV1_PARTIAL, st);
  return tc::launch<5, 0, false>(p, M, K_CONV1_PARTIAL, st);
}

bool tc_has_partial(const TcWeights *w) {
  return w->precision == BCTS_PREC_FP32 || w->precision == BCTS_PREC_BF16 || w->precision == BCTS_PREC_FP8;
}

// Parent partial maps Z = W_0 * slot1 + W_1 * slot2 + W_2 * slot3 + b, FP32 [n][400][32],
// from the sprite tables of weight channels 0-2.
int tc_conv1_partial(const TcWeights *w, const bcts_state *states, int64_t n, float *z, cudaStream_t st, int *d_err) {
  (void)d_err;
  return launch_partial_map(states, n, w->c1T, w->c1W, w->bias[0], z, st);
}

}  // namespace bcts

// ---------------------------------------------------------------------------
// Failure-path self-test: one bounded wait on an mbarrier that nothing ever
// arrives on.  It must give up after `limit` cycles and report through the
// error word, leaving the context usable.
// ---------------------------------------------------------------------------
namespace bcts {
namespace {
__global__ void wait_probe_kernel(int *d_err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) tc::wait_bar(tc::smem_u32(&bar), 0, &abort_flag, d_err, 7, limit);
}
}  // namespace
}  // namespace bcts

extern "C" int bcts_selftest_wait(int timeout_us) {
  if (timeout_us < 1 || timeout_us > 2000000) {
    bcts::set_thread_error("bcts_selftest_wait: timeout_us must be in [1, 2e6]");
    return BCTS_EINVAL;
  }
  int dev = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess) {
    cudaGetLastError();
    bcts::set_thread_error("bcts_selftest_wait: no CUDA device");
    return BCTS_ECUDA;
  }
  int *d_err = nullptr;
  if (cudaMalloc(&d_err, sizeof(int)) != cudaSuccess || cudaMemset(d_err, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    bcts::set_thread_error("bcts_selftest_wait: allocation failed");
    return BCTS_ENOMEM;
  }
  const long long limit = (long long)timeout_us * (long long)(khz > 0 ? khz : 2000000) / 1000;
  bcts::wait_probe_kernel<<<1, 32>>>(d_err, limit);
  int herr = 0;
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaDeviceSynchronize();
  const cudaError_t e3 = cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_err);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    bcts::set_thread_error("bcts_selftest_wait: CUDA error");
    return BCTS_ECUDA;
  }
  if (herr == 7) {
    bcts::set_thread_error("bcts_selftest_wait: the bounded wait ran out and reported it (expected)");
    return BCTS_ETIMEOUT;
  }
  bcts::set_thread_error("bcts_selftest_wait: the wait did not report a time-out");
  return BCTS_OK;
}
