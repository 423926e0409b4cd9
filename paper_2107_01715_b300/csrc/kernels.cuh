// kernels.cuh -- internal launchers shared by the library's translation units.
#pragma once

#include "common.cuh"

namespace bcts {

// env.cu
int launch_expand(const bcts_state *parents, const float *parent_R, int64_t n_parents, int A, float gamma_pow,
                  bcts_state *children, float *child_R, int8_t *child_reward, cudaStream_t stream);
int launch_render(const bcts_state *states, int64_t n, uint8_t *frames, cudaStream_t stream);
// One expansion level of up to kMaxListGroups independent trees in one launch
// (the batched form's (A, d) groups): group k expands n_child[k] children of
// parents[k] into children[k]; block_end is the running total of its blocks of
// 256 children.
constexpr int kMaxListGroups = 24;
struct ExpandList {
  int n = 0;
  const bcts_state *parents[kMaxListGroups];
  const float *parent_R[kMaxListGroups];
  bcts_state *children[kMaxListGroups];
  float *child_R[kMaxListGroups];
  uint32_t n_child[kMaxListGroups];
  uint32_t block_end[kMaxListGroups];
  int A[kMaxListGroups];
  float gamma_pow[kMaxListGroups];
};
int launch_expand_list(const ExpandList &L, cudaStream_t stream);
// The newest history slot only: frames [n][84][84] (7,056 bytes per state).
int launch_render_newest(const bcts_state *states, int64_t n, uint8_t *frames, cudaStream_t stream);
constexpr int kSlotBytes = kPix * kPix;  // 7,056

// Weights of the plain FP32 CUDA-core Q-network, in the layouts its kernels read:
//   c1w [32][256]  k = c*64 + ky*8 + kx, pre-scaled by 1/255
//   c2w [64][512]  k = (ky*4 + kx)*32 + c      (input NHWC)
//   c3w [64][576]  k = (ky*3 + kx)*64 + c
//   f1w [512][3136] k = (y*7 + x)*64 + c        (conv3 map NHWC-flattened)
//   f2w [A][512]
struct SimtWeights {
  const float *c1w, *c1b, *c2w, *c2b, *c3w, *c3b, *f1w, *f1b, *f2w, *f2b;
  int A;
};

// Scratch the plain path needs per chunk of `chunk` leaves (bytes).
size_t simt_scratch_bytes(int64_t chunk);

// Q-network on n frame stacks: q [n][A] (may be NULL), maxq [n] (may be NULL).
// node_A (may be NULL): per-node action count for the max (batched form).
int simt_qnet_forward(const SimtWeights &w, const uint8_t *frames, int64_t n, float *q, float *maxq,
                      void *scratch, cudaStream_t stream, const uint8_t *node_A = nullptr);

// Load the kernels of simt_qnet_forward on the current device now (see qnet_simt.cu).
int simt_preload();

// FC2 + max over actions on FP32 fc1 activations h [n][512] (one warp per node).
int launch_fc2_max(const float *h, const float *W2, const float *b2, int A, int64_t n, float *q, float *maxq,
                   cudaStream_t st, const uint8_t *node_A = nullptr);

// qnet_tc.cu (tensor-core paths)
struct TcWeights;  // defined in qnet_tc.cu
size_t tc_scratch_bytes(int64_t chunk, int precision);
// act_scale: FP8 activation scales of the conv1/conv2/conv3 output maps (NULL otherwise).
int tc_weights_create(const float *host_weights, int A, int precision, const float *act_scale, TcWeights **out,
                      std::string &err);
void tc_weights_destroy(TcWeights *w);
// Leaf conv1 from the parent partial maps: parent of leaf i = (leaf0 + i) / branch.
struct ZLeaf {
  const float *zmap;
  uint32_t leaf0, branch;
  const uint32_t *parent = nullptr;  // if set: parent of leaf i = parent[leaf0 + i] (mixed branching)
};
// Rendered frames as conv1's input (any frame source): history slot s of node i
// of a launch is the 84 x 84 uint8 frame at
//   src[s] + ((node0 + i) / div[s] - sub[s]) * stride[s].
// A search renders each node's newest frame when its level is expanded, so a
// node's stack is its own frame and its ancestors' (Alg. 1: the parent of x is
// x / A), and the roots' four slots.  With zmap set, conv1 runs the newest slot
// only (src[0]) and adds the parent's partial map (zparent[zleaf0 + i] if set,
// else (zleaf0 + i) / zbranch) before the ReLU.
struct FrameSrc {
  const uint8_t *src[4] = {};
  uint32_t div[4] = {1, 1, 1, 1}, sub[4] = {}, stride[4] = {};
  uint32_t node0 = 0;
  const float *zmap = nullptr;
  const uint32_t *zparent = nullptr;
  uint32_t zleaf0 = 0, zbranch = 1;
};
// The parents' partial maps Z [n][400][32] FP32 from rendered frames: conv1's
// weight channels 0-2 (plus its bias) over the parents' history slots 1-3, which
// fs.src[0..2] describe.
int tc_conv1_zmap_frames(const TcWeights *w, const FrameSrc &fs, int64_t n, float *z, cudaStream_t st, int *d_err);
// conv_tma_mask: conv2 (bit 0) / conv3 (bit 1) through the TMA im2col kernel of
// conv_tma.cu, conv2 (bit 2) / conv3 (bit 3) through the window kernel of
// conv_win.cu (before bits 0 / 1), conv2 through the tap-pair kernel of
// conv_pair.cu (bit 4, before all others; BF16 and FP32-class only), else the
// cp.async-gathered tc_gemm; -1 = this precision's default.
// fs (frames and states NULL): conv1 from rendered frames (see FrameSrc).
int tc_qnet_forward(const TcWeights *w, int A, const uint8_t *frames, const bcts_state *states, int64_t n, float *q,
                    float *maxq, void *scratch, cudaStream_t stream, int *d_err, const uint8_t *node_A = nullptr,
                    const ZLeaf *zl = nullptr, int conv_tma_mask = -1, const FrameSrc *fs = nullptr);
int tc_default_conv_mask(int precision);
bool tc_has_partial(const TcWeights *w);
// conv_tma.cu: conv2 (layer 2) or conv3 (layer 3) of n nodes on tcgen05 fed by TMA
// im2col loads.  mode: 0 BF16, 1 FP32-class split (hi + lo arrays), 2 E4M3.
struct ConvTmaArgs {
  const void *in_hi, *in_lo;    // NHWC input maps (lo: split mode)
  const void *w_hi, *w_lo;      // weights [64][kpad], K = (ky, kx, c)
  int kpad;                     // weight row length in elements
  const float *bias, *colscale; // colscale: FP8 per-channel weight x input activation scale
  float out_inv_scale;          // FP8: 1 / activation scale of the output map
  void *out_hi, *out_lo;        // NHWC output maps
  int64_t n;                    // nodes
  int *d_err;
};
int launch_conv_tma(int layer, int mode, const ConvTmaArgs &a, cudaStream_t st);
// conv_win.cu: the same layers with the A operand read in place from a window of
// the input map in shared memory (stride-1 form; conv2 on its space-to-depth
// view).  Same arguments and outputs.
int launch_conv_win(int layer, int mode, const ConvTmaArgs &a, cudaStream_t st);
// conv_pair.cu: conv2 with its weights resident in tensor memory and two filter
// taps of the space-to-depth view per M = 128, N = 128 instruction.  mode 0 BF16
// or 1 FP32-class split (E4M3: BCTS_EINVAL).  Same arguments and outputs.
int launch_conv_pair(int mode, const ConvTmaArgs &a, cudaStream_t st);
// leaf_conv1.cu: conv1 of n leaves (states) from their parents' partial maps, as
// ReLU(Z + the newest slot's term).  mode: 0 BF16, 1 FP32-class split (bf16 hi +
// lo), 2 E4M3 scaled by out_scale.  T [4 objects][2][2][32] and W3 [64][32]: the
// newest slot's (weight channel 3's) part of the sprite tables built with the
// tensor-core weights.
int launch_leaf_conv1(int mode, const bcts_state *states, int64_t n, const ZLeaf &zl, const float *T,
                      const float *W3, float out_scale, void *out_hi, void *out_lo, cudaStream_t st);
// The parents' partial maps (FP32, no ReLU) from the sprite tables of weight
// channels 0-2 (T [3][4][2][2][32] and W [3][64][32] first in the tables).
int launch_partial_map(const bcts_state *states, int64_t n, const float *T, const float *W, const float *bias,
                       float *Z, cudaStream_t st);
// The parents' partial maps Z [n][400][32] FP32 with this context's tables.
int tc_conv1_partial(const TcWeights *w, const bcts_state *states, int64_t n, float *z, cudaStream_t st, int *d_err);

// search.cu backup kernels
int launch_segment_max(const float *R, const float *maxq, int64_t n_seg, int64_t seg_len, float gamma_pow,
                       float *V, cudaStream_t stream);
// q0 rows are q_stride floats apart (root Q-values); r1, maxq1, V rows are A apart.
// exact_gev: the penalty is Lemma 2's exact bias gap instead of Eq. 7.
int launch_finalize(const float *q0, const float *maxq1, const float *r1, const float *V, int n, int A,
                    int depth, int A_stride, float gamma, float gamma_d, float corr, int32_t *action,
                    float *values, cudaStream_t stream, int q_stride = 0, int exact_gev = 0);

// Backup of several groups in one launch each for the segment maxima and the
// finalize step (the batched form): group k has roots root_end[k-1] ..
// root_end[k] - 1 and segments seg_end[k-1] .. seg_end[k] - 1 (n_k A_k each of
// seg_len[k] = A_k^(d_k - 1) leaves; none for d_k = 0), writes V[k] (order keys,
// n_k A_k words of storage), action[k], values[k] (rows A_stride apart).
// Segments must be shorter than the split threshold of launch_segment_max.
struct BackupList {
  int n = 0;
  const float *R[kMaxListGroups], *maxq[kMaxListGroups];
  float *V[kMaxListGroups];
  const float *q0[kMaxListGroups], *maxq1[kMaxListGroups], *r1[kMaxListGroups];
  int32_t *action[kMaxListGroups];
  float *values[kMaxListGroups];
  int64_t seg_end[kMaxListGroups], root_end[kMaxListGroups];
  uint32_t seg_len[kMaxListGroups];
  int A[kMaxListGroups], depth[kMaxListGroups];
  float gamma_d[kMaxListGroups], gev_e[kMaxListGroups], gev_o[kMaxListGroups];
  int A_stride = 0, q_stride = 0, exact_gev = 0;
  float gamma = 0.f, corr = 0.f;
};
int launch_backup_list(BackupList &L, cudaStream_t st);

}  // namespace bcts
