// search.cuh -- the search context shared by search.cu, mixed.cu and serve.cu.
#pragma once

#include <array>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace bcts {

struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
};
struct HostBuf {
  void *p = nullptr;
  size_t cap = 0;
};

struct ServeState;  // serve.cu
struct MixedState;  // mixed.cu

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int A = 0;          // action count of the search being run
  int A_create = 0;   // action count the context was created with (FC2 rows)
  int d = 0;
  float gamma = 0.99f;
  float corr = 1.0f;
  int precision = BCTS_PREC_FP32;
  bcts_options opt{};
  std::string err;

  SimtWeights simt{};
  TcWeights *tc = nullptr;
  // FP32-class (bf16 split) weights of a BF16 / FP8 context: the roots and the
  // depth-1 nodes are scored with them, so pi_o and the Bellman errors of
  // Prop. 1 carry no reduced-precision error; only the leaves use `tc`.
  TcWeights *tc_ref = nullptr;
  bool ref_eval = false;  // set while eval_nodes_ref runs
  bool tc_fused_render = false;
  bool exact_gev = false;  // Lemma 2's exact bias gap instead of Eq. 7
  // per-node export of the current search (bcts_search_tree), level-major; null otherwise
  float *tree_R = nullptr, *tree_V = nullptr;
  bool owns_weights = true;  // serving workers share their owner's weights
  int *d_err = nullptr;

  DevBuf simt_w, frames_buf, scratch_buf, q0_buf, maxq1_buf, V_buf, r1_buf, leafmax_buf;
  DevBuf lvl_buf[2], R_buf[2];
  DevBuf io_roots, io_action, io_values, mixed_buf, z_buf;
  // rendered frames of a search on the frame path (BCTS_FLAG_FRAMES): the roots'
  // full stacks and each inner level's newest frames
  DevBuf rootfr_buf, lvlfr_buf[kMaxDepth + 1];
  DevBuf pr_cand, pr_candR, pr_candQ, pr_par, pr_parR, pr_idx;  // pruned search
  int prune_keep = 0;  // > 0: run_search keeps this many nodes per root action and level (d >= 3)
  // plain searches replayed from CUDA graphs, keyed by (root count, the caller's
  // device pointers or 0 for the host API, stream)
  using GraphKey = std::array<uintptr_t, 5>;
  struct SearchGraph {
    cudaGraphExec_t exec = nullptr;
    uint64_t generation = 0;  // buffer generation the graph was captured with
    int64_t launches = 0;     // kernel launches one replay makes
    int calls = 0;
    uint64_t last_generation = 0;  // generation after the previous eager call
  };
  std::map<GraphKey, SearchGraph> sgraphs;
  int run_graphed(const GraphKey &key, cudaStream_t st, const std::function<int()> &enqueue);
  HostBuf host_stage;

  ServeState *serve = nullptr;
  MixedState *mixed = nullptr;
  Profiler *prof = nullptr;
  int64_t chunk_override = 0;    // leaf chunk chosen by the batched form's autotuner
  int conv_mask = -1;            // conv2/conv3 kernel variants of the leaf Q-network (-1: per-precision default)
  bool conv_mask_fixed = false;  // conv_mask set through BCTS_CONV_KERNELS (the batched form's tuner keeps it)
  uint64_t buf_generation = 1;   // bumped whenever a device buffer moves

  ~Ctx();
  int fail(int code, const std::string &msg);
  int ensure(DevBuf &b, size_t bytes);
  int ensure_host(HostBuf &b, size_t bytes);
  // nodes per Q-network pass when `count` nodes are to be scored (0: the largest pass)
  int64_t chunk_nodes(int64_t count = 0) const;
  size_t dev_mem = 0;  // device memory (bytes), for the pass size
  int eval_nodes(const bcts_state *states, int64_t count, float *q, float *maxq, cudaStream_t st,
                 const uint8_t *node_A = nullptr, const float *zmap = nullptr, uint32_t zbranch = 0,
                 const uint32_t *zparent = nullptr);
  // eval_nodes with the FP32-class weights (tc_ref) when the context has them
  int eval_nodes_ref(const bcts_state *states, int64_t count, float *q, float *maxq, cudaStream_t st,
                     const uint8_t *node_A = nullptr);
  // Q-network over nodes whose conv1 input is described by frame sources
  // (chunked; f.node0 is advanced per chunk)
  int eval_frames(const FrameSrc &f, int64_t count, float *q, float *maxq, cudaStream_t st, bool ref);
  int qnet_nodes(const bcts_state *states, const uint8_t *frames, int64_t cnt, float *q, float *maxq,
                 cudaStream_t st, const uint8_t *node_A = nullptr, const ZLeaf *zl = nullptr);
  int export_tree(const std::vector<int64_t> &N, int A_, int d_, const float *leafMax, cudaStream_t st);
  int run_search(const bcts_state *d_roots, int n, int A_, int d_, int32_t *d_action, float *d_values,
                 int A_stride, cudaStream_t st);
  int run_search_pruned(const bcts_state *d_roots, int n, int keep, int32_t *d_action, float *d_values,
                        int A_stride, cudaStream_t st);
  int run_mixed(const bcts_state *d_roots, const bcts_state *h_roots, const int32_t *depths,
                const int32_t *actions, int n, int32_t *d_action, float *d_values);
  int search_host(const bcts_state *roots, int n, const int32_t *depths, const int32_t *actions,
                  int32_t *out_action, float *out_values);
  int mixed_results(const int32_t *depths, const int32_t *actions, int n, int32_t *out_action, float *out_values);
};

void serve_shutdown(Ctx *c);
int64_t serve_launches(Ctx *c);
Profiler *profiler_create();
void profiler_destroy(Profiler *p);
int64_t profiler_total(const Profiler *p);
void profiler_add(Profiler *p, int64_t launches);
int profiler_read(Profiler *p, cudaStream_t st, int enable, double *out_ms, int64_t *out_launches,
                  int64_t *out_total);
bool profiler_on(const Profiler *p);
void mixed_destroy(MixedState *m);

}  // namespace bcts
