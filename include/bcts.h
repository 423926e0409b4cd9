/*
 * bcts.h -- C ABI of the B300 Batch-BFS / BCTS tree-search library (libbcts.so).
 *
 * The library implements the data-parallel hot path of "Improve Agents without
 * Retraining: Parallel Tree Search with Off-Policy Correction" (Hallak et al.,
 * NeurIPS 2021):
 *   - Alg. 1 (Batch-BFS): every node of one depth is expanded at once; state and
 *     accumulated reward are replicated A times, child = parent * A + a, the
 *     simulator advances all children, R += gamma^i r; at depth d the leaves are
 *     scored R += gamma^d max_a Q(s_d, a);
 *   - Eq. 1 / Eq. 2: the d-step Q estimate per root action and its argmax;
 *   - Prop. 1 and Sec. 3.3: Bellman errors delta(a) from the root and depth-1 Q;
 *   - Eq. 7: the Bellman penalty B(delta_e, delta_o, A, d), scaled by the swept
 *     multiplier c of Sec. 5.1;
 *   - Eq. 3 / Eq. 4: corrected root values and the BCTS action.
 * The simulator is a synthetic integer sprite environment (stand-in for Atari
 * via CuLE, Sec. 4) rendered to the 4-frame 84x84 uint8 stack of Sec. 5, and
 * leaves are scored by a Nature-DQN Q-network (stand-in for Rainbow, Sec. 5.1).
 *
 * Conventions for every entry point:
 *   - returns a status (BCTS_OK = 0, negative = error); never aborts, never
 *     exits; after an error bcts_last_error(ctx) (or bcts_last_error(NULL) for
 *     calls without a context) describes it;
 *   - "host" pointers are caller-owned host memory, "device" pointers are
 *     caller-owned device memory on the context's device; the library never
 *     frees caller memory;
 *   - `stream` arguments are a cudaStream_t passed as void*; NULL means the
 *     context's own stream (for calls without a context: the legacy default
 *     stream).  Device-pointer calls are asynchronous on that stream.
 *   - ties in every argmax are broken towards the lowest index.
 */
#ifndef BCTS_H
#define BCTS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BCTS_API __attribute__((visibility("default")))
#else
#define BCTS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
    BCTS_OK = 0,
    BCTS_PENDING = 1,     /* bcts_poll: request not finished yet */
    BCTS_EINVAL = -1,     /* bad argument */
    BCTS_ENOMEM = -2,     /* device or host allocation failed / over budget */
    BCTS_ECUDA = -3,      /* a CUDA call failed */
    BCTS_ETIMEOUT = -4,   /* a bounded wait ran out */
    BCTS_EBUSY = -5,      /* queue full */
    BCTS_ENOTICKET = -6,  /* unknown or already collected ticket */
    BCTS_EDEVICE = -7,    /* a kernel reported an error through its error word */
    BCTS_ENOKERNEL = -8   /* the requested path is not available on this device */
};

/* Leaf Q-network arithmetic. */
enum {
    BCTS_PREC_FP32 = 0,      /* FP32-class: tcgen05 BF16 split (hi+lo) products, FP32 accumulate */
    BCTS_PREC_BF16 = 1,      /* BF16 operands, FP32 accumulate */
    BCTS_PREC_FP8 = 2,       /* FP8 E4M3 operands, per-output-channel weight scales, FP32 accumulate */
    BCTS_PREC_FP32_SIMT = 3  /* plain FP32 on CUDA cores (the unoptimised baseline) */
};

/* Environment state, 80 bytes, little endian:
 *   pos[h][k] = (x, y) cell of object k at history slot h (slot 3 = newest),
 *               0 <= x, y <= 20; object 0 is the agent, 1 the reward, 2-3 hazards;
 *   vel[k]    = per-tick velocity of object k (object 0 unused, 0);
 *   tick      = step counter (drives the respawn hash);  pad = 0. */
typedef struct bcts_state {
    int16_t pos[4][4][2];
    int8_t vel[4][2];
    uint32_t tick;
    uint32_t pad;
} bcts_state;

/* Simulator description.  kind 0 = the sprite environment (the only one). */
typedef struct bcts_env_desc {
    int kind;
} bcts_env_desc;

typedef struct bcts_options {
    int precision;              /* BCTS_PREC_* (default BCTS_PREC_FP32) */
    size_t frame_budget_bytes;  /* serving admission budget: device bytes of in-flight requests (0 = 8 GiB) */
    int max_roots;              /* serving: requests fused per pass (0 = 64) */
    int flags;                  /* BCTS_FLAG_* bits, 0 = defaults */
    int leaf_chunk;             /* leaves rendered + scored per pass (0 = automatic) */
} bcts_options;

/* Option flags.  BCTS_FLAG_FRAMES: tensor-core precisions write every node's
 * frame stack to device memory and read it back in conv1 (by default conv1
 * renders its operand tiles from the node states on the fly and the frames of
 * the searched nodes never reach device memory). */
#define BCTS_FLAG_FRAMES 1
/* BCTS_FLAG_EXACT_GEV: the penalty of Eq. 3 is the exact bias gap
 * B_e(sigma_e, A, d) - B_o(sigma_o, A, d) of Lemma 2 (normal quantiles of
 * 1 - 1/(A^d - A^(d-1)) and 1 - 1/A^(d-1) plus the Euler-Mascheroni GEV term,
 * sigma = delta / sqrt(2) by Prop. 1) instead of its closed-form approximation
 * Eq. 7.  Both are scaled by gamma^d and the correction multiplier c. */
#define BCTS_FLAG_EXACT_GEV 2

typedef struct bcts_ctx bcts_ctx;

/* Number of FP32 Q-network parameters for A actions (PyTorch order, see bcts_create). */
BCTS_API size_t bcts_qnet_numel(int A);

/*
 * Create a search context on the current CUDA device.
 *   env          : NULL or {kind = 0}
 *   qnet_weights : host, bcts_qnet_numel(A) floats in PyTorch parameter order:
 *                  conv1.w[32][4][8][8], conv1.b[32], conv2.w[64][32][4][4],
 *                  conv2.b[64], conv3.w[64][64][3][3], conv3.b[64],
 *                  fc1.w[512][3136] (input flattened C,H,W), fc1.b[512],
 *                  fc2.w[A][512], fc2.b[A]; input pixels are scaled by 1/255.
 *                  Copied at create; the caller may free it afterwards.
 *   A            : action count, 1..18 (like Atari's full action set): actions
 *                  0..8 move the agent one cell noop, up, right, left, down,
 *                  up-right, up-left, down-right, down-left; 9..17 the same two
 *                  cells at a time
 *   d            : default search depth, 0..6 (Alg. 1's d; d = 0 returns pi_o)
 *   gamma        : discount in (0, 1]
 *   correction   : multiplier c of the Eq. 7 penalty (Sec. 5.1 sweeps it);
 *                  0 = vanilla tree search (Eq. 2), 1 = Eq. 3 as printed
 *   opt          : NULL = defaults
 *   out          : receives the context
 * Environment: BCTS_CONV_KERNELS = m (0..31), read here, fixes the kernels of the
 *   leaf Q-network's conv2 / conv3 (tensor-core precisions): bit 4 conv2 through
 *   the tap-pair kernel (weights in tensor memory; BF16 and FP32-class), else
 *   bit 2 / bit 3 the shared-memory window kernels, else bit 0 / bit 1 the TMA
 *   im2col kernels, else the cp.async gather; unset = the precision's measured
 *   default.  Every variant computes the same layer; they differ in speed and
 *   rounding order.
 * Errors: BCTS_EINVAL (bad A, d, gamma, NULL weights/out), BCTS_ENOMEM, BCTS_ECUDA.
 */
BCTS_API int bcts_create(const bcts_env_desc *env, const float *qnet_weights, int A, int d, float gamma,
                float correction, const bcts_options *opt, bcts_ctx **out);

/* Free every resource of the context (waits for its pending work). NULL is a no-op. */
BCTS_API void bcts_destroy(bcts_ctx *ctx);

/* Message of the last error on this context (or of the last context-free call
 * on this thread when ctx is NULL).  Valid until the next call on the context. */
BCTS_API const char *bcts_last_error(const bcts_ctx *ctx);

/*
 * Search n roots at the context's depth (Alg. 1 + Eq. 3/4), synchronously.
 *   roots           : host, n states
 *   out_action      : host, n int32 -- BCTS action per root (Eq. 4)
 *   out_root_values : host, n*A floats -- corrected d-step values (Eq. 3),
 *                     row i = root i; for d = 0 the root Q-values
 * Copies inputs to the device, runs, copies results back, synchronises.
 * n = 0 is a no-op.  Errors: BCTS_EINVAL, BCTS_ENOMEM, BCTS_ECUDA, BCTS_EDEVICE.
 */
BCTS_API int bcts_search(bcts_ctx *ctx, const bcts_state *roots, int n, int32_t *out_action, float *out_root_values);

/*
 * Per-node export (Sec. 4: since Batch-BFS advances the whole tree at once it
 * exposes the cumulative reward and the estimated value of every tree node; the
 * appendix's ablation trains DQN on values propagated from the tree nodes).
 * The same search as bcts_search_device (device pointers, asynchronous on
 * `stream`, the context's A and d), and for every node x at depth i = 1..d of
 * every root, stored level by level (level i: n * A^i floats in Alg. 1's order,
 * child of node k = k * A + a, after the n * (A + ... + A^(i-1)) floats of the
 * levels above):
 *   d_node_R[x] = sum over t < i of gamma^t r_t on the path from the root (Alg. 1's R)
 *   d_node_V[x] = max over the d - i remaining actions of
 *                 sum_t gamma^t r_t + gamma^(d-i) max_a Q(leaf, a),
 *                 the (d - i)-step value of x's state (at i = d: max_a Q(x, a)),
 * so R + gamma^i V is the best root-discounted return through x and the
 * uncorrected root value of action a is R + gamma V of depth-1 node a.  Each
 * array holds bcts_tree_nodes(n, A, d) floats (caller-owned device memory;
 * d = 0: none, the pointers may be NULL).  bcts_tree_nodes returns -1 for
 * invalid arguments or more than 2^40 nodes per level.
 */
BCTS_API int64_t bcts_tree_nodes(int n, int A, int d);
BCTS_API int bcts_search_tree(bcts_ctx *ctx, const bcts_state *d_roots, int n, int32_t *d_out_action,
                              float *d_out_root_values, float *d_node_R, float *d_node_V, void *stream);

/*
 * Pruned search (Sec. 4: an index array of unpruned states, updated at each
 * pruning step, traces the best root action; the paper leaves the criterion to
 * future work).  Host pointers, as bcts_search.  Within the subtree of each root
 * action a_0, the nodes of every level i = 2 .. d-1 are ranked by their
 * cumulative reward plus estimated value R + gamma^i max_a Q(s, a) (Alg. 1's R,
 * the context's Q-network) and only the `keep` best (lowest index among equal
 * scores, keep in [1, 256]) are expanded further; V(a_0) is the maximum of
 * R + gamma^d max_a Q over the surviving leaves.  Root Q, pi_o, the Bellman
 * errors and the penalty (Eq. 7, or Lemma 2 with BCTS_FLAG_EXACT_GEV) are the
 * full search's.  With d <= 2, or keep at least every level's candidate count,
 * it is bcts_search.  Work per root: A (keep A)^(d-2) A leaves instead of A^d.
 */
BCTS_API int bcts_search_pruned(bcts_ctx *ctx, const bcts_state *roots, int n, int keep, int32_t *out_action,
                                float *out_root_values);
/* The same with device pointers, asynchronous on `stream` (as bcts_search_device). */
BCTS_API int bcts_search_pruned_device(bcts_ctx *ctx, const bcts_state *d_roots, int n, int keep,
                                       int32_t *d_out_action, float *d_out_root_values, void *stream);

/* Same as bcts_search with device pointers, asynchronous on `stream`.  The
 * context's buffers are reused by the next search on the same context, so
 * searches on one context must not overlap (the library orders them on the
 * context's stream when stream is NULL). */
BCTS_API int bcts_search_device(bcts_ctx *ctx, const bcts_state *d_roots, int n, int32_t *d_out_action,
                       float *d_out_root_values, void *stream);

/*
 * Batched form: n roots, root i searched at depth d_i in [0, 6] with A_i actions
 * in [1, context A] (FC2 rows 0..A_i-1 are used).  Host pointers, synchronous.
 * out_root_values is n * (context A) floats; row i holds A_i values, the rest 0.
 * Roots are grouped by (A, d); each depth of each group expands in one launch,
 * and every Q-network evaluation of the call (roots, depth-1 nodes, leaves of
 * all groups) runs as one batch.  The second call with the same multiset of
 * (A, d) is captured into a CUDA graph, later ones replay it.  The leaf chunk
 * is autotuned per leaf-count bucket on first use (kept in memory, and in the
 * file named by the BCTS_TUNE_FILE environment variable when set).  Each root's
 * result is bit-identical to searching it alone.
 */
BCTS_API int bcts_search_mixed(bcts_ctx *ctx, const bcts_state *roots, const int32_t *depths, const int32_t *actions,
                      int n, int32_t *out_action, float *out_root_values);

/*
 * Serving form: continuous batching.  bcts_submit queues one decision request
 * (root, depth d in [0, 6], A in [1, context A]) and returns at once with a
 * ticket.  Three worker threads (each with its own stream and buffers, sharing
 * the context's weights) take queued requests in arrival order while the
 * device bytes they occupy in a pass fit the budget (frame_budget_bytes,
 * default 8 GiB; per request its node levels, per-leaf values and tables and
 * its leaves' parents' partial conv1 maps, about 310 MB at A = 18, d = 4; at
 * most max_roots per pass, default 64) and run each admitted set as one batched
 * pass (bcts_search_mixed), so up to three passes overlap on the device; while
 * one pass is on the device, a worker with fewer than about 1M queued leaves
 * waits up to 2 ms for more.  Requests complete independently.  bcts_poll waits
 * up to timeout_us microseconds (0 = do not wait, <0 = wait without limit) for
 * a ticket: BCTS_OK with out_action (1 int32) and out_root_values (A floats,
 * host) filled and the ticket released; BCTS_PENDING if not finished;
 * BCTS_ENOTICKET for unknown tickets.  Both are thread-safe.
 */
BCTS_API int bcts_submit(bcts_ctx *ctx, const bcts_state *root, int d, int A, uint64_t *out_ticket);
BCTS_API int bcts_poll(bcts_ctx *ctx, uint64_t ticket, int32_t *out_action, float *out_root_values, int timeout_us);

/* ---- step-level entry points (device pointers; Alg. 1's individual steps) ---- */

/*
 * Alg. 1 replicate + advance + accumulate: child c = p * A + a of parent p gets
 * state G(parent p, action a) and R[c] = R[p] + gamma_pow * r  (gamma_pow = gamma^i
 * at depth i).  parents: n_parents states; parent_R: n_parents floats (NULL =
 * zeros); children: n_parents*A states; child_R: n_parents*A floats (may be NULL);
 * child_reward: n_parents*A int8 rewards (may be NULL).  No context needed.
 */
BCTS_API int bcts_expand(const bcts_state *d_parents, const float *d_parent_R, int64_t n_parents, int A, float gamma_pow,
                bcts_state *d_children, float *d_child_R, int8_t *d_child_reward, void *stream);

/*
 * Alg. 1's backup and the BCTS correction as a step of their own (device
 * pointers, asynchronous on `stream`, no context, no allocation):
 *   d_leaf_R     : n * A^d floats, Alg. 1's accumulated discounted reward R of every
 *                  leaf, level order (leaf k of root i is i * A^d + k; child = parent * A + a)
 *   d_leaf_maxq  : n * A^d floats, max_a Q(leaf, a)
 *   d_q0         : n * A floats, root Q-values Q_0(s_0, .)
 *   d_r1         : n * A floats, the rewards r(s_0, a) of the depth-1 nodes
 *   d_maxq1      : n * A floats, max_a' Q(s_1^a, a') of the depth-1 nodes
 *   A in [1, 32], d in [0, 16], gamma in (0, 1], correction = c (Sec. 5.1),
 *   flags = 0 or BCTS_FLAG_EXACT_GEV (Lemma 2's gap instead of Eq. 7)
 *   d_out_action : n int32, Eq. 4;  d_out_values : n * A floats, Eq. 3
 * V(a_0) = max over the A^(d-1) leaves below root action a_0 of R + gamma^d maxq
 * (Alg. 1's leaf term and argmax; Eq. 1), delta(a) = r1 + gamma maxq1 - Q_0
 * (Prop. 1), delta_o = |delta(pi_o)|, delta_e = mean |delta(a)| over a != pi_o,
 * B by Eq. 7, values V(a) - [a != pi_o] gamma^d c B, action = lowest-index argmax.
 * d = 0: values = Q_0, action = pi_o (the leaf and depth-1 pointers may be NULL).
 * At d = 1 the leaves are the depth-1 nodes (pass d_r1 and d_maxq1 as the leaf
 * arrays).  d_out_values also holds the intermediate segment maxima, so it must
 * not overlap the inputs.  Errors: BCTS_EINVAL (bad sizes, NULL pointers, more
 * than 2^40 leaves per root action), BCTS_ECUDA.
 */
BCTS_API int bcts_backup(const float *d_leaf_R, const float *d_leaf_maxq, const float *d_q0, const float *d_r1,
                         const float *d_maxq1, int n, int A, int d, float gamma, float correction, int flags,
                         int32_t *d_out_action, float *d_out_values, void *stream);

/* One environment tick on the host: *out = G(*s, a), *reward (may be NULL) in
 * {-1, 0, 1}; a in [0, 18).  The same rules as bcts_expand (Alg. 1's simulator),
 * for callers that advance an episode by the chosen action.  No context, no GPU. */
BCTS_API int bcts_env_step(const bcts_state *s, int a, bcts_state *out, int *reward);

/* Render n states to n frame stacks, uint8 [n][4][84][84], channel h = history slot h. */
BCTS_API int bcts_render(const bcts_state *d_states, int64_t n, uint8_t *d_frames, void *stream);

/* ---- measurement ------------------------------------------------------------ */
/* Kernel classes timed by bcts_profile (and bcts_dnn_profile: the DNN
 * workload's forward-model layers are BCTS_KERN_DNN_MLP, its Q head
 * BCTS_KERN_DNN_Q, its per-child epilogues BCTS_KERN_EXPAND).  BCTS_KERN_CONV1 is conv1 over whole
 * frame stacks; when a search scores its leaves from their parents' partial
 * conv1 maps (frame-stacking linearity: the three older history slots of a
 * leaf are its parent's three newest), the parents' maps are
 * BCTS_KERN_CONV1_PARTIAL and the leaves' remaining slot BCTS_KERN_CONV1_LEAF. */
enum {
    BCTS_KERN_EXPAND = 0, BCTS_KERN_RENDER, BCTS_KERN_CONV1, BCTS_KERN_CONV2, BCTS_KERN_CONV3,
    BCTS_KERN_FC1, BCTS_KERN_FC2, BCTS_KERN_BACKUP, BCTS_KERN_CONV1_PARTIAL, BCTS_KERN_CONV1_LEAF,
    BCTS_KERN_DNN_MLP, BCTS_KERN_DNN_Q, BCTS_KERN_COUNT
};

/*
 * Per-kernel-class device time of this context's searches.  enable = 1 starts
 * recording (a CUDA event pair on the launching stream around every kernel),
 * 0 stops.  On each call the totals since the previous call are returned and
 * reset: out_ms[BCTS_KERN_COUNT] milliseconds and out_launches[BCTS_KERN_COUNT]
 * launches per class (either may be NULL); *out_total_launches (may be NULL)
 * counts every kernel launch of the context, recorded or not, including those
 * of its serving workers (bcts_submit).  Synchronises the context's pending
 * work.  Not for use while a search runs on another thread or served requests
 * are in flight.
 */
BCTS_API int bcts_profile(bcts_ctx *ctx, int enable, double *out_ms, int64_t *out_launches,
                          int64_t *out_total_launches);

/* Score n frame stacks with the context's Q-network in its precision: q [n][A] floats. */
BCTS_API int bcts_qnet(bcts_ctx *ctx, const uint8_t *d_frames, int64_t n, float *d_q, void *stream);

/* Failure-path self-test (no counterpart in the paper): runs one device wait on
 * an mbarrier that nothing arrives on, with the same bounded-wait code the
 * Q-network kernels use, limited to timeout_us microseconds (1 .. 2e6).  The
 * wait must give up and report through the device error word: the call returns
 * BCTS_ETIMEOUT when it did (the expected outcome) and BCTS_OK if no time-out
 * was reported.  Nothing faults, traps or hangs; the device stays usable. */
BCTS_API int bcts_selftest_wait(int timeout_us);

/* ---- DNN forward-model workload ----------------------------------------------
 * Sec. 4's second runtime workload: Batch-BFS over a randomly initialised
 * network standing in for a learned forward model (three hidden layers of
 * width 100 on a 100-wide state and a one-hot action).  Model, in the weights'
 * PyTorch order (FP32, flat, bcts_dnn_numel(A) floats):
 *   fm1.w [100][100 + A], fm1.b [100], fm2.w [100][100], fm2.b [100],
 *   fm3.w [100][100], fm3.b [100], fmo.w [101][100], fmo.b [101],
 *   q.w [A][100], q.b [A];
 *   x = [s; onehot(a)], h_k = ReLU(W_k h_(k-1) + b_k) (k = 1..3),
 *   o = fmo.w h_3 + fmo.b, s' = tanh(o[0..99]), r = o[100]   (the simulator G),
 *   Q(s, .) = q.w s + q.b                                     (the value network).
 * States are BCTS_DNN_STATE floats.  The search is the same as bcts_search
 * (Alg. 1, Prop. 1, Eq. 3/4 with Eq. 7, or Lemma 2 with BCTS_FLAG_EXACT_GEV in
 * flags), in FP32 on CUDA cores: A in [1, 32], d in [0, 16], n * A^d < 2^31.
 * Values: n x A floats.  Device roots (bcts_dnn_search_device) must be 16-byte
 * aligned.  Errors as for bcts_create / bcts_search; the context's message is
 * returned by bcts_dnn_last_error. */
#define BCTS_DNN_STATE 100
typedef struct bcts_dnn_ctx bcts_dnn_ctx;
BCTS_API size_t bcts_dnn_numel(int A);
BCTS_API int bcts_dnn_create(const float *weights, int A, int d, float gamma, float correction, int flags,
                             bcts_dnn_ctx **out);
BCTS_API void bcts_dnn_destroy(bcts_dnn_ctx *ctx);
BCTS_API int bcts_dnn_search(bcts_dnn_ctx *ctx, const float *roots, int n, int32_t *out_action, float *out_values);
BCTS_API int bcts_dnn_search_device(bcts_dnn_ctx *ctx, const float *d_roots, int n, int32_t *d_out_action,
                                    float *d_out_values, void *stream);
BCTS_API int bcts_dnn_profile(bcts_dnn_ctx *ctx, int enable, double *out_ms, int64_t *out_launches,
                              int64_t *out_total_launches);
BCTS_API const char *bcts_dnn_last_error(const bcts_dnn_ctx *ctx);

/* ---- allocation-free Q-network evaluation ------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory (code running inside an allocator or memory-pool
 * callback, engines that reserve the whole device before loading this library,
 * hosts that forbid cudaMalloc after start-up).  It needs no context.
 *
 * bcts_qnet_static scores n <= BCTS_STATIC_MAX_NODES frame stacks with the plain
 * FP32 Q-network (the same kernels as a context created with
 * BCTS_PREC_FP32_SIMT) and calls no cudaMalloc, cudaFree or other allocating
 * routine.  Its scratch -- the weights in the kernels' layout and the activation
 * maps -- is one static device array of about 18 MB, part of this entry point's
 * device code, which a GPU holds from the time that code is loaded on it until
 * the process exits.
 * Set-up: the CUDA runtime loads device code lazily (on first use) unless
 * CUDA_MODULE_LOADING=EAGER.  The first call on each device, made with that
 * device current, loads the kernels this entry point runs, places the array and
 * looks up its address (cudaGetSymbolAddress); n = 0 is enough.  Make that call
 * at start-up, before any allocation limit applies and before any stream
 * capture: later calls on the device then neither allocate nor load anything.
 * Cost: every call first rewrites the caller's weights into the kernels' layout
 * inside the array (about 1.69 M floats, 13.5 MB of extra reads and writes),
 * which for small batches can take longer than the network itself.
 *   d_qnet_weights : device, bcts_qnet_numel(A) floats, PyTorch order (as in bcts_create)
 *   A              : 1..18
 *   d_frames       : device, uint8 [n][4][84][84]
 *   n              : 0..BCTS_STATIC_MAX_NODES; larger n returns BCTS_EINVAL
 *   d_q            : device, n * A floats
 *   stream         : cudaStream_t as void*, NULL = legacy default stream
 * Every call on a device shares the one array and leaves
 * its contents behind; each call overwrites all of it that it reads, so nothing
 * needs clearing, but calls whose execution overlaps on the GPU (different
 * streams, or different host threads) race on the array and must be serialised
 * by the caller.  Errors: BCTS_EINVAL, BCTS_ECUDA (message in bcts_last_error(NULL)). */
#define BCTS_STATIC_MAX_NODES 128
BCTS_API int bcts_qnet_static(const float *d_qnet_weights, int A, const uint8_t *d_frames, int64_t n, float *d_q,
                              void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BCTS_H */
