// prune.cu -- pruned Batch-BFS.  Sec. 4 sketches pruning by an index array of
// unpruned states that is updated at each pruning step and then used to trace
// the best root action; it leaves the criterion open.  Here, within the subtree
// of each root action a_0 (a "group"), the nodes of every level i = 2 .. d-1
// are ranked by their cumulative reward plus estimated value, R + gamma^i
// max_a Q(s, a), and only the `keep` best (lowest candidate index among equal
// scores) are expanded further.  The survivors of a level are stored in
// increasing candidate order, so the candidates of the next level are
// survivor-index x A + a within each group, every group the same size, and
// V(a_0) is the plain segment maximum over the group's leaves.  Root Q, the
// depth-1 Bellman errors and the penalty are the full search's.
#include <string>
#include <vector>

#include "search.cuh"

namespace bcts {
namespace {

// One block per group: rank every candidate by (score desc, index asc), keep
// the first k, write their indices in increasing order to kept[g][0..k).
__global__ void prune_select_kernel(const float *__restrict__ R, const float *__restrict__ maxq, float gamma_i,
                                    int C, int k, int32_t *__restrict__ kept) {
  extern __shared__ float sc[];  // C scores, then C flags
  int *flag = reinterpret_cast<int *>(sc + C);
  const int64_t base = int64_t(blockIdx.x) * C;
  for (int j = threadIdx.x; j < C; j += blockDim.x) sc[j] = R[base + j] + gamma_i * maxq[base + j];
  __syncthreads();
  for (int j = threadIdx.x; j < C; j += blockDim.x) {
    const float s = sc[j];
    int rank = 0;
    for (int m = 0; m < C; ++m) {
      const float t = sc[m];
      rank += (t > s || (t == s && m < j)) ? 1 : 0;
    }
    flag[j] = rank < k ? 1 : 0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < C; j += blockDim.x) {
    if (!flag[j]) continue;
    int pos = 0;
    for (int m = 0; m < j; ++m) pos += flag[m];
    kept[int64_t(blockIdx.x) * k + pos] = j;
  }
}

// Survivors into the next level's parent array: node (g, s) <- candidate
// (g, kept[g][s]), 16 bytes per thread (a state is 5 x 16 bytes) plus R.
__global__ void prune_gather_kernel(const uint4 *__restrict__ cand, const float *__restrict__ candR,
                                    const int32_t *__restrict__ kept, int C, int k, int64_t n_out,
                                    uint4 *__restrict__ par, float *__restrict__ parR) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n_out * 5) return;
  const int64_t node = i / 5;
  const int part = int(i - node * 5);
  const int64_t g = node / k;
  const int64_t src = g * C + kept[node];
  par[node * 5 + part] = cand[src * 5 + part];
  if (part == 0) parR[node] = candR[src];
}

unsigned blocks_for(int64_t n) { return unsigned((n + 255) / 256); }

}  // namespace

int Ctx::run_search_pruned(const bcts_state *d_roots, int n, int keep, int32_t *d_action, float *d_values,
                           int A_stride, cudaStream_t st) {
  ProfilerGuard pg(prof);
  const int A_ = A_create, d_ = d;
  const int64_t G = int64_t(n) * A_;  // one group per (root, a_0)
  int rc;
  // widest candidate set of a level: A at level 2, keep * A afterwards
  const int64_t cmax = std::max<int64_t>(A_, int64_t(keep) * A_);  // <= 256 * 18 (the select kernel's shared memory)
  if (G * cmax > 0x7FFFFFFFLL) return fail(BCTS_EINVAL, "pruned search too large: n * A * keep * A exceeds 2^31 - 1");
  if ((rc = ensure(q0_buf, size_t(n) * A_ * 4)) != BCTS_OK) return rc;
  if ((rc = ensure(maxq1_buf, size_t(G) * 4)) != BCTS_OK) return rc;
  if ((rc = ensure(V_buf, size_t(G) * 4)) != BCTS_OK) return rc;
  if ((rc = ensure(r1_buf, size_t(G) * 4)) != BCTS_OK) return rc;
  if ((rc = ensure(pr_cand, size_t(G * cmax) * kStateBytes)) != BCTS_OK) return rc;
  if ((rc = ensure(pr_candR, size_t(G * cmax) * 4)) != BCTS_OK) return rc;
  if ((rc = ensure(pr_candQ, size_t(G * cmax) * 4)) != BCTS_OK) return rc;
  if ((rc = ensure(pr_par, size_t(G * std::max<int64_t>(keep < cmax ? keep : cmax, 1)) * kStateBytes)) != BCTS_OK)
    return rc;
  if ((rc = ensure(pr_parR, size_t(G * std::max<int64_t>(keep < cmax ? keep : cmax, 1)) * 4)) != BCTS_OK) return rc;
  if ((rc = ensure(pr_idx, size_t(G * std::max<int64_t>(keep < cmax ? keep : cmax, 1)) * 4)) != BCTS_OK) return rc;
  float *q0 = static_cast<float *>(q0_buf.p), *maxq1 = static_cast<float *>(maxq1_buf.p);
  float *V = static_cast<float *>(V_buf.p), *r1 = static_cast<float *>(r1_buf.p);
  bcts_state *cand = static_cast<bcts_state *>(pr_cand.p), *par = static_cast<bcts_state *>(pr_par.p);
  float *candR = static_cast<float *>(pr_candR.p), *candQ = static_cast<float *>(pr_candQ.p);
  float *parR = static_cast<float *>(pr_parR.p);
  int32_t *kept = static_cast<int32_t *>(pr_idx.p);
  // root Q and pi_o; depth 1 (one node per group) and its Q for the Bellman errors
  if ((rc = eval_nodes_ref(d_roots, n, q0, nullptr, st)) != BCTS_OK) return rc;
  if ((rc = launch_expand(d_roots, nullptr, n, A_, 1.f, par, r1, nullptr, st)) != BCTS_OK)
    return fail(rc, "expand launch failed");
  if ((rc = eval_nodes_ref(par, G, nullptr, maxq1, st)) != BCTS_OK) return rc;
  const float *curR = r1;
  int64_t S = 1;  // survivors per group
  double gprev = double(gamma);
  // candidates are survivor-index x A + a, so their conv1 can come from the
  // survivors' partial maps (frame stacking), as for the full search's leaves
  const bool use_z = tc && tc_fused_render && tc_has_partial(tc) &&
                     size_t(G) * std::max<int64_t>(1, std::min<int64_t>(keep, cmax)) * kP1 * kC1 * 4 <=
                         (size_t(8) << 30);
  for (int i = 2; i <= d_; ++i) {
    const double gi = gprev * double(gamma);
    const int64_t C = S * A_;
    const float *zmap = nullptr;
    if (use_z) {
      if ((rc = ensure(z_buf, size_t(G * S) * kP1 * kC1 * 4)) != BCTS_OK) return rc;
      const int64_t chunk = chunk_nodes(G * S);
      for (int64_t off = 0; off < G * S; off += chunk) {
        const int64_t k = G * S - off < chunk ? G * S - off : chunk;
        if ((rc = tc_conv1_partial(tc, par + off, k, static_cast<float *>(z_buf.p) + size_t(off) * kP1 * kC1, st,
                                   d_err)) != BCTS_OK)
          return fail(rc, "conv1 partial launch failed");
      }
      zmap = static_cast<const float *>(z_buf.p);
    }
    if ((rc = launch_expand(par, curR, G * S, A_, float(gprev), cand, candR, nullptr, st)) != BCTS_OK)
      return fail(rc, "expand launch failed");
    if ((rc = eval_nodes(cand, G * C, nullptr, candQ, st, nullptr, zmap, uint32_t(A_))) != BCTS_OK) return rc;
    if (i == d_) {
      // V(a_0): the maximum of R + gamma^d max Q over the group's leaves
      if ((rc = launch_segment_max(candR, candQ, G, C, float(gi), V, st)) != BCTS_OK)
        return fail(rc, "backup launch failed");
      break;
    }
    const int64_t k = keep < C ? keep : C;
    {
      ProfScope ps(K_BACKUP, st);
      prune_select_kernel<<<unsigned(G), 256, size_t(C) * 8, st>>>(candR, candQ, float(gi), int(C), int(k), kept);
      prune_gather_kernel<<<blocks_for(G * k * 5), 256, 0, st>>>(reinterpret_cast<const uint4 *>(cand), candR, kept,
                                                                  int(C), int(k), G * k, reinterpret_cast<uint4 *>(par),
                                                                  parR);
      if (cudaGetLastError() != cudaSuccess) return fail(BCTS_ECUDA, "pruning launch failed");
    }
    curR = parR;
    S = k;
    gprev = gi;
  }
  double gd = 1.0;
  for (int i = 0; i < d_; ++i) gd *= double(gamma);
  if ((rc = launch_finalize(q0, maxq1, r1, V, n, A_, d_, A_stride, gamma, float(gd), corr, d_action, d_values, st, 0,
                            exact_gev ? 1 : 0)) != BCTS_OK)
    return fail(rc, "finalize launch failed");
  return BCTS_OK;
}

}  // namespace bcts

extern "C" int bcts_search_pruned_device(bcts_ctx *ctx, const bcts_state *d_roots, int n, int keep, int32_t *d_action,
                                         float *d_values, void *stream) {
  if (!ctx) return BCTS_EINVAL;
  bcts::Ctx *c = reinterpret_cast<bcts::Ctx *>(ctx);
  if (n < 0 || keep < 1 || keep > 256 || (n > 0 && (!d_roots || !d_action || !d_values)))
    return c->fail(BCTS_EINVAL, "bcts_search_pruned_device: invalid argument");
  if (n == 0) return BCTS_OK;
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  c->prune_keep = keep;
  const int rc = c->run_search(d_roots, n, c->A_create, c->d, d_action, d_values, c->A_create, st);
  c->prune_keep = 0;
  return rc;
}

extern "C" int bcts_search_pruned(bcts_ctx *ctx, const bcts_state *roots, int n, int keep, int32_t *out_action,
                                  float *out_values) {
  if (!ctx) return BCTS_EINVAL;
  bcts::Ctx *c = reinterpret_cast<bcts::Ctx *>(ctx);
  if (n < 0 || keep < 1 || keep > 256 || (n > 0 && (!roots || !out_action || !out_values)))
    return c->fail(BCTS_EINVAL, "bcts_search_pruned: invalid argument");
  if (n == 0) return BCTS_OK;
  c->prune_keep = keep;
  const int rc = c->search_host(roots, n, nullptr, nullptr, out_action, out_values);
  c->prune_keep = 0;
  return rc;
}
