// mixed.cu -- batched form: many roots of mixed depth d and action count A in
// one search pass (the serving loop runs on it too).
//
// Roots are grouped by (A, d).  Per group the level-synchronous expansion of
// Alg. 1 runs as usual (one launch per level), but every Q-network evaluation
// of the pass runs once over the union of all groups' nodes: one pass over all
// roots, one over all depth-1 nodes, one over all leaves, so each persistent
// tensor-core layer kernel sees the whole batch.  The max over actions uses
// each node's own A (FC2 rows 0..A-1).  Backup and the Eq. 7 correction run
// per group.  For a composition seen before, the whole device part of the pass
// (copies included) is replayed from a captured CUDA graph.  The kernel
// configuration of the union leaf evaluation -- the leaf chunk and, for conv2
// and conv3 each, the TMA im2col kernel (taps per stage) or the cp.async gather
// (K blocks per stage) -- is picked by timing every candidate on the plan's own
// leaves on the first pass of a new (precision, leaf-count) bucket, and kept in
// memory (and in the file named by BCTS_TUNE_FILE).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <utility>
#include <vector>

#include "search.cuh"

namespace bcts {

struct MixedGroup {
  int A = 0, d = 0, n = 0;
  int root_off = 0;       // first sorted root
  int64_t l1_off = 0;     // first depth-1 node in the union level-1 buffer
  int64_t leaf_off = 0;   // first leaf in the union leaf buffer (d >= 2)
  int64_t nleaf = 0;      // n * A^d for d >= 2
  int64_t mid_off[kMaxDepth + 1] = {};  // first node of its level i (2 .. d-1) in the shared level buffer
  int64_t zoff = 0;       // first of its leaves' parents in the union partial-map buffer (d >= 2)
};

struct MixedPlan {
  int n = 0;
  std::vector<int> order;  // sorted position -> caller's root index
  std::vector<MixedGroup> groups;
  int64_t n1 = 0, nleaf = 0, mid = 0;
  int64_t mid_fill[kMaxDepth + 1] = {};  // nodes of all groups at each intermediate level
  int64_t nz = 0;       // leaves' parents of all groups (one partial conv1 map each)
  bool use_z = false;   // leaves' conv1 from the parents' partial maps
  std::string key;
};

// The union partial maps take 51.2 KB per parent; above this the batched form
// scores its leaves with whole-stack conv1 instead.
constexpr size_t kMaxZBytes = size_t(16) << 30;

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  uint64_t generation = 0;
  uint64_t last_use = 0;
};

// Bounds of the per-context caches: a serving stream produces a new batch
// composition nearly every pass, so neither map may grow without limit.
constexpr size_t kMaxGraphs = 64;
constexpr size_t kMaxSeen = 4096;

struct MixedState {
  DevBuf roots, q0, L1, r1, maxq1, nodeA1, mid[2], Rmid[2], leaves, Rleaf, maxq_leaf, nodeA_leaf, V, act, val, zbuf,
      zparent;
  HostBuf host;
  std::map<std::string, int> seen;
  std::map<std::string, GraphEntry> graphs;
  uint64_t use_clock = 0;
  struct Tuned {
    int64_t chunk;
    int conv_mask;
  };
  std::map<std::string, Tuned> tuned;  // (precision, leaf-count bucket) -> configuration
  bool tune_loaded = false;
  ~MixedState() {
    for (auto &kv : graphs)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    DevBuf *b[] = {&roots, &q0, &L1, &r1, &maxq1, &nodeA1, &mid[0], &mid[1], &Rmid[0], &Rmid[1],
                   &leaves, &Rleaf, &maxq_leaf, &nodeA_leaf, &V, &act, &val, &zbuf, &zparent};
    for (DevBuf *x : b)
      if (x->p) cudaFree(x->p);
    if (host.p) cudaFreeHost(host.p);
  }
};

void mixed_destroy(MixedState *m) { delete m; }

namespace {

int64_t ipow(int64_t a, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= a;
  return r;
}

std::string tune_file() {
  const char *f = std::getenv("BCTS_TUNE_FILE");
  return f ? std::string(f) : std::string();
}

int64_t leaf_bucket(int64_t nleaf) {
  int64_t b = 1;
  while (b < nleaf) b <<= 1;
  return b;
}

}  // namespace

// Buffers for a plan; bumps the generation when anything moves.
static int mixed_ensure(Ctx *c, MixedState *m, const MixedPlan &pl) {
  const int As = c->A_create;
  struct Need {
    DevBuf *b;
    size_t bytes;
  } need[] = {
      {&m->roots, size_t(pl.n) * kStateBytes},
      {&m->q0, size_t(pl.n) * As * 4},
      {&m->L1, size_t(std::max<int64_t>(pl.n1, 1)) * kStateBytes},
      {&m->r1, size_t(std::max<int64_t>(pl.n1, 1)) * 4},
      {&m->maxq1, size_t(std::max<int64_t>(pl.n1, 1)) * 4},
      {&m->nodeA1, size_t(std::max<int64_t>(pl.n1, 1))},
      {&m->mid[0], size_t(std::max<int64_t>(pl.mid, 1)) * kStateBytes},
      {&m->mid[1], size_t(std::max<int64_t>(pl.mid, 1)) * kStateBytes},
      {&m->Rmid[0], size_t(std::max<int64_t>(pl.mid, 1)) * 4},
      {&m->Rmid[1], size_t(std::max<int64_t>(pl.mid, 1)) * 4},
      {&m->leaves, size_t(std::max<int64_t>(pl.nleaf, 1)) * kStateBytes},
      {&m->Rleaf, size_t(std::max<int64_t>(pl.nleaf, 1)) * 4},
      {&m->maxq_leaf, size_t(std::max<int64_t>(pl.nleaf, 1)) * 4},
      {&m->nodeA_leaf, size_t(std::max<int64_t>(pl.nleaf, 1))},
      {&m->V, size_t(pl.n) * As * 4},
      {&m->act, size_t(pl.n) * 4},
      {&m->val, size_t(pl.n) * As * 4},
      {&m->zbuf, pl.use_z ? size_t(pl.nz) * kP1 * kC1 * 4 : 1},
      {&m->zparent, pl.use_z ? size_t(std::max<int64_t>(pl.nleaf, 1)) * 4 : 1},
  };
  for (auto &x : need) {
    const int rc = c->ensure(*x.b, x.bytes);  // bumps the context's buffer generation when it moves
    if (rc != BCTS_OK) return rc;
  }
  const size_t host_bytes = size_t(pl.n) * (kStateBytes + 4 + As * 4) + 64;
  if (host_bytes > m->host.cap) {
    const int rc = c->ensure_host(m->host, host_bytes);
    if (rc != BCTS_OK) return rc;
    c->buf_generation++;
  }
  return BCTS_OK;
}

// Parent (in the union partial-map buffer) of each of a group's leaves.
__global__ void zparent_fill_kernel(uint32_t *__restrict__ zp, int64_t n, int A, uint32_t zoff) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) zp[i] = zoff + uint32_t(i / A);
}

// Every device step of one pass, in stream order (capturable: no allocation,
// no synchronisation).  Inputs are in the pinned staging area.
static int mixed_enqueue(Ctx *c, MixedState *m, const MixedPlan &pl, cudaStream_t st) {
  const int As = c->A_create;
  char *hs = static_cast<char *>(m->host.p);
  const size_t in_b = size_t(pl.n) * kStateBytes;
  int rc;
  BCTS_CUDA_TRY(cudaMemcpyAsync(m->roots.p, hs, in_b, cudaMemcpyHostToDevice, st), c->err);
  const bcts_state *roots = static_cast<const bcts_state *>(m->roots.p);
  float *q0 = static_cast<float *>(m->q0.p);
  c->A = As;
  // root evaluation over all roots (all As columns; each root reads its first A)
  if ((rc = c->eval_nodes_ref(roots, pl.n, q0, nullptr, st)) != BCTS_OK) return rc;
  bcts_state *L1 = static_cast<bcts_state *>(m->L1.p);
  float *r1 = static_cast<float *>(m->r1.p);
  uint8_t *nA1 = static_cast<uint8_t *>(m->nodeA1.p);
  // One expansion launch per level for all groups that reach it (work lists of up
  // to kMaxListGroups groups).  dst(g) gives a group's destination states and R.
  auto expand_level = [&](const std::vector<const MixedGroup *> &gs, auto src, auto dst, double gp) -> int {
    for (size_t s0 = 0; s0 < gs.size(); s0 += kMaxListGroups) {
      ExpandList L;
      uint32_t blocks = 0;
      for (size_t k = s0; k < gs.size() && L.n < kMaxListGroups; ++k) {
        const MixedGroup &g = *gs[k];
        const auto sp = src(g);
        const auto dp = dst(g);
        L.parents[L.n] = sp.first;
        L.parent_R[L.n] = sp.second;
        L.children[L.n] = dp.first;
        L.child_R[L.n] = dp.second;
        L.A[L.n] = g.A;
        L.gamma_pow[L.n] = float(gp);
        L.n_child[L.n] = uint32_t(dp.count);
        blocks += uint32_t((dp.count + 255) / 256);
        L.block_end[L.n] = blocks;
        ++L.n;
      }
      if (launch_expand_list(L, st) != BCTS_OK) return c->fail(BCTS_ECUDA, "expand launch failed");
    }
    return BCTS_OK;
  };
  struct Dst {
    bcts_state *first;
    float *second;
    int64_t count;
  };
  {
    std::vector<const MixedGroup *> gs;
    for (const MixedGroup &g : pl.groups)
      if (g.d >= 1) gs.push_back(&g);
    rc = expand_level(
        gs, [&](const MixedGroup &g) { return std::make_pair(roots + g.root_off, static_cast<const float *>(nullptr)); },
        [&](const MixedGroup &g) { return Dst{L1 + g.l1_off, r1 + g.l1_off, int64_t(g.n) * g.A}; }, 1.0);
    if (rc != BCTS_OK) return rc;
    for (const MixedGroup *g : gs)
      BCTS_CUDA_TRY(cudaMemsetAsync(nA1 + g->l1_off, g->A, size_t(g->n) * g->A, st), c->err);
  }
  float *maxq1 = static_cast<float *>(m->maxq1.p);
  if (pl.n1 > 0 && (rc = c->eval_nodes_ref(L1, pl.n1, nullptr, maxq1, st, nA1)) != BCTS_OK) return rc;
  bcts_state *leaves = static_cast<bcts_state *>(m->leaves.p);
  float *Rleaf = static_cast<float *>(m->Rleaf.p);
  uint8_t *nAl = static_cast<uint8_t *>(m->nodeA_leaf.p);
  // levels 1 .. d-1 -> 2 .. d: a group's level i lives in L1 (i = 1) or at its
  // offset in mid[i & 1] (2 <= i < d); its last expansion writes its leaves
  int maxd = 0;
  for (const MixedGroup &g : pl.groups) maxd = std::max(maxd, g.d);
  double gp = 1.0;
  auto level_src = [&](const MixedGroup &g, int i) {
    if (i == 1) return std::make_pair(static_cast<const bcts_state *>(L1 + g.l1_off), static_cast<const float *>(r1 + g.l1_off));
    return std::make_pair(static_cast<const bcts_state *>(static_cast<bcts_state *>(m->mid[i & 1].p) + g.mid_off[i]),
                          static_cast<const float *>(static_cast<float *>(m->Rmid[i & 1].p) + g.mid_off[i]));
  };
  for (int i = 1; i < maxd; ++i) {
    gp *= double(c->gamma);
    std::vector<const MixedGroup *> gs;
    for (const MixedGroup &g : pl.groups) {
      if (g.d <= i) continue;
      gs.push_back(&g);
      if (i == g.d - 1 && pl.use_z) {
        // the leaves' parents: their partial conv1 maps, and each leaf's parent index
        const int64_t cnt = int64_t(g.n) * ipow(g.A, i);
        const bcts_state *cur = level_src(g, i).first;
        float *z = static_cast<float *>(m->zbuf.p) + size_t(g.zoff) * kP1 * kC1;
        const int64_t chunk = c->chunk_nodes(cnt);
        for (int64_t off = 0; off < cnt; off += chunk) {
          const int64_t k = cnt - off < chunk ? cnt - off : chunk;
          if ((rc = tc_conv1_partial(c->tc, cur + off, k, z + size_t(off) * kP1 * kC1, st, c->d_err)) != BCTS_OK)
            return c->fail(rc, "conv1 partial launch failed");
        }
        zparent_fill_kernel<<<unsigned((g.nleaf + 255) / 256), 256, 0, st>>>(
            static_cast<uint32_t *>(m->zparent.p) + g.leaf_off, g.nleaf, g.A, uint32_t(g.zoff));
        if (cudaGetLastError() != cudaSuccess) return c->fail(BCTS_ECUDA, "parent table launch failed");
      }
    }
    rc = expand_level(
        gs, [&](const MixedGroup &g) { return level_src(g, i); },
        [&](const MixedGroup &g) {
          const int64_t cnt = int64_t(g.n) * ipow(g.A, i + 1);
          if (i + 1 == g.d) return Dst{leaves + g.leaf_off, Rleaf + g.leaf_off, cnt};
          return Dst{static_cast<bcts_state *>(m->mid[(i + 1) & 1].p) + g.mid_off[i + 1],
                     static_cast<float *>(m->Rmid[(i + 1) & 1].p) + g.mid_off[i + 1], cnt};
        },
        gp);
    if (rc != BCTS_OK) return rc;
  }
  for (const MixedGroup &g : pl.groups)
    if (g.d >= 2) BCTS_CUDA_TRY(cudaMemsetAsync(nAl + g.leaf_off, g.A, size_t(g.nleaf), st), c->err);
  float *maxq_leaf = static_cast<float *>(m->maxq_leaf.p);
  if (pl.nleaf > 0 &&
      (rc = c->eval_nodes(leaves, pl.nleaf, nullptr, maxq_leaf, st, nAl,
                          pl.use_z ? static_cast<const float *>(m->zbuf.p) : nullptr, 0,
                          pl.use_z ? static_cast<const uint32_t *>(m->zparent.p) : nullptr)) != BCTS_OK)
    return rc;
  // backup of every group: one segment-max and one finalize launch per work list
  float *V = static_cast<float *>(m->V.p);
  int32_t *act = static_cast<int32_t *>(m->act.p);
  float *val = static_cast<float *>(m->val.p);
  // groups whose subtrees are too long for one warp per segment (A^(d-1) >= 8192
  // leaves) back up with their own launches
  std::vector<const MixedGroup *> listed;
  for (const MixedGroup &g : pl.groups) {
    if (g.d >= 1 && ipow(g.A, g.d - 1) >= 8192) {
      double gd = 1.0;
      for (int i = 0; i < g.d; ++i) gd *= double(c->gamma);
      float *gV = V + size_t(g.root_off) * As;
      if ((rc = launch_segment_max(Rleaf + g.leaf_off, maxq_leaf + g.leaf_off, int64_t(g.n) * g.A,
                                   ipow(g.A, g.d - 1), float(gd), gV, st)) != BCTS_OK ||
          (rc = launch_finalize(q0 + size_t(g.root_off) * As, maxq1 + g.l1_off, r1 + g.l1_off, gV, g.n, g.A, g.d,
                                As, c->gamma, float(gd), c->corr, act + g.root_off, val + size_t(g.root_off) * As,
                                st, As, c->exact_gev ? 1 : 0)) != BCTS_OK)
        return c->fail(rc, "backup launch failed");
    } else {
      listed.push_back(&g);
    }
  }
  for (size_t s0 = 0; s0 < listed.size(); s0 += kMaxListGroups) {
    BackupList L;
    L.A_stride = As;
    L.q_stride = As;
    L.exact_gev = c->exact_gev ? 1 : 0;
    L.gamma = c->gamma;
    L.corr = c->corr;
    int64_t segs = 0, nroots = 0;
    for (size_t k = s0; k < listed.size() && L.n < kMaxListGroups; ++k) {
      const MixedGroup &g = *listed[k];
      double gd = 1.0;
      for (int i = 0; i < g.d; ++i) gd *= double(c->gamma);
      const int j = L.n;
      L.R[j] = g.d == 1 ? r1 + g.l1_off : (g.d >= 2 ? Rleaf + g.leaf_off : nullptr);
      L.maxq[j] = g.d == 1 ? maxq1 + g.l1_off : (g.d >= 2 ? maxq_leaf + g.leaf_off : nullptr);
      L.V[j] = V + size_t(g.root_off) * As;  // [n_g][A_g] inside the group's rows
      L.q0[j] = q0 + size_t(g.root_off) * As;
      L.maxq1[j] = g.d >= 1 ? maxq1 + g.l1_off : nullptr;
      L.r1[j] = g.d >= 1 ? r1 + g.l1_off : nullptr;
      L.action[j] = act + g.root_off;
      L.values[j] = val + size_t(g.root_off) * As;
      L.A[j] = g.A;
      L.depth[j] = g.d;
      L.seg_len[j] = g.d >= 1 ? uint32_t(ipow(g.A, g.d - 1)) : 1u;
      L.gamma_d[j] = float(gd);
      segs += g.d >= 1 ? int64_t(g.n) * g.A : 0;
      nroots += g.n;
      L.seg_end[j] = segs;
      L.root_end[j] = nroots;
      ++L.n;
    }
    if ((rc = launch_backup_list(L, st)) != BCTS_OK) return c->fail(rc, "backup launch failed");
  }
  BCTS_CUDA_TRY(cudaMemcpyAsync(hs + in_b, act, size_t(pl.n) * 4, cudaMemcpyDeviceToHost, st), c->err);
  BCTS_CUDA_TRY(
      cudaMemcpyAsync(hs + in_b + size_t(pl.n) * 4, val, size_t(pl.n) * As * 4, cudaMemcpyDeviceToHost, st),
      c->err);
  return BCTS_OK;
}

static void load_tune(MixedState *m) {
  m->tune_loaded = true;
  const std::string f = tune_file();
  if (f.empty()) return;
  std::ifstream in(f);
  std::string line;
  while (std::getline(in, line)) {  // lines: "<precision>:<bucket> <chunk> <conv mask>"
    std::istringstream ss(line);
    std::string k;
    int64_t v;
    int mask;
    if (ss >> k >> v >> mask) m->tuned[k] = {v, mask};
  }
}

static void save_tune(MixedState *m) {
  const std::string f = tune_file();
  if (f.empty()) return;
  std::ofstream out(f);
  for (auto &kv : m->tuned) out << kv.first << " " << kv.second.chunk << " " << kv.second.conv_mask << "\n";
}

// Pick the union-leaf configuration for this bucket by timing the candidates
// (leaf chunk x conv2 / conv3 kernel variant) on the plan's own leaves (first
// pass of a new bucket only; each candidate is run once to size its scratch and
// once timed).  The candidate kernels sum every output's products in the same
// order as the precision's default ones (conv2 through the same one of its
// three summation orders as the default; conv3 through any of its three
// kernels), so a root's result does not depend on the bucket its pass falls
// into.  A mask fixed through BCTS_CONV_KERNELS is kept; only the chunk is tuned
// then.
// conv2's summation order under a kernel mask: 0 im2col rows (cp.async gather or
// TMA im2col), 1 shared-memory windows, 2 tap pairs (E4M3 has no tap-pair kernel).
static int conv2_order(int mask, int precision) {
  if ((mask & 16) && precision != BCTS_PREC_FP8) return 2;
  return (mask & 4) ? 1 : 0;
}
static int autotune(Ctx *c, MixedState *m, const MixedPlan &pl, cudaStream_t st) {
  if (c->opt.leaf_chunk > 0 || pl.nleaf < 65536 || c->precision == BCTS_PREC_FP32_SIMT) return BCTS_OK;
  if (!m->tune_loaded) load_tune(m);
  const int dm = c->conv_mask_fixed ? c->conv_mask : tc_default_conv_mask(c->precision);
  const std::string key = std::to_string(c->precision) + ":" + std::to_string(leaf_bucket(pl.nleaf)) +
                          (c->conv_mask_fixed ? ":m" + std::to_string(dm) : std::string());
  auto it = m->tuned.find(key);
  const int order = conv2_order(dm, c->precision);
  if (it != m->tuned.end() && conv2_order(it->second.conv_mask, c->precision) == order) {
    c->chunk_override = it->second.chunk;
    c->conv_mask = it->second.conv_mask;
    return BCTS_OK;
  }
  const int64_t chunks[] = {32768, 65536, 0};  // 0: the automatic pass size (Ctx::chunk_nodes)
  // conv2 / conv3 kernels: bits 0 / 1 TMA im2col, bits 2 / 3 shared-memory
  // windows, bit 4 conv2 tap pairs
  std::vector<int> masks;
  if (c->conv_mask_fixed) {
    masks.push_back(dm);
  } else {
    const std::vector<int> c2s = order == 2 ? std::vector<int>{16} : (order == 1 ? std::vector<int>{4} : std::vector<int>{0, 1});
    for (int c2 : c2s)
      for (int c3 : {0, 2, 8}) masks.push_back(c2 | c3);
  }
  float best_ms = 1e30f;
  MixedState::Tuned best{32768, -1};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = BCTS_OK;
  for (int64_t chunk : chunks) {
    for (int mask : masks) {
      c->chunk_override = chunk;
      c->conv_mask = mask;
      float ms = 0.f;
      for (int rep = 0; rep < 2 && rc == BCTS_OK; ++rep) {
        cudaEventRecord(e0, st);
        rc = c->eval_nodes(static_cast<bcts_state *>(m->leaves.p), pl.nleaf, nullptr,
                           static_cast<float *>(m->maxq_leaf.p), st, static_cast<uint8_t *>(m->nodeA_leaf.p));
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
      }
      if (rc != BCTS_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = {chunk, mask};
      }
    }
    if (rc != BCTS_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != BCTS_OK) return rc;
  c->chunk_override = best.chunk;
  c->conv_mask = best.conv_mask;
  m->tuned[key] = best;
  save_tune(m);
  return BCTS_OK;
}

int Ctx::run_mixed(const bcts_state *, const bcts_state *h_roots, const int32_t *depths, const int32_t *actions,
                   int n, int32_t *, float *) {
  const int As = A_create;
  for (int i = 0; i < n; ++i)
    if (depths[i] < 0 || depths[i] > kMaxDepth || actions[i] < 1 || actions[i] > As)
      return fail(BCTS_EINVAL, "bcts_search_mixed: root " + std::to_string(i) + " has depth or A out of range");
  if (!mixed) mixed = new MixedState();
  MixedState *m = mixed;
  // plan: sort roots by (A, d)
  MixedPlan pl;
  pl.n = n;
  pl.order.resize(n);
  for (int i = 0; i < n; ++i) pl.order[i] = i;
  std::stable_sort(pl.order.begin(), pl.order.end(), [&](int a, int b) {
    return actions[a] != actions[b] ? actions[a] < actions[b] : depths[a] < depths[b];
  });
  std::ostringstream key;
  for (int i = 0; i < n;) {
    MixedGroup g;
    g.A = actions[pl.order[i]];
    g.d = depths[pl.order[i]];
    g.root_off = i;
    int j = i;
    while (j < n && actions[pl.order[j]] == g.A && depths[pl.order[j]] == g.d) ++j;
    g.n = j - i;
    g.l1_off = pl.n1;
    if (g.d >= 1) pl.n1 += int64_t(g.n) * g.A;
    if (g.d >= 2) {
      g.nleaf = int64_t(g.n) * ipow(g.A, g.d);
      g.leaf_off = pl.nleaf;
      pl.nleaf += g.nleaf;
      g.zoff = pl.nz;
      pl.nz += int64_t(g.n) * ipow(g.A, g.d - 1);
      // intermediate levels 2 .. d-1: every group's level i in one buffer (mid[i & 1])
      for (int lv = 2; lv < g.d; ++lv) {
        g.mid_off[lv] = pl.mid_fill[lv];
        pl.mid_fill[lv] += int64_t(g.n) * ipow(g.A, lv);
        pl.mid = std::max<int64_t>(pl.mid, pl.mid_fill[lv]);
      }
    }
    if (pl.nleaf > 0x7FFFFFFFLL) return fail(BCTS_EINVAL, "batched search too large: more than 2^31 - 1 leaves");
    key << g.A << "x" << g.d << "x" << g.n << ";";
    pl.groups.push_back(g);
    i = j;
  }
  key << "p" << precision;
  pl.key = key.str();
  pl.use_z = tc && tc_fused_render && tc_has_partial(tc) && pl.nleaf > 0 &&
             size_t(pl.nz) * kP1 * kC1 * sizeof(float) <= kMaxZBytes;
  int rc;
  if ((rc = mixed_ensure(this, m, pl)) != BCTS_OK) return rc;
  char *hs = static_cast<char *>(m->host.p);
  for (int i = 0; i < n; ++i) std::memcpy(hs + size_t(i) * kStateBytes, h_roots + pl.order[i], kStateBytes);
  if ((rc = autotune(this, m, pl, stream)) != BCTS_OK) return rc;
  if (m->seen.size() >= kMaxSeen) m->seen.clear();
  const int times_seen = m->seen[pl.key]++;
  auto git = m->graphs.find(pl.key);
  if (git != m->graphs.end() && git->second.generation == buf_generation && git->second.exec) {
    git->second.last_use = ++m->use_clock;
    BCTS_CUDA_TRY(cudaGraphLaunch(git->second.exec, stream), err);
    profiler_add(prof, git->second.launches);
  } else if (times_seen >= 1) {
    // second pass of this composition: capture it, then replay from now on
    if (git != m->graphs.end()) {
      if (git->second.exec) cudaGraphExecDestroy(git->second.exec);
      m->graphs.erase(git);
    }
    if (m->graphs.size() >= kMaxGraphs) {  // evict the least recently launched graph
      auto lru = m->graphs.begin();
      for (auto it = m->graphs.begin(); it != m->graphs.end(); ++it)
        if (it->second.last_use < lru->second.last_use) lru = it;
      if (lru->second.exec) cudaGraphExecDestroy(lru->second.exec);
      m->graphs.erase(lru);
    }
    Profiler *counter = profiler_create();
    cudaGraph_t graph = nullptr;
    BCTS_CUDA_TRY(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), err);
    int64_t launches = 0;
    {
      ProfilerGuard pg(counter);  // counts launches, records no events
      rc = mixed_enqueue(this, m, pl, stream);
      launches = profiler_total(counter);
    }
    const cudaError_t ce = cudaStreamEndCapture(stream, &graph);
    profiler_destroy(counter);
    if (rc != BCTS_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc != BCTS_OK ? rc : fail(BCTS_ECUDA, std::string("graph capture failed: ") + cudaGetErrorString(ce));
    }
    GraphEntry e;
    const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      return fail(BCTS_ECUDA, std::string("graph instantiate failed: ") + cudaGetErrorString(ie));
    }
    e.launches = launches;
    e.generation = buf_generation;
    e.last_use = ++m->use_clock;
    m->graphs[pl.key] = e;
    BCTS_CUDA_TRY(cudaGraphLaunch(e.exec, stream), err);
    profiler_add(prof, launches);
  } else {
    ProfilerGuard pg(prof);
    if ((rc = mixed_enqueue(this, m, pl, stream)) != BCTS_OK) return rc;
  }
  return BCTS_OK;
}

// Host part of the batched form: results come back in sorted order; scatter.
int Ctx::mixed_results(const int32_t *depths, const int32_t *actions, int n, int32_t *out_action,
                       float *out_values) {
  (void)depths;
  (void)actions;
  MixedState *m = mixed;
  const int As = A_create;
  // the same stable order the plan used
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return actions[a] != actions[b] ? actions[a] < actions[b] : depths[a] < depths[b];
  });
  const char *hs = static_cast<const char *>(m->host.p);
  const int32_t *hact = reinterpret_cast<const int32_t *>(hs + size_t(n) * kStateBytes);
  const float *hval = reinterpret_cast<const float *>(hs + size_t(n) * kStateBytes + size_t(n) * 4);
  for (int i = 0; i < n; ++i) {
    out_action[order[i]] = hact[i];
    std::memcpy(out_values + size_t(order[i]) * As, hval + size_t(i) * As, size_t(As) * 4);
  }
  return BCTS_OK;
}

}  // namespace bcts

extern "C" int bcts_search_mixed(bcts_ctx *ctx, const bcts_state *roots, const int32_t *depths,
                                 const int32_t *actions, int n, int32_t *out_action, float *out_values) {
  if (!ctx) return BCTS_EINVAL;
  bcts::Ctx *c = reinterpret_cast<bcts::Ctx *>(ctx);
  if (n < 0 || (n > 0 && (!roots || !depths || !actions || !out_action || !out_values)))
    return c->fail(BCTS_EINVAL, "bcts_search_mixed: invalid argument");
  if (n == 0) return BCTS_OK;
  const int saved_mask = c->conv_mask;
  int rc = c->run_mixed(nullptr, roots, depths, actions, n, nullptr, nullptr);
  if (rc != BCTS_OK) {
    cudaStreamSynchronize(c->stream);
    c->chunk_override = 0;
    c->conv_mask = saved_mask;
    return rc;
  }
  int herr = 0;
  BCTS_CUDA_TRY(cudaStreamSynchronize(c->stream), c->err);
  BCTS_CUDA_TRY(cudaMemcpy(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost), c->err);
  c->chunk_override = 0;
  c->conv_mask = saved_mask;
  if (herr != 0) {
    cudaMemset(c->d_err, 0, sizeof(int));
    return c->fail(BCTS_EDEVICE, "a kernel reported error code " + std::to_string(herr));
  }
  return c->mixed_results(depths, actions, n, out_action, out_values);
}
