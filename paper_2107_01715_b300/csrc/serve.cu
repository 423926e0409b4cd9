// serve.cu -- serving form: continuous batching of decision requests.
//
// bcts_submit queues a request (root, d, A) and returns a ticket at once.  Three
// worker threads, each with its own stream and buffers (a context sharing the
// owner's weights), repeatedly take as many queued requests as the pass limit
// and the admission budget allow and run them as one batched search pass (the
// mixed form: every Q-network evaluation of the pass in one batch).  Requests
// that arrive while passes are on the GPU wait only for the next free worker,
// so up to three passes overlap on the device.  A request is admitted while the
// device bytes its part of a pass occupies (request_cost) fit in what the
// budget has left; a request larger than the whole budget runs alone.
// bcts_poll returns a request's result as soon as its pass has finished.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "search.cuh"

namespace bcts {

struct ServeRequest {
  bcts_state root;
  int d = 0, A = 0;
  int status = BCTS_PENDING;
  int32_t action = -1;
  std::vector<float> values;
  size_t cost = 0;    // device bytes it occupies in a pass (request_cost)
  size_t leaves = 0;  // A^d
};

struct ServeState {
  Ctx *owner = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, ServeRequest> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  size_t budget = 0, inflight = 0;
  int max_batch = 64;
  int busy_workers = 0;
  size_t queued_leaves = 0;  // leaves of the queued requests
  static constexpr int kWorkers = 3;
  std::thread worker[kWorkers];
  Ctx *wctx[kWorkers] = {};
};

namespace {

// batching window (measured, Poisson arrivals, BF16, 4 s, two runs each: 500 us
// against 2 ms gives p50 1.27 / 2.34 ms instead of 1.60 / 2.77 ms at 300 / 500
// req/s, the same p99 and the same saturated throughput at 2,000 req/s)
constexpr auto kWindow = std::chrono::microseconds(500);
constexpr size_t kFullPassLeaves = size_t(1) << 20;  // about 1M leaves keep all SMs busy

// Device bytes one request occupies in a batched pass (mixed.cu's buffers): its
// node levels (80-byte state + FP32 R each; intermediate levels ping-pong), per
// leaf its max Q, action count and parent index, the FP32 partial conv1 map of
// each of its leaves' parents (51,200 bytes), and its root's and depth-1 nodes'
// values.  The Q-network's activation maps of a leaf chunk are a per-worker
// constant, not charged per request.
size_t request_cost(int A, int d) {
  size_t lvl[kMaxDepth + 2] = {1};
  for (int i = 1; i <= d; ++i) lvl[i] = lvl[i - 1] * size_t(A);
  size_t bytes = size_t(kStateBytes) + 3 * size_t(A) * 4 + 16;  // root, q0 / V / values
  if (d >= 1) bytes += lvl[1] * (kStateBytes + 4 + 4 + 1);       // depth 1: state, r, max Q, A
  for (int i = 2; i < d; ++i) bytes += lvl[i] * (kStateBytes + 4);
  if (d >= 2) bytes += lvl[d] * (kStateBytes + 4 + 4 + 1 + 4) + lvl[d - 1] * size_t(kP1) * kC1 * 4;
  return bytes;
}

// A context that shares `o`'s weights and owns its own stream and buffers.
Ctx *clone_ctx(const Ctx *o) {
  Ctx *c = new Ctx();
  c->device = o->device;
  c->A = c->A_create = o->A_create;
  c->d = o->d;
  c->gamma = o->gamma;
  c->corr = o->corr;
  c->precision = o->precision;
  c->opt = o->opt;
  // serving passes rarely repeat a composition: a fixed leaf chunk instead of
  // timing candidates on the first pass of every new size
  if (c->opt.leaf_chunk <= 0) c->opt.leaf_chunk = 32768;
  c->simt = o->simt;
  c->tc = o->tc;
  c->tc_ref = o->tc_ref;
  c->conv_mask = o->conv_mask;
  c->dev_mem = o->dev_mem;
  c->conv_mask_fixed = o->conv_mask_fixed;
  c->tc_fused_render = o->tc_fused_render;
  c->exact_gev = o->exact_gev;
  c->owns_weights = false;
  c->prof = profiler_create();
  if (cudaSetDevice(o->device) != cudaSuccess || cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess || cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return nullptr;
  }
  return c;
}

void worker_loop(ServeState *s, int w) {
  Ctx *c = s->wctx[w];
  cudaSetDevice(c->device);
  std::vector<uint64_t> batch;
  std::vector<bcts_state> roots;
  std::vector<int32_t> depths, actions, out_act;
  std::vector<float> out_val;
  for (;;) {
    size_t cost = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
      if (s->stop && s->queue.empty()) return;
      // batching window: while another pass keeps the GPU busy, a small queue
      // waits (up to kWindow) for more requests, so that passes stay large
      // enough to fill the device instead of splitting the load into many
      // small passes; an idle device starts at once
      const auto until = std::chrono::steady_clock::now() + kWindow;
      while (!s->stop && s->busy_workers > 0 && int(s->queue.size()) < s->max_batch &&
             s->queued_leaves < kFullPassLeaves) {
        if (s->cv_work.wait_until(lk, until) == std::cv_status::timeout) break;
      }
      if (s->queue.empty()) continue;
      batch.clear();
      // admission: FIFO while the pass limit and the budget allow (the first
      // request of a pass is always admitted once nothing else is in flight)
      while (!s->queue.empty() && int(batch.size()) < s->max_batch) {
        ServeRequest &r = s->reqs[s->queue.front()];
        const bool fits = s->inflight + cost + r.cost <= s->budget;
        if (!fits && !(batch.empty() && s->inflight == 0)) break;
        cost += r.cost;
        s->queued_leaves -= r.leaves;
        batch.push_back(s->queue.front());
        s->queue.pop_front();
      }
      if (batch.empty()) {
        // nothing fits until another pass finishes
        s->cv_work.wait(lk, [&] { return s->stop || s->inflight == 0 || s->queue.empty(); });
        continue;
      }
      s->inflight += cost;
      ++s->busy_workers;
      roots.resize(batch.size());
      depths.resize(batch.size());
      actions.resize(batch.size());
      for (size_t i = 0; i < batch.size(); ++i) {
        const ServeRequest &r = s->reqs[batch[i]];
        roots[i] = r.root;
        depths[i] = r.d;
        actions[i] = r.A;
      }
    }
    const int n = int(batch.size());
    out_act.assign(n, -1);
    out_val.assign(size_t(n) * c->A_create, 0.f);
    int rc = bcts_search_mixed(reinterpret_cast<bcts_ctx *>(c), roots.data(), depths.data(), actions.data(), n,
                               out_act.data(), out_val.data());
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (int i = 0; i < n; ++i) {
        auto it = s->reqs.find(batch[i]);
        if (it == s->reqs.end()) continue;
        ServeRequest &r = it->second;
        r.status = rc;
        if (rc == BCTS_OK) {
          r.action = out_act[i];
          r.values.assign(out_val.begin() + size_t(i) * c->A_create,
                          out_val.begin() + size_t(i) * c->A_create + r.A);
        }
      }
      s->inflight -= cost;
      --s->busy_workers;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

// Kernel launches of the serving workers since the last call (their counters reset).
int64_t serve_launches(Ctx *c) {
  ServeState *s = c->serve;
  if (!s) return 0;
  int64_t total = 0;
  for (Ctx *w : s->wctx) {
    if (!w || !w->prof) continue;
    int64_t t = 0;
    profiler_read(w->prof, w->stream, 0, nullptr, nullptr, &t);
    total += t;
  }
  return total;
}

void serve_shutdown(Ctx *c) {
  ServeState *s = c->serve;
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->worker)
    if (t.joinable()) t.join();
  for (Ctx *w : s->wctx) delete w;
  delete s;
  c->serve = nullptr;
}

static int serve_start(Ctx *c) {
  if (c->serve) return BCTS_OK;
  ServeState *s = new ServeState();
  s->owner = c;
  s->budget = c->opt.frame_budget_bytes ? c->opt.frame_budget_bytes : (size_t(8) << 30);
  s->max_batch = c->opt.max_roots > 0 ? c->opt.max_roots : 64;
  for (int w = 0; w < ServeState::kWorkers; ++w) {
    s->wctx[w] = clone_ctx(c);
    if (!s->wctx[w]) {
      for (Ctx *x : s->wctx) delete x;
      delete s;
      return c->fail(BCTS_ECUDA, "serving worker set-up failed");
    }
  }
  for (int w = 0; w < ServeState::kWorkers; ++w) s->worker[w] = std::thread(worker_loop, s, w);
  c->serve = s;
  return BCTS_OK;
}

}  // namespace bcts

static std::mutex g_serve_start_mu;

extern "C" int bcts_submit(bcts_ctx *ctx, const bcts_state *root, int d, int A, uint64_t *out_ticket) {
  if (!ctx) return BCTS_EINVAL;
  bcts::Ctx *c = reinterpret_cast<bcts::Ctx *>(ctx);
  if (!root || !out_ticket || d < 0 || d > bcts::kMaxDepth || A < 1 || A > c->A_create) {
    bcts::set_thread_error("bcts_submit: invalid argument");
    return BCTS_EINVAL;
  }
  {
    std::lock_guard<std::mutex> lk(g_serve_start_mu);
    const int rc = bcts::serve_start(c);
    if (rc != BCTS_OK) return rc;
  }
  bcts::ServeState *s = c->serve;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t t = s->next_ticket++;
    bcts::ServeRequest &r = s->reqs[t];
    r.root = *root;
    r.d = d;
    r.A = A;
    r.cost = bcts::request_cost(A, d);
    r.leaves = 1;
    for (int i = 0; i < d; ++i) r.leaves *= size_t(A);
    s->queued_leaves += r.leaves;
    s->queue.push_back(t);
    *out_ticket = t;
  }
  s->cv_work.notify_one();
  return BCTS_OK;
}

extern "C" int bcts_poll(bcts_ctx *ctx, uint64_t ticket, int32_t *out_action, float *out_values, int timeout_us) {
  if (!ctx) return BCTS_EINVAL;
  bcts::Ctx *c = reinterpret_cast<bcts::Ctx *>(ctx);
  bcts::ServeState *s = c->serve;
  if (!s) return BCTS_ENOTICKET;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return BCTS_ENOTICKET;
  auto done = [&] {
    auto j = s->reqs.find(ticket);
    return j == s->reqs.end() || j->second.status != BCTS_PENDING;
  };
  if (!done() && timeout_us != 0) {
    if (timeout_us < 0)
      s->cv_done.wait(lk, done);
    else
      s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done);
  }
  it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return BCTS_ENOTICKET;
  bcts::ServeRequest &r = it->second;
  if (r.status == BCTS_PENDING) return BCTS_PENDING;
  const int st = r.status;
  if (st == BCTS_OK) {
    if (out_action) *out_action = r.action;
    if (out_values) std::memcpy(out_values, r.values.data(), r.values.size() * sizeof(float));
  }
  s->reqs.erase(it);
  return st;
}
