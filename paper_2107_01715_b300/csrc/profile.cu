// profile.cu -- per-kernel-class device timing with CUDA events, and the launch
// counter behind bcts_profile.
#include <vector>

#include "search.cuh"

namespace bcts {

static_assert(int(K_COUNT) == int(BCTS_KERN_COUNT), "kernel classes must match the public enum");

struct Profiler {
  bool on = false;
  struct Pair {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Pair> pending;
  std::vector<cudaEvent_t> pool;
  std::vector<int> open_kind;
  std::vector<cudaEvent_t> open_ev;
  double ms[K_COUNT] = {};
  int64_t launches[K_COUNT] = {};
  int64_t total = 0;

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void drain() {
    for (auto &p : pending) {
      float t = 0.f;
      if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess)
        ms[p.kind] += t;
      cudaGetLastError();
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  ~Profiler() {
    drain();
    for (auto e : pool) cudaEventDestroy(e);
  }
};

Profiler *&thread_profiler() {
  static thread_local Profiler *p = nullptr;
  return p;
}

void prof_begin(int kind, cudaStream_t st) {
  Profiler *p = thread_profiler();
  if (!p) return;
  p->total++;
  p->launches[kind]++;
  if (!p->on) return;
  cudaEvent_t e = p->get();
  cudaEventRecord(e, st);
  p->open_kind.push_back(kind);
  p->open_ev.push_back(e);
}

void prof_end(int kind, cudaStream_t st) {
  Profiler *p = thread_profiler();
  if (!p || !p->on || p->open_ev.empty()) return;
  cudaEvent_t a = p->open_ev.back();
  p->open_ev.pop_back();
  p->open_kind.pop_back();
  cudaEvent_t b = p->get();
  cudaEventRecord(b, st);
  p->pending.push_back({kind, a, b});
  if (p->pending.size() > 4096) p->drain();
}

Profiler *profiler_create() { return new Profiler(); }
bool profiler_on(const Profiler *p) { return p && p->on; }
int64_t profiler_total(const Profiler *p) { return p->total; }
void profiler_add(Profiler *p, int64_t launches) { p->total += launches; }
void profiler_destroy(Profiler *p) { delete p; }

}  // namespace bcts

namespace bcts {
// Totals since the last read (then reset), recording switched on or off.
int profiler_read(Profiler *p, cudaStream_t st, int enable, double *out_ms, int64_t *out_launches,
                  int64_t *out_total) {
  cudaStreamSynchronize(st);
  p->drain();
  for (int k = 0; k < K_COUNT; ++k) {
    if (out_ms) out_ms[k] = p->ms[k];
    if (out_launches) out_launches[k] = p->launches[k];
    p->ms[k] = 0.0;
    p->launches[k] = 0;
  }
  if (out_total) *out_total = p->total;
  p->total = 0;
  p->on = enable != 0;
  return BCTS_OK;
}
}  // namespace bcts

extern "C" int bcts_profile(bcts_ctx *ctx, int enable, double *out_ms, int64_t *out_launches,
                            int64_t *out_total) {
  if (!ctx) return BCTS_EINVAL;
  bcts::Ctx *c = reinterpret_cast<bcts::Ctx *>(ctx);
  const int rc = bcts::profiler_read(c->prof, c->stream, enable, out_ms, out_launches, out_total);
  if (out_total) *out_total += bcts::serve_launches(c);  // the serving workers' launches too
  return rc;
}

