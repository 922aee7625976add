// mg_batch.cu -- batched setup of many independent levels (hierarchies of
// lattices of uneven volume, different m', k and aggregates).
//
// mg_batch_create validates the level descriptors, tunes the smoother's slab
// width (2 or 4 pairs of right-hand sides per CTA) once per distinct problem
// shape by timing both variants, runs every level once (so every kernel is
// loaded and configured before the capture), then captures every level's four setup calls
// into one CUDA graph that forks over S streams from the caller's stream and
// joins back: small levels run side by side and fill the GPU, and one
// cudaGraphLaunch replaces a few thousand kernel launches.  With
// n_streams <= 0 the stream count is tuned too (S = 1, 2, 4, 8: the fastest
// graph is kept).  mg_batch_launch replays the graph.
#include <chrono>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "mg_common.cuh"

// ---------------------------------------------------------------------------
// tuning table: problem shape -> slab width of the smoother passes
// ---------------------------------------------------------------------------
namespace mg {
namespace {
using ShapeKey = std::tuple<int, int, int, int, int, int, int>;
ShapeKey shape_key(const Geom& g) {
  return ShapeKey{g.L[0], g.L[1], g.L[2], g.L[3], g.m, g.prec, 0};
}
std::mutex g_tune_mu;
std::map<ShapeKey, int>& tune_table() {
  static auto* t = new std::map<ShapeKey, int>();  // never destroyed: safe at exit
  return *t;
}
thread_local bool t_timing_suspended = false;
}  // namespace

int tuned_pairs(const Geom& g) {
  std::lock_guard<std::mutex> l(g_tune_mu);
  auto it = tune_table().find(shape_key(g));
  return it == tune_table().end() ? 0 : it->second;
}

void set_tuned_pairs(const Geom& g, int pairs) {
  std::lock_guard<std::mutex> l(g_tune_mu);
  tune_table()[shape_key(g)] = pairs;
}

bool timing_suspended() { return t_timing_suspended; }

namespace {
struct SuspendTiming {
  bool old;
  SuspendTiming() : old(t_timing_suspended) { t_timing_suspended = true; }
  ~SuspendTiming() { t_timing_suspended = old; }
};

mg_status batch_fail(mg_status st, const char* what, cudaError_t e = cudaSuccess) {
  char msg[512];  // the size of the library's error message slot
  if (e != cudaSuccess)
    std::snprintf(msg, sizeof msg, "mg_batch: %s: %s", what, cudaGetErrorString(e));
  else
    std::snprintf(msg, sizeof msg, "mg_batch: %s", what);
  set_last_error(msg);
  return st;
}

mg_status run_level(const mg_level_desc& d, cudaStream_t s) {
  mg_status st = mg_smooth_testvecs(&d.prob, d.U, d.C, d.psi0, d.psi, d.ws_smooth,
                                    d.ws_smooth_bytes, s);
  if (st != MG_OK) return st;
  st = mg_chiral_truncate(&d.prob, d.psi, d.Uk, d.sigma, nullptr, d.blk_flags, d.ws_trunc,
                          d.ws_trunc_bytes, s);
  if (st != MG_OK) return st;
  st = mg_build_prolongator(&d.prob, d.Uk, d.P, s);
  if (st != MG_OK) return st;
  return mg_coarsen(&d.prob, d.U, d.C, d.P, d.X, d.Y, nullptr, 0, s);
}

// elapsed milliseconds of fn() enqueued on s (one warm-up, one timed run)
template <typename F>
float time_on(cudaStream_t s, F fn) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  fn();
  cudaEventRecord(a, s);
  fn();
  cudaEventRecord(b, s);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

struct Captured {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

mg_status capture(const std::vector<mg_level_desc>& lv, int S, Captured* out) {
  SuspendTiming no_timing;  // event records do not belong in the graph
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> side(S, nullptr);
  std::vector<cudaEvent_t> join(S, nullptr);
  cudaEvent_t fork = nullptr;
  mg_status st = MG_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  for (int i = 0; i < S && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    st = batch_fail(MG_ERR_CUDA, "stream setup", e);
  } else {
    cudaEventRecord(fork, cap);
    for (int i = 0; i < S; ++i) cudaStreamWaitEvent(side[i], fork, 0);
    for (size_t i = 0; i < lv.size() && st == MG_OK; ++i) st = run_level(lv[i], side[i % S]);
    for (int i = 0; i < S; ++i) {
      cudaEventRecord(join[i], side[i]);
      cudaStreamWaitEvent(cap, join[i], 0);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    if (st == MG_OK && e != cudaSuccess) st = batch_fail(MG_ERR_CUDA, "capture", e);
    if (st == MG_OK) {
      e = cudaGraphInstantiate(&out->exec, g, 0);
      if (e != cudaSuccess) st = batch_fail(MG_ERR_CUDA, "graph instantiation", e);
      out->graph = g;
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  for (int i = 0; i < S; ++i) {
    if (side[i]) cudaStreamDestroy(side[i]);
    if (join[i]) cudaEventDestroy(join[i]);
  }
  if (fork) cudaEventDestroy(fork);
  if (cap) cudaStreamDestroy(cap);
  return st;
}

void release(Captured& c) {
  if (c.exec) cudaGraphExecDestroy(c.exec);
  if (c.graph) cudaGraphDestroy(c.graph);
  c = Captured{};
}
}  // namespace
}  // namespace mg

using namespace mg;

struct mg_batch {
  Captured cap;
  int n_streams = 1;
  float ms_tuned = 0.f;
  std::vector<mg_level_desc> levels;
};

extern "C" {

mg_status mg_batch_create(const mg_level_desc* levels, int n, int n_streams, void* stream,
                          mg_batch** out) {
  if (!out) return batch_fail(MG_ERR_INVALID, "NULL output handle");
  *out = nullptr;
  if (!levels || n < 1) return batch_fail(MG_ERR_INVALID, "no levels");
  if (n_streams > 64) return batch_fail(MG_ERR_INVALID, "more than 64 streams");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<mg_level_desc> lv(levels, levels + n);
  // validation (every call checks again when it is captured)
  for (int i = 0; i < n; ++i) {
    const mg_level_desc& d = lv[i];
    Geom g;
    if (make_geom(&d.prob, &g) != MG_OK) {
      char msg[320];
      std::snprintf(msg, sizeof msg, "level %d: %s", i, mg_last_error());
      return batch_fail(MG_ERR_INVALID, msg);
    }
    if (!d.U || !d.psi0 || !d.psi || !d.Uk || !d.sigma || !d.blk_flags || !d.P || !d.X ||
        !d.Y || !d.ws_smooth || !d.ws_trunc) {
      char msg[96];
      std::snprintf(msg, sizeof msg, "level %d: NULL array", i);
      return batch_fail(MG_ERR_INVALID, msg);
    }
  }
  // tune the smoother's slab width once per shape (2 smoother iterations
  // stand in for the full count: the passes are the same)
  for (int i = 0; i < n; ++i) {
    Geom g;
    make_geom(&lv[i].prob, &g);
    if (tuned_pairs(g) != 0 || g.m % 8 != 0) continue;
    mg_level_desc d = lv[i];
    d.prob.mr_iters = 2;
    float best = 1e30f;
    int best_p = 4;
    for (int p : {4, 2}) {
      set_tuned_pairs(g, p);
      SuspendTiming no_timing;
      const float ms = time_on(s, [&] {
        mg_smooth_testvecs(&d.prob, d.U, d.C, d.psi0, d.psi, d.ws_smooth, d.ws_smooth_bytes, s);
      });
      if (ms < best) {
        best = ms;
        best_p = p;
      }
    }
    set_tuned_pairs(g, best_p);
  }
  // one short run of every level before the capture: each kernel the graph
  // will hold is loaded and configured (function attributes) outside it
  for (int i = 0; i < n; ++i) {
    mg_level_desc d = lv[i];
    d.prob.mr_iters = 1;
    SuspendTiming no_timing;
    const mg_status st = run_level(d, s);
    if (st != MG_OK) return st;
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return batch_fail(MG_ERR_CUDA, "tuning", e);

  auto* b = new mg_batch();
  b->levels = lv;
  std::vector<int> cands;
  if (n_streams > 0) {
    cands.push_back(std::min(n_streams, n));
  } else {
    for (int S : {1, 2, 4, 8})
      if (S <= n) cands.push_back(S);
  }
  for (int S : cands) {
    Captured c;
    mg_status st = capture(lv, S, &c);
    if (st != MG_OK) {
      release(b->cap);
      delete b;
      return st;
    }
    float ms = 0.f;
    if (cands.size() > 1) {
      ms = time_on(s, [&] { cudaGraphLaunch(c.exec, s); });
      e = cudaGetLastError();
      if (e != cudaSuccess) {
        release(c);
        release(b->cap);
        delete b;
        return batch_fail(MG_ERR_CUDA, "tuning launch", e);
      }
    }
    if (!b->cap.exec || ms < b->ms_tuned) {
      release(b->cap);
      b->cap = c;
      b->n_streams = S;
      b->ms_tuned = ms;
    } else {
      release(c);
    }
  }
  *out = b;
  return MG_OK;
}

mg_status mg_batch_launch(mg_batch* batch, void* stream) {
  if (!batch || !batch->cap.exec) return batch_fail(MG_ERR_INVALID, "NULL batch");
  const cudaError_t e = cudaGraphLaunch(batch->cap.exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return batch_fail(MG_ERR_CUDA, "cudaGraphLaunch", e);
  return MG_OK;
}

int mg_batch_streams(const mg_batch* batch) { return batch ? batch->n_streams : 0; }

void mg_batch_destroy(mg_batch* batch) {
  if (!batch) return;
  release(batch->cap);
  delete batch;
}

int mg_tuned_pairs(const mg_problem* prob) {
  Geom g;
  if (make_geom(prob, &g) != MG_OK) return -1;
  const int p = tuned_pairs(g);
  return p != 0 ? p : (g.m % 8 == 0 ? 4 : 2);
}

}  // extern "C"
