// mg_abi.cu -- the extern "C" entry points declared in include/mg.h:
// argument validation, workspace layout and kernel dispatch.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "mg_common.cuh"

namespace mg {

namespace {
thread_local char g_err[512] = "";

mg_status fail(mg_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return st;
}

mg_status cuda_status(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return MG_OK;
  return fail(MG_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

}  // namespace

// Validate the problem and fill the geometry.
mg_status make_geom(const mg_problem* p, Geom* g) {
  if (!p) return fail(MG_ERR_INVALID, "problem is NULL");
  long V = 1;
  int nb = 1;
  for (int i = 0; i < 4; ++i) {
    if (p->dims[i] < 1 || p->block[i] < 1)
      return fail(MG_ERR_SHAPE, "dims and block extents must be >= 1");
    if (p->dims[i] % p->block[i] != 0)
      return fail(MG_ERR_SHAPE, "block extent %d does not divide lattice extent %d (direction %d)",
                  p->block[i], p->dims[i], i);
    V *= p->dims[i];
    nb *= p->block[i];
  }
  if (V > (1L << 30)) return fail(MG_ERR_SHAPE, "volume %ld too large", V);
  if (p->precision != MG_PREC_FP32 && p->precision != MG_PREC_MIXED &&
      p->precision != MG_PREC_MIXED_FP16)
    return fail(MG_ERR_UNSUPPORTED, "precision %d not implemented", p->precision);
  if (p->n_vec < 4 || p->n_vec > kMaxM || p->n_vec % 4 != 0)
    return fail(MG_ERR_UNSUPPORTED, "n_vec must be a multiple of 4 in [4, %d], got %d", kMaxM,
                p->n_vec);
  if (6 * nb < p->n_vec)
    return fail(MG_ERR_SHAPE, "block has 6*|Lambda| = %d rows < n_vec = %d", 6 * nb, p->n_vec);
  if (p->k < 1 || p->k > p->n_vec || p->k > kMaxK)
    return fail(MG_ERR_SHAPE, "k = %d must be in [1, min(n_vec, %d)]", p->k, kMaxK);
  if (!(p->xi > 0)) return fail(MG_ERR_INVALID, "xi must be positive");
  for (int i = 0; i < 4; ++i) {
    g->L[i] = p->dims[i];
    g->b[i] = p->block[i];
    g->Lc[i] = p->dims[i] / p->block[i];
  }
  g->V = V;
  g->nb = nb;
  g->nblk = V / nb;
  g->m = p->n_vec;
  g->prec = p->precision;
  g->k = p->k;
  g->niter = p->mr_iters;
  g->m0 = p->m0;
  g->xi = p->xi;
  double wsum = 0;
  for (int i = 0; i < 4; ++i) {
    const double w = i == 3 ? 1.0 / p->xi : 1.0;
    g->hw[i] = (float)(-0.5 * w);
    wsum += w;
  }
  g->diag = (float)(p->m0 + wsum);
  return MG_OK;
}

// Validates a level-l (l >= 1) problem.  full = false checks only what the
// stencil apply reads (dims, nc); full = true also the aggregation and the
// truncation parameters and fills g as the fine-level kernels of the
// truncation and the prolongator read it (rps = nc rows per site and
// chirality).
mg_status make_cgeom(const mg_coarse_problem* p, StencilGeom* sg, Geom* g, bool full) {
  if (!p) return fail(MG_ERR_INVALID, "problem is NULL");
  long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (p->dims[i] < 1) return fail(MG_ERR_SHAPE, "dims extents must be >= 1");
    V *= p->dims[i];
  }
  if (V > (1L << 26)) return fail(MG_ERR_SHAPE, "coarse volume %ld too large", V);
  if (p->nc < 1 || p->nc > 32)
    return fail(MG_ERR_UNSUPPORTED, "nc = %d must be in [1, 32]", p->nc);
  for (int i = 0; i < 4; ++i) sg->L[i] = p->dims[i];
  sg->V = V;
  sg->n = 2 * p->nc;
  if (!full) return MG_OK;
  int nb = 1;
  for (int i = 0; i < 4; ++i) {
    if (p->block[i] < 1) return fail(MG_ERR_SHAPE, "block extents must be >= 1");
    if (p->dims[i] % p->block[i] != 0)
      return fail(MG_ERR_SHAPE, "block extent %d does not divide lattice extent %d (direction %d)",
                  p->block[i], p->dims[i], i);
    nb *= p->block[i];
  }
  if (p->n_vec < 4 || p->n_vec > kMaxM || p->n_vec % 4 != 0)
    return fail(MG_ERR_UNSUPPORTED, "n_vec must be a multiple of 4 in [4, %d], got %d", kMaxM,
                p->n_vec);
  if (p->nc * nb < p->n_vec)
    return fail(MG_ERR_SHAPE, "block has nc*|Lambda| = %d rows < n_vec = %d", p->nc * nb,
                p->n_vec);
  if (p->k < 1 || p->k > p->n_vec || p->k > kMaxK)
    return fail(MG_ERR_SHAPE, "k = %d must be in [1, min(n_vec, %d)]", p->k, kMaxK);
  *g = Geom{};
  for (int i = 0; i < 4; ++i) {
    g->L[i] = p->dims[i];
    g->b[i] = p->block[i];
    g->Lc[i] = p->dims[i] / p->block[i];
  }
  g->V = V;
  g->nb = nb;
  g->nblk = V / nb;
  g->m = p->n_vec;
  g->k = p->k;
  g->niter = p->mr_iters;
  g->xi = 1.0;
  g->prec = MG_PREC_FP32;
  g->rps = p->nc;
  g->cps = 2 * p->nc;
  return MG_OK;
}

SmoothWs smooth_ws_layout(const Geom& g) {
  SmoothWs w{};
  // one spinor field: complex64 or, in the mixed-precision path, two FP16 per complex
  const size_t field = (g.prec == MG_PREC_MIXED_FP16 ? 4 : 8) * (size_t)g.V * 12 * g.m;
  size_t o = 0;
  w.ra = o; o = align256(o + field);
  w.wa = o; o = align256(o + field);
  w.ps = o; o = align256(o + field);
  w.rb = o; o = align256(o + field);
  // partial sums: one per (right-hand side, patch of 32 sites of a timeslice)
  const size_t npatch = ((size_t)(g.V / g.L[3]) + 31) / 32;
  w.part = o; o = align256(o + sizeof(double) * 4 * npatch * g.m);
  w.alpha = o; o = align256(o + sizeof(float2) * g.m);
  w.alpha_b = o; o = align256(o + sizeof(float2) * g.m);
  w.scale = o; o = align256(o + sizeof(float) * g.m);
  w.bytes = o;
  return w;
}

TruncWs trunc_ws_layout(const Geom& g) {
  TruncWs w{};
  const size_t nbc = 2 * (size_t)g.nblk;
  const size_t mm = (size_t)g.m * g.m;
  size_t o = 0;
  w.gram = o; o = align256(o + sizeof(double2) * nbc * mm);
  w.r1 = o; o = align256(o + sizeof(double2) * nbc * mm);
  w.z1 = o; o = align256(o + sizeof(float2) * nbc * mm);
  w.w2 = o; o = align256(o + sizeof(float2) * nbc * g.m * g.k);
  w.hm = o; o = align256(o + sizeof(double2) * nbc * mm);
  w.flags = o; o = align256(o + sizeof(int32_t) * nbc);
  w.q1 = w.qmax = 0;
  if (g.prec != MG_PREC_FP32 && tc_supported(g)) {
    // tensor-core path: Q1 = A R1^-1 of every block-chirality (as large as psi)
    // and the largest entry of each
    w.q1 = o; o = align256(o + sizeof(float2) * nbc * (size_t)g.cps * g.nb / 2 * g.m);
    w.qmax = o; o = align256(o + sizeof(float) * nbc);
  }
  w.bytes = o;
  return w;
}

void set_last_error(const char* msg) { std::snprintf(g_err, sizeof g_err, "%s", msg); }

// ---------------------------------------------------------------------------
// per-kernel timing
// ---------------------------------------------------------------------------
namespace {
struct TimingRec {
  int kind;
  cudaEvent_t a, b;
};
struct TimingState {
  std::mutex mu;
  std::atomic<bool> on{false};
  std::vector<std::string> kinds;
  std::vector<int64_t> launches;
  std::vector<double> ms;
  std::vector<TimingRec> pending;
  std::vector<cudaEvent_t> pool;
};
TimingState& timing() {
  static TimingState* t = new TimingState();  // never destroyed: safe at exit
  return *t;
}
cudaEvent_t pool_get(TimingState& t) {
  if (!t.pool.empty()) {
    cudaEvent_t e = t.pool.back();
    t.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

int timing_begin(const char* name, cudaStream_t s) {
  TimingState& t = timing();
  if (!t.on.load(std::memory_order_relaxed) || timing_suspended()) return -1;
  std::lock_guard<std::mutex> g(t.mu);
  int kind = -1;
  for (size_t i = 0; i < t.kinds.size(); ++i)
    if (t.kinds[i] == name) kind = (int)i;
  if (kind < 0) {
    kind = (int)t.kinds.size();
    t.kinds.emplace_back(name);
    t.launches.push_back(0);
    t.ms.push_back(0.0);
  }
  TimingRec r{kind, pool_get(t), pool_get(t)};
  cudaEventRecord(r.a, s);
  t.pending.push_back(r);
  return (int)t.pending.size() - 1;
}

void timing_end(int token, cudaStream_t s) {
  if (token < 0) return;
  TimingState& t = timing();
  std::lock_guard<std::mutex> g(t.mu);
  if (token < (int)t.pending.size()) cudaEventRecord(t.pending[token].b, s);
}

}  // namespace mg

using namespace mg;

extern "C" {

mg_status mg_timing_enable(int on) {
  timing().on.store(on != 0);
  return MG_OK;
}

int mg_timing_read(mg_timing_entry* out, int max) {
  TimingState& t = timing();
  std::lock_guard<std::mutex> g(t.mu);
  bool ok = true;
  for (const TimingRec& r : t.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
      ok = false;
    t.ms[r.kind] += ms;
    t.launches[r.kind] += 1;
    t.pool.push_back(r.a);
    t.pool.push_back(r.b);
  }
  t.pending.clear();
  int n = 0;
  for (size_t i = 0; i < t.kinds.size() && n < max; ++i) {
    if (t.launches[i] == 0) continue;
    if (out) {
      std::snprintf(out[n].name, sizeof out[n].name, "%s", t.kinds[i].c_str());
      out[n].launches = t.launches[i];
      out[n].ms = t.ms[i];
    }
    ++n;
  }
  std::fill(t.launches.begin(), t.launches.end(), 0);
  std::fill(t.ms.begin(), t.ms.end(), 0.0);
  if (!ok) {
    fail(MG_ERR_CUDA, "mg_timing_read: event query failed");
    return -1;
  }
  return n;
}

mg_status mg_sync_status(void* stream) {
  int st = 0;
  const cudaError_t e = read_device_status(&st, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(MG_ERR_CUDA, "mg_sync_status: %s", cudaGetErrorString(e));
  if (st & 1)
    return fail(MG_ERR_TIMEOUT,
                "a smoother or operator pass gave up waiting for its staged input; its "
                "outputs are not valid");
  if (st & 2)
    return fail(MG_ERR_TIMEOUT,
                "a tensor-core Gram gave up waiting for its matrix multiplies; the "
                "truncation's outputs are not valid");
  return MG_OK;
}

mg_status mg_random_starts(const mg_problem* prob, void* psi0, void* stream) {
  Geom g;
  mg_status st = make_geom(prob, &g);
  if (st != MG_OK) return st;
  if (!psi0) return fail(MG_ERR_INVALID, "mg_random_starts: NULL array");
  return cuda_status(launch_random_starts(g, prob->seed, static_cast<float2*>(psi0),
                                          static_cast<cudaStream_t>(stream)),
                     "mg_random_starts");
}

mg_status mg_random_links(const mg_problem* prob, double eps, void* U, void* stream) {
  Geom g;
  mg_status st = make_geom(prob, &g);
  if (st != MG_OK) return st;
  if (!U) return fail(MG_ERR_INVALID, "mg_random_links: NULL array");
  if (!(eps >= 0.0 && eps <= 1.0))
    return fail(MG_ERR_INVALID, "mg_random_links: eps %g outside [0, 1]", eps);
  return cuda_status(launch_random_links(g, prob->seed, eps, static_cast<float2*>(U),
                                         static_cast<cudaStream_t>(stream)),
                     "mg_random_links");
}

mg_status mg_selftest_timeout(int32_t polls, void* stream) {
  if (polls < 1 || polls > (1 << 20))
    return fail(MG_ERR_INVALID, "mg_selftest_timeout: polls %d out of [1, 1048576]", polls);
  return cuda_status(launch_selftest_timeout(polls, static_cast<cudaStream_t>(stream)),
                     "mg_selftest_timeout");
}

const char* mg_last_error(void) { return g_err; }

const char* mg_version(void) { return "chiral-mg-gb300 0.1 (sm_103a)"; }

size_t mg_workspace_size(const mg_problem* prob, int which) {
  Geom g;
  if (make_geom(prob, &g) != MG_OK) return 0;
  switch (which) {
    case MG_CALL_SMOOTH: return smooth_ws_layout(g).bytes;
    case MG_CALL_TRUNCATE: return trunc_ws_layout(g).bytes;
    case MG_CALL_COARSEN: return 0;
    default: fail(MG_ERR_INVALID, "unknown call id %d", which); return 0;
  }
}

mg_status mg_clover_field(const mg_problem* prob, const void* U, void* C, void* stream) {
  Geom g;
  mg_status st = make_geom(prob, &g);
  if (st != MG_OK) return st;
  if (!U || !C) return fail(MG_ERR_INVALID, "mg_clover_field: NULL array");
  return cuda_status(launch_clover(g, prob->csw, static_cast<const float2*>(U),
                                   static_cast<float2*>(C), static_cast<cudaStream_t>(stream)),
                     "mg_clover_field");
}

mg_status mg_apply_dirac(const mg_problem* prob, const void* U, const void* C, const void* in,
                         void* out, void* ws, size_t ws_bytes, void* stream) {
  Geom g;
  mg_status st = make_geom(prob, &g);
  if (st != MG_OK) return st;
  if (!U || !in || !out || !ws) return fail(MG_ERR_INVALID, "mg_apply_dirac: NULL array");
  if (in == out) return fail(MG_ERR_INVALID, "mg_apply_dirac: out aliases in");
  const size_t need = smooth_ws_layout(g).bytes;
  if (ws_bytes < need)
    return fail(MG_ERR_INVALID, "mg_apply_dirac: workspace %zu < %zu bytes", ws_bytes, need);
  return cuda_status(launch_dirac(g, static_cast<const float2*>(U), static_cast<const float2*>(C),
                                  static_cast<const float2*>(in), static_cast<float2*>(out),
                                  static_cast<char*>(ws), static_cast<cudaStream_t>(stream)),
                     "mg_apply_dirac");
}

mg_status mg_smooth_testvecs(const mg_problem* prob, const void* U, const void* C,
                             const void* psi0, void* psi, void* ws, size_t ws_bytes,
                             void* stream) {
  Geom g;
  mg_status st = make_geom(prob, &g);
  if (st != MG_OK) return st;
  if (g.niter < 1) return fail(MG_ERR_INVALID, "mr_iters must be >= 1");
  if (!U || !psi0 || !psi || !ws) return fail(MG_ERR_INVALID, "mg_smooth_testvecs: NULL array");
  const size_t need = smooth_ws_layout(g).bytes;
  if (ws_bytes < need)
    return fail(MG_ERR_INVALID, "mg_smooth_testvecs: workspace %zu < %zu bytes", ws_bytes, need);
  return cuda_status(launch_smoother(g, static_cast<const float2*>(U),
                                     static_cast<const float2*>(C),
                                     static_cast<const float2*>(psi0), static_cast<float2*>(psi),
                                     static_cast<char*>(ws), static_cast<cudaStream_t>(stream)),
                     "mg_smooth_testvecs");
}

mg_status mg_chiral_truncate(const mg_problem* prob, const void* psi, void* Uk, double* sigma,
                             void* coarse_tv, int32_t* blk_flags, void* ws, size_t ws_bytes,
                             void* stream) {
  Geom g;
  mg_status st = make_geom(prob, &g);
  if (st != MG_OK) return st;
  if (!psi || !Uk || !sigma || !blk_flags || !ws)
    return fail(MG_ERR_INVALID, "mg_chiral_truncate: NULL array");
  const size_t need = trunc_ws_layout(g).bytes;
  if (ws_bytes < need)
    return fail(MG_ERR_INVALID, "mg_chiral_truncate: workspace %zu < %zu bytes", ws_bytes, need);
  return cuda_status(
      launch_truncate(g, static_cast<const float2*>(psi), static_cast<float2*>(Uk), sigma,
                      static_cast<float2*>(coarse_tv), blk_flags, static_cast<char*>(ws),
                      static_cast<cudaStream_t>(stream)),
      "mg_chiral_truncate");
}

mg_status mg_build_prolongator(const mg_problem* prob, const void* Uk, void* P, void* stream) {
  Geom g;
  mg_status st = make_geom(prob, &g);
  if (st != MG_OK) return st;
  if (!Uk || !P) return fail(MG_ERR_INVALID, "mg_build_prolongator: NULL array");
  return cuda_status(launch_prolongator(g, static_cast<const float2*>(Uk),
                                        static_cast<float2*>(P), static_cast<cudaStream_t>(stream)),
                     "mg_build_prolongator");
}

mg_status mg_coarsen(const mg_problem* prob, const void* U, const void* C, const void* P,
                     void* X, void* Y, void* ws, size_t ws_bytes, void* stream) {
  (void)ws;
  (void)ws_bytes;
  Geom g;
  mg_status st = make_geom(prob, &g);
  if (st != MG_OK) return st;
  if (!U || !P || !X || !Y) return fail(MG_ERR_INVALID, "mg_coarsen: NULL array");
  return cuda_status(launch_coarsen(g, static_cast<const float2*>(U),
                                    static_cast<const float2*>(C), static_cast<const float2*>(P),
                                    static_cast<float2*>(X), static_cast<float2*>(Y),
                                    static_cast<cudaStream_t>(stream)),
                     "mg_coarsen");
}

// shared memory the coarse apply may stage per coarse site: the launch limit
// that launch_coarse_apply (mg_coarsen.cu) sets for its kernel
constexpr size_t kCoarseApplyMaxStage = 200000;

mg_status mg_coarse_apply(const mg_problem* prob, const void* X, const void* Y,
                          const void* v_in, void* v_out, int32_t nrhs, void* stream) {
  Geom g;
  mg_status st = make_geom(prob, &g);
  if (st != MG_OK) return st;
  if (!X || !Y || !v_in || !v_out) return fail(MG_ERR_INVALID, "mg_coarse_apply: NULL array");
  if (nrhs < 1 || nrhs > 64) return fail(MG_ERR_INVALID, "nrhs = %d must be in [1, 64]", nrhs);
  if (v_in == v_out) return fail(MG_ERR_INVALID, "mg_coarse_apply: v_out aliases v_in");
  // the nine source vectors of a coarse site are staged in shared memory
  const size_t stage = sizeof(float2) * 9 * (size_t)(2 * g.k) * nrhs;
  if (stage > kCoarseApplyMaxStage)
    return fail(MG_ERR_UNSUPPORTED,
                "mg_coarse_apply: 9 x 2k x nrhs = %zu complex numbers exceed the %zu bytes of "
                "staging (nrhs <= %zu at k = %d)",
                stage / sizeof(float2), kCoarseApplyMaxStage,
                kCoarseApplyMaxStage / (sizeof(float2) * 9 * (size_t)(2 * g.k)), g.k);
  return cuda_status(launch_coarse_apply(g, static_cast<const float2*>(X),
                                         static_cast<const float2*>(Y),
                                         static_cast<const float2*>(v_in),
                                         static_cast<float2*>(v_out), nrhs,
                                         static_cast<cudaStream_t>(stream)),
                     "mg_coarse_apply");
}

// ---------------------------------------------------------------------------
// levels l >= 1
// ---------------------------------------------------------------------------
namespace {
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
}  // namespace

size_t mg_coarse_workspace_size(const mg_coarse_problem* prob, int which) {
  StencilGeom sg;
  Geom g;
  if (make_cgeom(prob, &sg, &g, true) != MG_OK) return 0;
  switch (which) {
    case MG_CALL_SMOOTH: return stencil_smooth_ws_layout(sg, g.m).bytes;
    case MG_CALL_TRUNCATE: return trunc_ws_layout(g).bytes;
    case MG_CALL_COARSEN: return 0;
    default: fail(MG_ERR_INVALID, "unknown call %d", which); return 0;
  }
}

mg_status mg_coarse_op_apply(const mg_coarse_problem* prob, const void* X, const void* Y,
                             const void* v_in, void* v_out, int32_t nrhs, void* stream) {
  StencilGeom sg;
  Geom g;
  mg_status st = make_cgeom(prob, &sg, &g, false);
  if (st != MG_OK) return st;
  if (!X || !Y || !v_in || !v_out) return fail(MG_ERR_INVALID, "mg_coarse_op_apply: NULL array");
  if (!aligned16(X) || !aligned16(Y) || !aligned16(v_in) || !aligned16(v_out))
    return fail(MG_ERR_INVALID, "mg_coarse_op_apply: arrays must be 16-byte aligned");
  if (nrhs < 1 || nrhs > 64) return fail(MG_ERR_INVALID, "nrhs = %d must be in [1, 64]", nrhs);
  if (v_in == v_out) return fail(MG_ERR_INVALID, "mg_coarse_op_apply: v_out aliases v_in");
  return cuda_status(launch_stencil_apply(sg, static_cast<const float2*>(X),
                                          static_cast<const float2*>(Y),
                                          static_cast<const float2*>(v_in),
                                          static_cast<float2*>(v_out), nrhs,
                                          static_cast<cudaStream_t>(stream)),
                     "mg_coarse_op_apply");
}

mg_status mg_coarse_smooth_testvecs(const mg_coarse_problem* prob, const void* X, const void* Y,
                                    const void* psi0, void* psi, void* ws, size_t ws_bytes,
                                    void* stream) {
  StencilGeom sg;
  Geom g;
  mg_status st = make_cgeom(prob, &sg, &g, true);
  if (st != MG_OK) return st;
  if (g.niter < 1) return fail(MG_ERR_INVALID, "mr_iters must be >= 1");
  if (!X || !Y || !psi0 || !psi || !ws)
    return fail(MG_ERR_INVALID, "mg_coarse_smooth_testvecs: NULL array");
  if (!aligned16(X) || !aligned16(Y) || !aligned16(psi0) || !aligned16(psi) || !aligned16(ws))
    return fail(MG_ERR_INVALID, "mg_coarse_smooth_testvecs: arrays must be 16-byte aligned");
  const size_t need = stencil_smooth_ws_layout(sg, g.m).bytes;
  if (ws_bytes < need)
    return fail(MG_ERR_INVALID, "mg_coarse_smooth_testvecs: workspace %zu < %zu bytes", ws_bytes,
                need);
  return cuda_status(launch_stencil_smoother(sg, g.m, g.niter, static_cast<const float2*>(X),
                                             static_cast<const float2*>(Y),
                                             static_cast<const float2*>(psi0),
                                             static_cast<float2*>(psi), static_cast<char*>(ws),
                                             static_cast<cudaStream_t>(stream)),
                     "mg_coarse_smooth_testvecs");
}

mg_status mg_coarse_chiral_truncate(const mg_coarse_problem* prob, const void* psi, void* Uk,
                                    double* sigma, void* coarse_tv, int32_t* blk_flags, void* ws,
                                    size_t ws_bytes, void* stream) {
  StencilGeom sg;
  Geom g;
  mg_status st = make_cgeom(prob, &sg, &g, true);
  if (st != MG_OK) return st;
  if (!psi || !Uk || !sigma || !blk_flags || !ws)
    return fail(MG_ERR_INVALID, "mg_coarse_chiral_truncate: NULL array");
  if (!aligned16(psi)) return fail(MG_ERR_INVALID, "mg_coarse_chiral_truncate: psi not 16-byte aligned");
  const size_t need = trunc_ws_layout(g).bytes;
  if (ws_bytes < need)
    return fail(MG_ERR_INVALID, "mg_coarse_chiral_truncate: workspace %zu < %zu bytes", ws_bytes,
                need);
  return cuda_status(
      launch_truncate(g, static_cast<const float2*>(psi), static_cast<float2*>(Uk), sigma,
                      static_cast<float2*>(coarse_tv), blk_flags, static_cast<char*>(ws),
                      static_cast<cudaStream_t>(stream)),
      "mg_coarse_chiral_truncate");
}

mg_status mg_coarse_build_prolongator(const mg_coarse_problem* prob, const void* Uk, void* P,
                                      void* stream) {
  StencilGeom sg;
  Geom g;
  mg_status st = make_cgeom(prob, &sg, &g, true);
  if (st != MG_OK) return st;
  if (!Uk || !P) return fail(MG_ERR_INVALID, "mg_coarse_build_prolongator: NULL array");
  return cuda_status(launch_prolongator(g, static_cast<const float2*>(Uk),
                                        static_cast<float2*>(P), static_cast<cudaStream_t>(stream)),
                     "mg_coarse_build_prolongator");
}

mg_status mg_coarse_coarsen(const mg_coarse_problem* prob, const void* X, const void* Y,
                            const void* P, void* X2, void* Y2, void* stream) {
  StencilGeom sg;
  Geom g;
  mg_status st = make_cgeom(prob, &sg, &g, true);
  if (st != MG_OK) return st;
  if (!X || !Y || !P || !X2 || !Y2) return fail(MG_ERR_INVALID, "mg_coarse_coarsen: NULL array");
  if (!aligned16(X) || !aligned16(Y))
    return fail(MG_ERR_INVALID, "mg_coarse_coarsen: X and Y must be 16-byte aligned");
  return cuda_status(launch_stencil_galerkin(g, static_cast<const float2*>(X),
                                             static_cast<const float2*>(Y),
                                             static_cast<const float2*>(P),
                                             static_cast<float2*>(X2), static_cast<float2*>(Y2),
                                             static_cast<cudaStream_t>(stream)),
                     "mg_coarse_coarsen");
}

}  // extern "C"
