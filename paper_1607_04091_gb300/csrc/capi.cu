// extern "C" entry points of libgs (declared in include/gs.h): validation,
// plan lifetime, applies in the caller's sample order, error reporting.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cstring>

#include <atomic>

#include "gs_internal.h"

namespace gs {

static thread_local char g_detail[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
  va_end(ap);
}

gs_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return GS_ECUDA;
}

// ---------------------------------------------------------------- tracing
namespace {
struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
};
struct Profiler {
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  std::mutex mu;
};
Profiler& profiler() {
  static Profiler p;
  return p;
}
cudaEvent_t take_event(Profiler& p) {
  if (!p.pool.empty()) {
    cudaEvent_t e = p.pool.back();
    p.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

bool prof_on() { return profiler().on; }

void prof_begin(const char* name, cudaStream_t st) {
  Profiler& p = profiler();
  std::lock_guard<std::mutex> g(p.mu);
  ProfRec r{name, take_event(p), take_event(p)};
  cudaEventRecord(r.a, st);
  p.recs.push_back(r);
}

void prof_end(cudaStream_t st) {
  Profiler& p = profiler();
  std::lock_guard<std::mutex> g(p.mu);
  if (!p.recs.empty()) cudaEventRecord(p.recs.back().b, st);
}

template <typename R>
static void free_graphs(PrecData<R>& D) {
  for (int i = 0; i < 2; ++i)
    if (D.cg_exec[i]) cudaGraphExecDestroy(D.cg_exec[i]);
}

static void free_prec_f(PrecData<float>& D) {
  void* ps[] = {D.frac, D.win, D.w, D.bf, D.deap, D.tw, D.grid, D.hbuf, D.ftmp, D.side, D.part, D.corner, D.hs, D.hp, D.lat,
                D.vx, D.vs, D.vp, D.vr, D.vq, D.vz};
  for (void* p : ps)
    if (p) cudaFree(p);
}
static void free_prec_d(PrecData<double>& D) {
  void* ps[] = {D.frac, D.win, D.w, D.bf, D.deap, D.tw, D.grid, D.hbuf, D.ftmp, D.side, D.part, D.corner, D.hs, D.hp, D.lat,
                D.vx, D.vs, D.vp, D.vr, D.vq, D.vz};
  for (void* p : ps)
    if (p) cudaFree(p);
}

static void free_plan(Plan* P) {
  void* ps[] = {P->perm, P->fl, P->xi_sorted, P->bin_start, P->work, P->work_start, P->work_order, P->wcol, P->wcol_start,
                P->red, P->scal, P->flag, P->y64, P->r64, P->x64};
  for (void* p : ps)
    if (p) cudaFree(p);
  free_graphs(P->d);
  free_graphs(P->f);
  for (int i = 0; i < 2; ++i)
    if (P->solve_exec[i]) cudaGraphExecDestroy(P->solve_exec[i]);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  for (int i = 0; i < 3; ++i) {
    if (P->aux[i]) cudaStreamDestroy(P->aux[i]);
    if (P->ev_fork[i]) cudaEventDestroy(P->ev_fork[i]);
    if (P->ev_join[i]) cudaEventDestroy(P->ev_join[i]);
  }
  free_prec_d(P->d);
  free_prec_f(P->f);
}

// Work-item size by measurement: for each candidate size the work items are
// rebuilt and float32 T and T^H (sorted sample order, as inside the solver) are
// timed back to back; the fastest size stays.  The applies of the chosen plan
// differ from those of a fixed-size plan only in how the partial sums group.
static gs_status autotune_chunk(Plan* P, cudaStream_t st) {
  static const int cand[] = {128, 192, 256, 384, 512, 768, 1024};
  C<float>* x = P->f.vp;
  C<float>* y = P->f.vq;
  GS_CUDA(cudaMemsetAsync(x, 0, P->ncoef * sizeof(C<float>), st));
  GS_CUDA(cudaMemsetAsync(y, 0, P->M * sizeof(C<float>), st));
  cudaEvent_t e0, e1;
  GS_CUDA(cudaEventCreate(&e0));
  GS_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 0.0f;
  gs_status s = GS_OK;
  for (int c : cand) {
    s = set_work(P, c, st);
    if (s != GS_OK) break;
    float ms = 0.0f;
    for (int rep = 0; rep < 2 && s == GS_OK; ++rep) {  // rep 0 warms up
      if (rep == 1 && cudaEventRecord(e0, st) != cudaSuccess) s = GS_ECUDA;
      for (int k = 0; k < (rep ? 3 : 1) && s == GS_OK; ++k) {
        s = apply_T<float>(P, P->f, x, y, nullptr, st);
        if (s == GS_OK) s = apply_TH<float>(P, P->f, y, x, nullptr, st);
      }
    }
    if (s != GS_OK) break;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      s = cuda_fail(cudaGetLastError(), "autotune timing");
      break;
    }
    if (best == 0 || ms < best_ms) {
      best = c;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != GS_OK) return s;
  return set_work(P, best, st);
}

static gs_status make_plan(gs_plan* out, int dims, const double* xi, int64_t M, int p, int J,
                           double bandwidth, const double* weights, const gs_opts* opts, void* stream) {
  if (!out) {
    set_error("out is NULL");
    return GS_EINVAL;
  }
  *out = nullptr;
  if (!xi || M < 1 || M > ((int64_t)1 << 31) - 1) {
    set_error("need xi != NULL and 1 <= M < 2^31 (M = %lld)", (long long)M);
    return GS_EINVAL;
  }
  if (p < 1 || p > GS_MAX_P) {
    set_error("p = %d outside 1..%d", p, GS_MAX_P);
    return GS_EINVAL;
  }
  if (J < 1 || J > 20 || (dims == 2 && J > 13) || (1LL << J) < 2LL * p) {
    set_error("J = %d invalid for p = %d (need 2^J >= 2p, J <= 20 in 1D, <= 13 in 2D)", J, p);
    return GS_EINVAL;
  }
  for (int64_t i = 0; i < M * dims; ++i)
    if (!std::isfinite(xi[i])) {
      set_error("xi[%lld] is not finite", (long long)i);
      return GS_EINVAL;
    }
  if (weights)
    for (int64_t i = 0; i < M; ++i)
      if (!std::isfinite(weights[i]) || weights[i] < 0.0) {
        set_error("weights[%lld] is negative or not finite", (long long)i);
        return GS_EINVAL;
      }
  gs_opts o = {8, 4, 2, -1, 0, 0};
  if (opts) o = *opts;
  if (o.kb_m_hi < 2 || o.kb_m_hi > 8 || o.kb_m_lo < 2 || o.kb_m_lo > 8 || (o.sigma != 2 && o.sigma != 4) ||
      o.chunk < -1 || o.chunk > (1 << 20) || o.lattice < 0 || o.lattice > 2) {
    set_error("bad options: kb_m_hi = %d, kb_m_lo = %d (2..8), sigma = %d (2 or 4), chunk = %d (-1..2^20), "
              "lattice = %d (0..2)", o.kb_m_hi, o.kb_m_lo, o.sigma, o.chunk, o.lattice);
    return GS_EINVAL;
  }
  gs_plan_s* h = new (std::nothrow) gs_plan_s();
  if (!h) {
    set_error("host allocation failed");
    return GS_ENOMEM;
  }
  Plan* P = &h->P;
  P->dims = dims;
  P->p = p;
  P->J = J;
  P->b = (p == 1) ? 0 : p;
  P->M = M;
  P->N = (int64_t)1 << J;
  P->ncoef = (dims == 1) ? P->N : P->N * P->N;
  P->sigma = o.sigma;
  P->n = P->N * o.sigma;
  P->m_hi = o.kb_m_hi;
  P->m_lo = o.kb_m_lo;
  P->bandwidth = bandwidth;
  P->chunk = o.chunk > 0 ? o.chunk : 0;
  if (dims == 2 && ((o.kb_m_hi != 4 && o.kb_m_hi != 6 && o.kb_m_hi != 8) ||
                    (o.kb_m_lo != 4 && o.kb_m_lo != 6 && o.kb_m_lo != 8))) {
    set_error("2D plans take Kaiser-Bessel half-widths 4, 6 or 8 (kb_m_hi = %d, kb_m_lo = %d)", o.kb_m_hi, o.kb_m_lo);
    delete h;
    return GS_EINVAL;
  }
  int mmax = o.kb_m_hi > o.kb_m_lo ? o.kb_m_hi : o.kb_m_lo;
  const int tile = (dims == 1) ? TILE1 : TILE2;
  const int64_t eff_tile = P->n < tile ? P->n : tile;
  bool nfft_ok = (eff_tile >= mmax) && (P->n >= 2 * mmax);
  if (dims == 1 && P->n > (1 << 20)) nfft_ok = false;  // four-step FFT: n1, n2 <= 1024
  if (dims == 2 && P->n > 1024) nfft_ok = false;  // float64 column-pass tiles in shared memory
  if (o.direct == 1) P->direct = 1;
  else if (o.direct == 0) {
    if (!nfft_ok) {
      set_error("NFFT path needs n = sigma 2^J >= 2 m, a tile >= m and n <= %d", dims == 1 ? (1 << 20) : 1024);
      delete h;
      return GS_EUNSUPPORTED;
    }
    P->direct = 0;
  } else {
    // direct evaluation (one thread per sample or coefficient, a sincos per entry)
    // only for tiny problems; the NFFT path is faster from ~2^16 entries
    P->direct = (!nfft_ok || (double)M * (double)P->ncoef <= 65536.0) ? 1 : 0;
  }
  if (!P->direct && o.lattice != 1) {
    // Sec. 3.2: samples on the lattice (1/sigma) Z^d (exactly, in double) make the
    // NDFT an FFT; sigma is a power of two, so sigma xi is exact
    bool on = true;
    for (int64_t i = 0; i < M * dims && on; ++i) {
      const double v = xi[i] * (double)o.sigma;
      on = (v == std::rint(v));
    }
    P->lattice = on ? 1 : 0;
  }
  if (o.lattice == 2 && !P->lattice) {
    set_error("lattice = 2: the samples are not all on the lattice (1/sigma) Z^d of an NFFT-path plan");
    delete h;
    return GS_EINVAL;
  }
  if (!build_constants(p, &P->k)) {
    set_error("boundary construction failed for p = %d", p);
    delete h;
    return GS_EUNSUPPORTED;
  }
  static std::atomic<uint64_t> next_uid{1};
  P->uid = next_uid.fetch_add(1);
  GS_CUDA(cudaGetDevice(&P->dev));
  GS_CUDA(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
  for (int i = 0; i < 3; ++i) {
    GS_CUDA(cudaStreamCreateWithFlags(&P->aux[i], cudaStreamNonBlocking));
    GS_CUDA(cudaEventCreateWithFlags(&P->ev_fork[i], cudaEventDisableTiming));
    GS_CUDA(cudaEventCreateWithFlags(&P->ev_join[i], cudaEventDisableTiming));
  }
  gs_status s = build_plan(P, xi, weights, (cudaStream_t)stream);
  if (s == GS_OK && o.chunk == -1 && !P->direct) s = autotune_chunk(P, (cudaStream_t)stream);
  if (s != GS_OK) {
    free_plan(P);
    delete h;
    return s;
  }
  *out = h;
  return GS_OK;
}

gs_status take_device_timeout(Plan* P) {
  int v = 0;
  GS_CUDA(cudaMemcpy(&v, P->flag + FL_TIMEOUT, sizeof(int), cudaMemcpyDeviceToHost));
  if (v == 0) return GS_OK;
  GS_CUDA(cudaMemset(P->flag + FL_TIMEOUT, 0, sizeof(int)));
  set_error("a bounded device wait gave up (a tensor-core kernel of this plan skipped its output)");
  return GS_ETIMEOUT;
}

}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_plan_1d(gs_plan* out, const double* xi, int64_t M, int p, int J, double bandwidth,
                     const double* weights, const gs_opts* opts, void* stream) {
  return make_plan(out, 1, xi, M, p, J, bandwidth, weights, opts, stream);
}

gs_status gs_plan_2d(gs_plan* out, const double* xi, int64_t M, int p, int J, const double* weights,
                     const gs_opts* opts, void* stream) {
  return make_plan(out, 2, xi, M, p, J, 0.0, weights, opts, stream);
}

void gs_plan_destroy(gs_plan plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  free_plan(&plan->P);
  delete plan;
}

gs_status gs_plan_sizes(gs_plan plan, int* dims, int64_t* M, int64_t* N, int64_t* ncoef) {
  if (!plan) {
    set_error("plan is NULL");
    return GS_EINVAL;
  }
  if (dims) *dims = plan->P.dims;
  if (M) *M = plan->P.M;
  if (N) *N = plan->P.N;
  if (ncoef) *ncoef = plan->P.ncoef;
  return GS_OK;
}

gs_status gs_apply_T(gs_plan plan, int precision, const void* x, void* y, void* stream) {
  if (!plan || !x || !y) {
    set_error("plan, x and y must be non-NULL");
    return GS_EINVAL;
  }
  Plan* P = &plan->P;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == GS_FP64)
    return apply_T<double>(P, P->d, (const double2*)x, (double2*)y, P->perm, st);
  if (precision == GS_FP32)
    return apply_T<float>(P, P->f, (const float2*)x, (float2*)y, P->perm, st);
  set_error("unknown precision %d", precision);
  return GS_EINVAL;
}

gs_status gs_apply_TH(gs_plan plan, int precision, const void* y, void* x, void* stream) {
  if (!plan || !x || !y) {
    set_error("plan, x and y must be non-NULL");
    return GS_EINVAL;
  }
  Plan* P = &plan->P;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == GS_FP64)
    return apply_TH<double>(P, P->d, (const double2*)y, (double2*)x, P->perm, st);
  if (precision == GS_FP32)
    return apply_TH<float>(P, P->f, (const float2*)y, (float2*)x, P->perm, st);
  set_error("unknown precision %d", precision);
  return GS_EINVAL;
}

gs_status gs_solve(gs_plan plan, const void* y, void* x, const gs_solve_opts* opts, gs_solve_info* info,
                   void* stream) {
  if (!plan || !x || !y) {
    set_error("plan, x and y must be non-NULL");
    return GS_EINVAL;
  }
  gs_solve_opts o = {1e-6, 1000, GS_SOLVE_MIXED, 0, 8, 0.0};
  if (opts) o = *opts;
  // default: each float32 pass gains three orders before the float64 residual is
  // re-formed; the restart keeps float32 drift out of long passes (ill-conditioned
  // problems) and costs few iterations on well-conditioned ones
  if (o.inner_rtol == 0.0) o.inner_rtol = 1e-3;
  if (!(o.tol > 0.0) || o.maxit < 1 || (o.mode != GS_SOLVE_FP64 && o.mode != GS_SOLVE_MIXED) || o.max_outer < 1 ||
      !(o.inner_rtol > 0.0 && o.inner_rtol < 1.0)) {
    set_error("bad solve options (tol > 0, maxit >= 1, mode 0/1, max_outer >= 1, 0 < inner_rtol < 1)");
    return GS_EINVAL;
  }
  if (plan->P.M <= plan->P.ncoef) {
    // Sec. 2: the least-squares reconstruction needs more samples than coefficients
    set_error("gs_solve: M = %lld samples must exceed the %lld coefficients (stable sampling, Sec. 2)",
              (long long)plan->P.M, (long long)plan->P.ncoef);
    return GS_EINVAL;
  }
  gs_status r = solve(&plan->P, (const double*)y, (double*)x, o, info, (cudaStream_t)stream);
  const gs_status t = take_device_timeout(&plan->P);
  if (t != GS_OK) {
    if (info) info->status = t;
    return t;
  }
  return r;
}

gs_status gs_boundary_constants(int p, double* h, double* UL, double* VL, double* v0L, double* UR, double* VR,
                                double* v0R) {
  if (p < 1 || p > GS_MAX_P) {
    set_error("p = %d outside 1..%d", p, GS_MAX_P);
    return GS_EINVAL;
  }
  Constants c;
  if (!build_constants(p, &c)) {
    set_error("boundary construction failed for p = %d", p);
    return GS_EUNSUPPORTED;
  }
  if (h)
    for (int j = 0; j < 2 * p; ++j) h[j] = c.h[j];
  if (p == 1) return GS_OK;
  const EdgeConst* sides[2] = {&c.left, &c.right};
  double* Us[2] = {UL, UR};
  double* Vs[2] = {VL, VR};
  double* v0s[2] = {v0L, v0R};
  for (int q = 0; q < 2; ++q) {
    for (int i = 0; i < p; ++i) {
      if (Us[q])
        for (int j = 0; j < p; ++j) Us[q][i * p + j] = sides[q]->U[i][j];
      if (Vs[q])
        for (int j = 0; j < 2 * p - 1; ++j) Vs[q][i * (2 * p - 1) + j] = sides[q]->V[i][j];
      if (v0s[q]) v0s[q][i] = sides[q]->v10[i];
    }
  }
  return GS_OK;
}

gs_status gs_profile(int on) {
  Profiler& p = profiler();
  std::lock_guard<std::mutex> g(p.mu);
  p.on = (on != 0);
  return GS_OK;
}

gs_status gs_profile_report(char* buf, int64_t len) {
  if (!buf || len < 3) {
    set_error("buffer too small");
    return GS_EINVAL;
  }
  Profiler& p = profiler();
  std::lock_guard<std::mutex> g(p.mu);
  std::map<std::string, std::pair<long, double>> agg;
  for (ProfRec& r : p.recs) {
    float ms = 0.0f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    auto& v = agg[r.name];
    v.first += 1;
    v.second += ms;
    p.pool.push_back(r.a);
    p.pool.push_back(r.b);
  }
  p.recs.clear();
  std::string out = "{";
  bool first = true;
  for (auto& kv : agg) {
    char tmp[256];
    snprintf(tmp, sizeof(tmp), "%s\"%s\": [%ld, %.6f]", first ? "" : ", ", kv.first.c_str(), kv.second.first,
             kv.second.second);
    out += tmp;
    first = false;
  }
  out += "}";
  if ((int64_t)out.size() + 1 > len) {
    set_error("report needs %zu bytes", out.size() + 1);
    return GS_EINVAL;
  }
  memcpy(buf, out.c_str(), out.size() + 1);
  return GS_OK;
}

gs_status gs_solve_batch(const gs_plan* plans, int B, const void* const* y, void* const* x,
                         const gs_solve_opts* opts, gs_solve_info* infos, void* stream) {
  if (!plans || !y || !x || B < 1) {
    set_error("need plans, y, x non-NULL and B >= 1");
    return GS_EINVAL;
  }
  gs_solve_opts o = {1e-6, 1000, GS_SOLVE_MIXED, 0, 8, 0.0};
  if (opts) o = *opts;
  // default: each float32 pass gains three orders before the float64 residual is
  // re-formed; the restart keeps float32 drift out of long passes (ill-conditioned
  // problems) and costs few iterations on well-conditioned ones
  if (o.inner_rtol == 0.0) o.inner_rtol = 1e-3;
  if (!(o.tol > 0.0) || o.maxit < 1 || (o.mode != GS_SOLVE_FP64 && o.mode != GS_SOLVE_MIXED) || o.max_outer < 1 ||
      !(o.inner_rtol > 0.0 && o.inner_rtol < 1.0)) {
    set_error("bad solve options (tol > 0, maxit >= 1, mode 0/1, max_outer >= 1, 0 < inner_rtol < 1)");
    return GS_EINVAL;
  }
  std::vector<Plan*> ps(B);
  std::vector<const double*> ys(B);
  std::vector<double*> xs(B);
  for (int i = 0; i < B; ++i) {
    if (!plans[i] || !y[i] || !x[i]) {
      set_error("plans[%d], y[%d] and x[%d] must be non-NULL", i, i, i);
      return GS_EINVAL;
    }
    ps[i] = &plans[i]->P;
    if (ps[i]->M <= ps[i]->ncoef) {
      set_error("plans[%d]: M = %lld samples must exceed the %lld coefficients (stable sampling, Sec. 2)", i,
                (long long)ps[i]->M, (long long)ps[i]->ncoef);
      return GS_EINVAL;
    }
    ys[i] = (const double*)y[i];
    xs[i] = (double*)x[i];
  }
  std::vector<Plan*> sorted = ps;
  std::sort(sorted.begin(), sorted.end());
  if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
    set_error("a plan appears twice in the batch (its workspaces would be shared)");
    return GS_EINVAL;
  }
  gs_status r = solve_batch(ps.data(), B, ys.data(), xs.data(), o, infos, (cudaStream_t)stream);
  for (int i = 0; i < B; ++i) {
    const gs_status t = take_device_timeout(ps[i]);
    if (t != GS_OK) {
      if (infos) infos[i].status = t;
      r = t;
    }
  }
  return r;
}

const char* gs_strerror(gs_status s) {
  switch (s) {
    case GS_OK: return "success";
    case GS_EINVAL: return "invalid argument";
    case GS_ENOMEM: return "out of memory";
    case GS_ECUDA: return "CUDA error";
    case GS_ENOTCONV: return "not converged";
    case GS_EBREAKDOWN: return "CGLS breakdown";
    case GS_ETIMEOUT: return "device wait timed out";
    case GS_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* gs_last_error_detail(void) { return g_detail; }

}  // extern "C"
