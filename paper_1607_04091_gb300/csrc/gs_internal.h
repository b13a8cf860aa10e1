// Internal declarations of libgs: plan layout, complex helpers, error handling.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gs.h"

#define GS_MAX_P 6
#define GS_MAX_B (2 * GS_MAX_P)  // boundary columns per dimension (left + right)

namespace gs {

// ------------------------------------------------------------------ host constants
struct EdgeConst {
  int p;
  double U[GS_MAX_P][GS_MAX_P];           // H / sqrt2 (App. A.1)
  double V[GS_MAX_P][2 * GS_MAX_P - 1];   // h / sqrt2, columns m = p..3p-2
  double v10[GS_MAX_P];                   // v1(0) = (I - U)^-1 V 1
  double nest_residual;
};

struct Constants {
  int p;
  double h[2 * GS_MAX_P];  // taps k = -p+1..p at index k + p - 1, sum = 1
  double mu1, mu2;         // int x phi, int x^2 phi
  EdgeConst left, right;
};

bool daubechies_taps(int p, double* h);
bool build_constants(int p, Constants* c);

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
gs_status cuda_fail(cudaError_t e, const char* what);
#define GS_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return gs::cuda_fail(e_, #call); \
  } while (0)
// return a failed status to the caller
#define GS_TRY(x)               \
  do {                          \
    gs_status s_ = (x);         \
    if (s_ != GS_OK) return s_; \
  } while (0)

// ------------------------------------------------------------------ tracing
// When enabled (gs_profile), every wrapped launch records a CUDA event pair on
// its stream; gs_profile_report aggregates them per kernel name.
void prof_begin(const char* name, cudaStream_t st);
void prof_end(cudaStream_t st);
bool prof_on();
#define GS_LAUNCH(name, st, ...)            \
  do {                                      \
    const bool p_ = gs::prof_on();          \
    if (p_) gs::prof_begin((name), (st));   \
    __VA_ARGS__;                            \
    if (p_) gs::prof_end((st));             \
  } while (0)
template <typename R> constexpr const char* pname(const char* f32, const char* f64) {
  return sizeof(R) == 4 ? f32 : f64;
}

// ------------------------------------------------------------------ complex
template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };
template <typename R> using C = typename Cx<R>::T;

// ------------------------------------------------------------------ plan
constexpr int TILE2 = 16;   // 2D spread tile edge (grid points); >= every KB half-width
constexpr int TILE1 = 128;  // 1D spread tile length
constexpr double WIN64_BYTES = 4.0 * (1 << 30);  // largest float64 window table of a plan
constexpr int CHUNK2 = 512; // samples per 2D spread work item (load balance)
constexpr int CHUNK1 = 512;

// Per-precision device tables and workspaces (R = double or float).
template <typename R>
struct PrecData {
  int m = 0;            // KB half-width (taps per dim 2m)
  double beta = 0;      // KB shape pi (2 - 1/sigma)
  // per-sample tables, sorted order
  R* frac = nullptr;    // [dims][M] fractional grid coordinate in [0, 1)
  R* win = nullptr;     // [M][dims][2m] window values phi(frac + m - 1 - a); float64: may be absent
  C<R>* w = nullptr;    // [dims][M] interior factor (x factor carries sqrt(mu))
  C<R>* bf = nullptr;   // [dims][M][2b] boundary factors: left k=0..b-1 then right k=0..b-1
  R* deap = nullptr;    // [N] 1/psi(k_i) per coefficient index i (interior only)
  C<R>* tw = nullptr;   // [n/2] exp(-2 pi i k / n)
  // workspaces
  C<R>* grid = nullptr;   // n^dims (2D: [lx][ly])
  C<R>* hbuf = nullptr;   // 2D: N x n, row j of the x transform ([j][lx])
  C<R>* ftmp = nullptr;   // 1D, n >= 4096: n, the four-step FFT's intermediate
  C<R>* side = nullptr;   // 2D: [2][2b][n]  (0: x-sides along y, 1: y-sides along x)
  C<R>* part = nullptr;   // spread partials, per work item
  C<R>* corner = nullptr; // 2D: (2b)^2 corner adjoint, 1D: 2b boundary adjoint
  C<R>* hs = nullptr;     // 2D float32: N x n, x transforms of the rows of s (CGNR)
  C<R>* hp = nullptr;     // 2D float32: N x n, x transforms of the rows of p (CGNR)
  C<R>* lat = nullptr;    // 2D lattice plans: per-bin side-line partials [bin][2][2b][tile]
  int64_t part_stride = 0;
  // solver vectors (sorted order for M-vectors)
  C<R>* vx = nullptr;  // ncoef
  C<R>* vs = nullptr;  // ncoef
  C<R>* vp = nullptr;  // ncoef
  C<R>* vr = nullptr;  // M
  C<R>* vq = nullptr;  // M
  C<R>* vz = nullptr;  // ncoef (T^H q in the normal-equation recursion)
  // captured CG pass (while-conditional graph), [0] CGLS form, [1] CGNR form
  cudaGraphExec_t cg_exec[2] = {nullptr, nullptr};
  bool cg_failed[2] = {false, false};
};

struct Plan {
  int dims = 1, p = 1, J = 0, b = 0, sigma = 2, direct = 0;
  int lattice = 0;  // 1: every sigma xi is an integer: exact pick / fold instead of KB windows
  int m_hi = 8, m_lo = 4;
  double bandwidth = 0.0;
  int64_t M = 0, N = 0, n = 0, ncoef = 0;
  Constants k;
  int dev = 0;
  // binning (sorted order)
  int32_t* perm = nullptr;   // perm[s] = caller index of sorted sample s
  int32_t* fl = nullptr;     // [dims][M] floor of the grid coordinate (mod n)
  double* xi_sorted = nullptr; // [dims][M] frequencies (direct mode, tables)
  int nbx = 0, nby = 0, nbins = 0, tile = 0;
  int32_t* bin_start = nullptr;  // [nbins + 1] sample range of each bin
  int32_t* work = nullptr;       // [nwork][3] (bin, s0, s1)
  int32_t* work_start = nullptr; // [nbins + 1] work items of each bin
  int32_t* work_order = nullptr; // [nwork] item indices, most samples first (launch order)
  int32_t* wcol = nullptr;       // work items grouped by bin column (bx), then row
  int32_t* wcol_start = nullptr; // [nbx + 1] offsets into wcol
  int nwork = 0;
  int chunk = 0;                 // samples per work item at most (near-equal split of a bin)
  int work_cap = 0;              // work items the partial-sum buffers hold
  std::vector<int32_t> bin_start_h;  // host copy of bin_start (work lists are rebuilt from it)
  PrecData<double> d;
  PrecData<float> f;
  // FP64 scratch for reductions and solver scalars
  double* red = nullptr;    // partial sums (>= 4096)
  double* scal = nullptr;   // solver scalars
  int* flag = nullptr;      // solver stop flag
  double* y64 = nullptr;    // M, sorted-order data (complex128)
  double* r64 = nullptr;    // M, FP64 residual (complex128)
  double* x64 = nullptr;    // ncoef complex128 accumulator
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
  // side branches of an apply or CG step: 0, 1 the partial reductions of the 2D
  // adjoint, 2 the step length of CG (see fork_aux / join_aux)
  cudaStream_t aux[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork[3] = {nullptr, nullptr, nullptr}, ev_join[3] = {nullptr, nullptr, nullptr};
  cudaGraphExec_t solve_exec[2] = {nullptr, nullptr};  // whole mixed solve as one graph [zero, given start]
  bool solve_graph_failed = false;
  bool solve_kernels_warm = false;  // the solve's kernels ran once outside any capture
  uint64_t uid = 0;                 // unique per plan in the process (batch-graph cache key)
  int last_iters = 0;               // CG iterations of the last graph solve (batch schedule cost)
  // the 2D spread and the partial-tile reductions launch as programmatic dependents
  // of the kernel before them, so that their CTAs' set-up overlaps its end; off for
  // a plan once it is solved in a batch (see solve_batch)
  bool pdl = true;
};

// Work launched on side_stream(P, st, i) between fork_aux(P, st, i) and
// join_aux(P, st, i) runs after everything enqueued on st before the fork and
// before everything enqueued on st after the join, concurrently with st in
// between; inside a stream capture the two become parallel branches of the
// graph.  With tracing on, the branch is st itself, so that each launch's event
// pair times that kernel alone.
inline cudaStream_t side_stream(Plan* P, cudaStream_t st, int i) { return prof_on() ? st : P->aux[i]; }
inline gs_status fork_aux(Plan* P, cudaStream_t st, int i) {
  if (prof_on()) return GS_OK;
  GS_CUDA(cudaEventRecord(P->ev_fork[i], st));
  GS_CUDA(cudaStreamWaitEvent(P->aux[i], P->ev_fork[i], 0));
  return GS_OK;
}
inline gs_status join_aux(Plan* P, cudaStream_t st, int i) {
  if (prof_on()) return GS_OK;
  GS_CUDA(cudaEventRecord(P->ev_join[i], P->aux[i]));
  GS_CUDA(cudaStreamWaitEvent(st, P->ev_join[i], 0));
  return GS_OK;
}

// implemented in tables.cu
gs_status build_plan(Plan* P, const double* xi, const double* mu_host, cudaStream_t st);
// (re)build the work items of every bin with at most `chunk` samples each, and
// grow the partial-sum buffers to hold them
gs_status set_work(Plan* P, int chunk, cudaStream_t st);
// implemented in nfft.cu / direct.cu.  perm != NULL: samples in the caller's
// order (y[perm[s]]); perm == NULL: samples in the plan's sorted order.
// norm_part != NULL (2D plans only): the interpolation also writes, per work
// item i, the sum of |y_s|^2 over its samples to norm_part[i] (nwork values).
template <typename R> struct PComb;
template <typename R>
gs_status nfft_T(Plan* P, PrecData<R>& D, const C<R>* x, C<R>* y, const int32_t* perm, cudaStream_t st,
                 double* norm_part = nullptr, const PComb<R>* pc = nullptr, bool df = false);
// out = x transforms of the coefficient rows of v (N x n), the first pass of T
template <typename R>
gs_status row_transform(Plan* P, PrecData<R>& D, const C<R>* v, C<R>* out, cudaStream_t st);
// Solver scalars (float64 slots of Plan::scal) and stop flags (Plan::flag[0]);
// Plan::flag[FL_ARRIVE] counts the CTAs of a fused CG step that have finished.
enum { S_GAMMA = 0, S_DELTA, S_ALPHA, S_BETA, S_GNEW, S_THR2, S_S0, S_ITER, S_MAXIT, S_TMP, S_LOOP };
enum { F_RUN = 0, F_CONV = 1, F_BREAK = 2, F_MAXIT = 3 };
constexpr int FL_ARRIVE = 4;
// Plan::flag[FL_TIMEOUT] != 0: a bounded device wait of a kernel gave up (the
// kernel skipped its output); gs_solve reports it as GS_ETIMEOUT and clears it.
constexpr int FL_TIMEOUT = 8;
// GS_OK, or GS_ETIMEOUT (flag cleared) when a kernel of the plan recorded a
// timed-out wait; synchronises with the device
gs_status take_device_timeout(Plan* P);

// The vector update of a CG step fused into the adjoint's last pass (2D plans):
// after z = T^H q, x += alpha p and s -= alpha z over all coefficients, with the
// per-CTA partial sums of the new ||s||^2 in part (one per coefficient row, N
// values); skipped while flag[0] != 0.  join_branch >= 0: side branch to join
// before that pass (where alpha is computed).
// With scal != NULL the last CTA to finish also closes the step: it sums the
// partials in row order into gamma' = ||s||^2 and sets beta = gamma'/gamma, the
// iteration count and the stop flag (what k_beta_p does otherwise).
// With hs != NULL the direction of this step is formed here too: before the
// update, p = s + beta p (beta of the previous step, read before the closing
// overwrites it) on the interior columns of each row, whose other entries the
// forward pass updated (PComb); after it, the row's x transform of the new s
// goes to hs, from which the next forward pass forms that of the next p.
template <typename R> struct CgStep {
  C<R>* x;
  C<R>* p;
  C<R>* s;
  const double* alpha;
  int* flag;
  double* part;
  int join_branch;
  double* scal;
  C<R>* hs;
  const double* beta;
};
// The direction update p = s + beta p of a 2D CGNR step, fused into the forward
// apply of T p (whose first pass it replaces): the x transform of p is formed
// from those of s and of the previous p, hp = hs + beta hp (the transform is
// linear), written back to hp; the x-boundary columns of p (also the corners),
// which the apply reads as coefficients, become s + beta p in place.  beta = 0
// takes s alone.  Nothing is written while flag[0] != F_RUN.
template <typename R> struct PComb {
  const C<R>* hs;
  C<R>* hp;
  const C<R>* s;
  C<R>* p;
  const double* beta;
  const int* flag;
};
template <typename R>
gs_status nfft_TH(Plan* P, PrecData<R>& D, const C<R>* y, C<R>* z, const int32_t* perm, cudaStream_t st,
                  const CgStep<R>* cg = nullptr);
template <typename R>
gs_status nfft_TH_scratch(Plan* P, PrecData<R>& D, const C<R>* y, C<R>* z, const int32_t* perm, C<R>* part,
                          cudaStream_t st);
template <typename R>
gs_status direct_T(Plan* P, PrecData<R>& D, const C<R>* x, C<R>* y, const int32_t* perm, cudaStream_t st);
template <typename R>
gs_status direct_TH(Plan* P, PrecData<R>& D, const C<R>* y, C<R>* z, const int32_t* perm, cudaStream_t st);
template <typename R>
inline gs_status apply_T(Plan* P, PrecData<R>& D, const C<R>* x, C<R>* y, const int32_t* perm, cudaStream_t st) {
  return P->direct ? direct_T<R>(P, D, x, y, perm, st) : nfft_T<R>(P, D, x, y, perm, st);
}
template <typename R>
inline gs_status apply_TH(Plan* P, PrecData<R>& D, const C<R>* y, C<R>* z, const int32_t* perm, cudaStream_t st) {
  return P->direct ? direct_TH<R>(P, D, y, z, perm, st) : nfft_TH<R>(P, D, y, z, perm, st);
}
// per-sample 2D kernels (persample2d_f32.cu / persample2d_f64.cu)
template <typename R>
gs_status launch_interp2d(Plan* P, PrecData<R>& D, const C<R>* x, C<R>* y, const int32_t* perm, cudaStream_t st,
                         double* norm_part = nullptr, const C<R>* hrows = nullptr,  // hrows: row transforms [D.hbuf]
                         bool df = false);  // float64: double-float arithmetic (k_interp2d_df)
template <typename R>
gs_status launch_spread2d(Plan* P, PrecData<R>& D, const C<R>* u, const int32_t* perm, C<R>* part, cudaStream_t st);
// exact lattice path (lattice.cu): T's per-sample pick after the forward passes,
// T^H's folds into the grid, side lines and boundary channels before the inverse
// passes (same tables and workspaces as the NFFT path)
template <typename R>
gs_status lattice_pick(Plan* P, PrecData<R>& D, const C<R>* x, C<R>* y, const int32_t* perm, cudaStream_t st,
                       double* norm_part, const C<R>* hrows);
template <typename R>
gs_status lattice_fold(Plan* P, PrecData<R>& D, const C<R>* u, const int32_t* perm, cudaStream_t st);
template <typename R>
gs_status gather_sorted(Plan* P, const C<R>* y_user, C<R>* y_sorted, cudaStream_t st);
template <typename R>
gs_status scatter_user(Plan* P, const C<R>* y_sorted, C<R>* y_user, cudaStream_t st);
// implemented in solve.cu
gs_status solve(Plan* P, const double* y, double* x, const gs_solve_opts& o, gs_solve_info* info,
                cudaStream_t st);
gs_status solve_batch(Plan** plans, int B, const double* const* y, double* const* x, const gs_solve_opts& o,
                      gs_solve_info* infos, cudaStream_t st);

inline int ilog2(int64_t n) {
  int l = 0;
  while ((int64_t(1) << l) < n) ++l;
  return l;
}

}  // namespace gs

struct gs_plan_s {
  gs::Plan P;
};
