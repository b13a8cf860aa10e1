// Least-squares solve x = argmin ||T x - y|| (Sec. 2, eq. least_squares) by
// CGLS, the conjugate-gradient method on the normal equations whose cost is the
// products with T and T^H (Sec. 6.3):
//   r = y - T x; s = T^H r; p = s; gamma = ||s||^2
//   repeat: q = T p; alpha = gamma/||q||^2; x += alpha p; r -= alpha q;
//           s = T^H r; gamma' = ||s||^2; p = s + (gamma'/gamma) p
//   until ||s|| <= tol ||T^H y||.
// Dot products, norms and step scalars are float64 on the device in every mode;
// vectors stay in the plan's sorted sample order.  GS_SOLVE_MIXED runs the CGLS
// passes with float32 applies on the current residual and refines x in float64:
// after each pass r = y - T x is formed with a float64 forward apply, and its
// adjoint (float32, exact enough because r is small) gives the stop test.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <thread>
#include <vector>

#include <cstring>

#include "gs_internal.h"

namespace gs {

namespace {

constexpr int RED_BLOCKS = 512;
// scalars of the device-side mixed solve (solve graph)
enum { G_TOL2 = 20, G_MAXIT, G_MAXOUT, G_IRTOL2, G_HB2, G_HY2, G_THR2, G_NS2, G_OUTER, G_TOTAL, G_NR2, G_STOP,
       G_WARM };

template <typename T> __device__ inline double sqn(T v) { return (double)v.x * v.x + (double)v.y * v.y; }

template <typename R>
__global__ void k_norm2(const C<R>* __restrict__ v, int64_t n, double* __restrict__ part,
                        const int* __restrict__ flag) {
  __shared__ double sh[256];
  if (flag && flag[0] != F_RUN) return;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += sqn(v[i]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__device__ double block_sum(const double* part, int np) {
  __shared__ double sh[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) a += part[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  return sh[0];
}

// store the finished sum into scal[slot]
__global__ void k_store(const double* part, int np, double* scal, int slot, const int* flag) {
  if (flag && flag[0] != F_RUN) return;
  double s = block_sum(part, np);
  if (threadIdx.x == 0) scal[slot] = s;
}

// alpha = gamma / ||q||^2, gamma = ||s||^2 of the last iteration (S_GNEW, which
// k_beta_p writes while its other blocks still read the previous S_GAMMA)
__global__ void k_alpha(const double* part, int np, double* scal, int* flag) {
  if (flag[0] != F_RUN) return;
  double d = block_sum(part, np);
  if (threadIdx.x == 0) {
    const double gam = scal[S_GNEW];
    scal[S_GAMMA] = gam;
    scal[S_DELTA] = d;
    double a = gam / d;
    if (!(d > 0.0) || !isfinite(a)) flag[0] = F_BREAK;
    else scal[S_ALPHA] = a;
  }
}

// gamma' = ||s||^2, beta = gamma'/gamma, stop test, and p = s + beta p, in one
// grid: every block forms the same sum of the partials in the same order; block
// 0 records the scalars and the stop flag.  The stop flag is read once per
// block (it may change while the grid runs; a block that sees it set skips its
// part of p, which the ending loop no longer reads).
template <typename R>
__global__ void k_beta_p(const double* __restrict__ part, int np, C<R>* __restrict__ p,
                         const C<R>* __restrict__ s, int64_t n, double* scal, int* flag) {
  __shared__ int run;
  if (threadIdx.x == 0) run = (flag[0] == F_RUN);
  __syncthreads();
  if (!run) return;
  const double g = block_sum(part, np);
  const double beta = g / scal[S_GAMMA];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    scal[S_BETA] = beta;
    scal[S_GNEW] = g;
    scal[S_ITER] += 1.0;
    if (!isfinite(beta)) flag[0] = F_BREAK;
    else if (g <= scal[S_THR2]) flag[0] = F_CONV;
    else if (scal[S_ITER] >= scal[S_MAXIT]) flag[0] = F_MAXIT;
  }
  if (!isfinite(beta)) return;
  const R bt = (R)beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    C<R> v = p[i], sv = s[i];
    v.x = sv.x + bt * v.x;
    v.y = sv.y + bt * v.y;
    p[i] = v;
  }
}

// x += alpha p and s -= alpha z (both ncoef), with the partial sums of the new
// ||s||^2 per block (fixed order: threads, then a tree over the block)
template <typename R>
__global__ void k_update_xs(C<R>* __restrict__ x, const C<R>* __restrict__ p, C<R>* __restrict__ s,
                            const C<R>* __restrict__ z, int64_t n, const double* scal, const int* flag,
                            double* __restrict__ part) {
  __shared__ double sh[256];
  if (flag[0] != F_RUN) return;
  const R a = (R)scal[S_ALPHA];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    C<R> v = x[i], pv = p[i];
    v.x += a * pv.x;
    v.y += a * pv.y;
    x[i] = v;
    C<R> sv = s[i], zv = z[i];
    sv.x -= a * zv.x;
    sv.y -= a * zv.y;
    s[i] = sv;
    acc += sqn(sv);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int t = blockDim.x / 2; t > 0; t >>= 1) {
    if (threadIdx.x < t) sh[threadIdx.x] += sh[threadIdx.x + t];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// x += alpha p (ncoef) and r -= alpha q (M)
template <typename R>
__global__ void k_update_xr(C<R>* __restrict__ x, const C<R>* __restrict__ p, int64_t nc, C<R>* __restrict__ r,
                            const C<R>* __restrict__ q, int64_t M, const double* scal, const int* flag) {
  if (flag[0] != F_RUN) return;
  const R a = (R)scal[S_ALPHA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc + M; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nc) {
      C<R> v = x[i], pv = p[i];
      v.x += a * pv.x;
      v.y += a * pv.y;
      x[i] = v;
    } else {
      int64_t k = i - nc;
      C<R> v = r[k], qv = q[k];
      v.x -= a * qv.x;
      v.y -= a * qv.y;
      r[k] = v;
    }
  }
}

template <typename R>
__global__ void k_copy(C<R>* __restrict__ dst, const C<R>* __restrict__ src, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void k_sub64(double2* __restrict__ r, const double2* __restrict__ y, const double2* __restrict__ q,
                        int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 a = y[i], b = q[i];
    r[i] = make_double2(a.x - b.x, a.y - b.y);
  }
}

__global__ void k_to32(float2* __restrict__ o, const double2* __restrict__ in, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// scalars for a new CGLS pass: gamma = ||s0||^2 (already in S_TMP), thresholds
__global__ void k_init_pass(double* scal, int* flag, double thr2, double maxit) {
  scal[S_GAMMA] = scal[S_TMP];
  scal[S_GNEW] = scal[S_TMP];
  scal[S_BETA] = 0.0;  // the first direction of a pass is p = s
  flag[FL_ARRIVE] = 0;
  scal[S_S0] = scal[S_TMP];
  scal[S_THR2] = thr2;
  scal[S_ITER] = 0.0;
  scal[S_LOOP] = 0.0;
  scal[S_MAXIT] = maxit;
  flag[0] = (scal[S_TMP] <= thr2) ? F_CONV : F_RUN;
}

inline int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g < 1184 ? (g < 1 ? 1 : g) : 1184);
}

template <typename R>
gs_status norm2_into(Plan* P, const C<R>* v, int64_t n, int slot, const int* flag, cudaStream_t st) {
  GS_LAUNCH("solve_norm2", st, k_norm2<R><<<RED_BLOCKS, 256, 0, st>>>(v, n, P->red, flag));
  GS_LAUNCH("solve_store", st, k_store<<<1, 256, 0, st>>>(P->red, RED_BLOCKS, P->scal, slot, flag));
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

// Condition of the while node of a captured CG pass: runs once per iteration,
// unconditionally, and counts the iterations itself, so the loop ends after at
// most scal[S_MAXIT] iterations whatever the stop flag holds.
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int* flag, double* scal) {
  const double c = scal[S_LOOP] + 1.0;
  scal[S_LOOP] = c;
  cudaGraphSetConditional(h, (flag[0] == F_RUN && c < scal[S_MAXIT]) ? 1u : 0u);
}
// enter the loop only if the pass has work
__global__ void k_loop_enter(cudaGraphConditionalHandle h, const int* flag, const double* scal) {
  cudaGraphSetConditional(h, (flag[0] == F_RUN && scal[S_MAXIT] >= 1.0) ? 1u : 0u);
}

// One iteration of CG in either of two equivalent forms:
//   CGLS (normal_eq = false): rhs r in D.vr, updated as r -= alpha q, s = T^H r;
//   CGNR (normal_eq = true):  s updated as s -= alpha T^H q, never re-formed from r,
//     so no large cancellation when r is nearly orthogonal to the range of T.
template <typename R>
gs_status cg_iteration(Plan* P, PrecData<R>& D, bool normal_eq, cudaStream_t st) {
  const int64_t nc = P->ncoef, M = P->M;
  // q = T p with ||q||^2 partials: per work item from the 2D interpolation, else a grid reduction
  int np = RED_BLOCKS;
  gs_status s;
  // 2D CGNR: the step is closed by the adjoint's last pass (no separate beta / p
  // kernel), and p = s + beta p is formed where it is read: its x transform in the
  // forward column pass (from those of s and of the previous p, so that T p needs
  // no row pass), its boundary columns there too, its interior columns in the
  // adjoint's last pass, which also transforms the rows of the new s
  const bool fused = normal_eq && !P->direct && P->dims == 2;
  if (!P->direct && P->dims == 2) {
    np = P->nwork;
    const PComb<R> pc{D.hs, D.hp, D.vs, D.vp, P->scal + S_BETA, P->flag};
    s = nfft_T<R>(P, D, D.vp, D.vq, nullptr, st, P->red, fused ? &pc : nullptr);
    if (s != GS_OK) return s;
  } else {
    s = apply_T<R>(P, D, D.vp, D.vq, nullptr, st);
    if (s != GS_OK) return s;
    GS_LAUNCH("cgls_norm2", st, k_norm2<R><<<RED_BLOCKS, 256, 0, st>>>(D.vq, M, P->red, P->flag));
  }
  // ||s||^2 partials go after the ||q||^2 ones
  double* red_s = P->red + std::max<int64_t>(P->nwork, RED_BLOCKS);
  const int gs = grid_for(nc);
  int np_s = gs;  // number of ||s||^2 partials
  if (normal_eq) {
    // alpha on a side branch: only the update after T^H q needs it
    GS_TRY(fork_aux(P, st, 2));
    cudaStream_t a2 = side_stream(P, st, 2);
    GS_LAUNCH("cgls_scalar", a2, k_alpha<<<1, 256, 0, a2>>>(P->red, np, P->scal, P->flag));
    GS_CUDA(cudaGetLastError());
    if (!P->direct && P->dims == 2) {
      // 2D: the x and s update runs in the adjoint's last pass, one partial per coefficient row
      const CgStep<R> cg{D.vx, D.vp, D.vs, P->scal + S_ALPHA, P->flag, red_s, 2, P->scal, D.hs, P->scal + S_BETA};
      GS_TRY(nfft_TH<R>(P, D, D.vq, D.vz, nullptr, st, &cg));
      np_s = (int)P->N;
    } else {
      s = apply_TH<R>(P, D, D.vq, D.vz, nullptr, st);
      if (s != GS_OK) return s;
      GS_TRY(join_aux(P, st, 2));
      GS_LAUNCH("cgls_axpy", st,
                k_update_xs<R><<<gs, 256, 0, st>>>(D.vx, D.vp, D.vs, D.vz, nc, P->scal, P->flag, red_s));
    }
  } else {
    GS_LAUNCH("cgls_scalar", st, k_alpha<<<1, 256, 0, st>>>(P->red, np, P->scal, P->flag));
    GS_LAUNCH("cgls_axpy", st,
              k_update_xr<R><<<grid_for(nc + M), 256, 0, st>>>(D.vx, D.vp, nc, D.vr, D.vq, M, P->scal, P->flag));
    s = apply_TH<R>(P, D, D.vr, D.vs, nullptr, st);
    if (s != GS_OK) return s;
    GS_LAUNCH("cgls_norm2", st, k_norm2<R><<<gs, 256, 0, st>>>(D.vs, nc, red_s, P->flag));
  }
  if (!fused)
    GS_LAUNCH("cgls_scalar", st, k_beta_p<R><<<gs, 256, 0, st>>>(red_s, np_s, D.vp, D.vs, nc, P->scal, P->flag));
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

// CG iterations per execution of a captured while body.  An iteration that
// starts after the stop flag is set changes nothing (every kernel of the step
// tests the flag), so the body may hold several; the condition kernel, which
// counts body executions and bounds the loop, and the re-evaluation of the
// while node then come once per CG_UNROLL iterations.
constexpr int CG_UNROLL = 2;

// Capture a whole CG pass as one graph: [enter kernel] -> while(cond) { CG_UNROLL iterations; cond kernel }.
template <typename R>
gs_status build_cg_graph(Plan* P, PrecData<R>& D, bool normal_eq, cudaStream_t st, cudaGraphExec_t* out) {
  cudaStream_t cs = P->cap_stream;
  // eager applies into the scratch vectors q and z (recomputed before any use)
  // so that kernel attributes are set outside capture
  GS_CUDA(cudaStreamSynchronize(st));
  {
    gs_status s = apply_T<R>(P, D, D.vp, D.vq, nullptr, cs);
    if (s == GS_OK) s = apply_TH<R>(P, D, D.vq, D.vz, nullptr, cs);
    if (s != GS_OK) return s;
  }
  GS_CUDA(cudaStreamSynchronize(cs));
  cudaGraph_t g = nullptr;
  GS_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaGraphConditionalHandleCreate");
  }
  // entry node
  e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    k_loop_enter<<<1, 1, 0, cs>>>(h, P->flag, P->scal);
    cudaGraph_t gg = nullptr;
    e = cudaStreamEndCapture(cs, &gg);
  }
  cudaGraphNode_t enter = nullptr;
  size_t nn = 1;
  if (e == cudaSuccess) e = cudaGraphGetNodes(g, &enter, &nn);
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t wnode = nullptr;
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&wnode, g, &enter, nullptr, 1, &cp);
  }
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      gs_status s = GS_OK;
      for (int u = 0; u < CG_UNROLL && s == GS_OK; ++u) s = cg_iteration<R>(P, D, normal_eq, cs);
      k_loop_cond<<<1, 1, 0, cs>>>(h, P->flag, P->scal);
      cudaGraph_t bb = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(cs, &bb);
      if (s != GS_OK) {
        cudaGraphDestroy(g);
        return s;
      }
      e = e2;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "capturing the CG pass graph");
  return GS_OK;
}

// One CG pass in precision R from d = 0: D.vx <- d.  s0 = T^H r must already be
// in D.vs, ||s0||^2 in scal[S_TMP] (and r in D.vr for the CGLS form).  The pass
// runs as one captured graph when possible (no host polling, exact stop), else
// as host-driven launches that check the stop flag every `check` iterations
// (also when tracing is on or the environment sets GS_NO_GRAPHS, e.g. for
// profilers that replay kernels one by one).
template <typename R>
gs_status cgls_pass(Plan* P, PrecData<R>& D, double thr2, int maxit, int check, bool normal_eq, cudaStream_t st,
                    int* iters, int* stop) {
  const int64_t nc = P->ncoef;
  GS_CUDA(cudaMemsetAsync(D.vx, 0, nc * sizeof(C<R>), st));
  GS_LAUNCH("solve_copy", st, k_copy<R><<<grid_for(nc), 256, 0, st>>>(D.vp, D.vs, nc));
  if (normal_eq && !P->direct && P->dims == 2) GS_TRY(row_transform<R>(P, D, D.vs, D.hs, st));
  GS_LAUNCH("solve_init_pass", st, k_init_pass<<<1, 1, 0, st>>>(P->scal, P->flag, thr2, (double)maxit));
  GS_CUDA(cudaGetLastError());
  int hflag = F_RUN;
  double hit = 0;
  const int gi = normal_eq ? 1 : 0;
  bool graphed = false;
  static const bool no_graphs = std::getenv("GS_NO_GRAPHS") != nullptr;
  if (!prof_on() && !no_graphs && !D.cg_failed[gi]) {
    if (!D.cg_exec[gi]) {
      if (build_cg_graph<R>(P, D, normal_eq, st, &D.cg_exec[gi]) != GS_OK) {
        D.cg_failed[gi] = true;
        D.cg_exec[gi] = nullptr;
        cudaGetLastError();
      }
    }
    if (D.cg_exec[gi]) {
      GS_CUDA(cudaGraphLaunch(D.cg_exec[gi], st));
      graphed = true;
    }
  }
  if (graphed) {
    GS_CUDA(cudaMemcpyAsync(&hflag, P->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaMemcpyAsync(&hit, P->scal + S_ITER, sizeof(double), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
  } else {
    int done = 0;
    while (true) {
      GS_CUDA(cudaMemcpyAsync(&hflag, P->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
      GS_CUDA(cudaMemcpyAsync(&hit, P->scal + S_ITER, sizeof(double), cudaMemcpyDeviceToHost, st));
      GS_CUDA(cudaStreamSynchronize(st));
      if (hflag != F_RUN || done >= maxit) break;
      for (int k = 0; k < check; ++k) {
        gs_status s = cg_iteration<R>(P, D, normal_eq, st);
        if (s != GS_OK) return s;
        ++done;
      }
    }
  }
  *iters = (int)hit;
  *stop = hflag;
  return GS_OK;
}

template <typename R>
__global__ void k_addto(double2* __restrict__ x, const C<R>* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 v = x[i];
    v.x += (double)d[i].x;
    v.y += (double)d[i].y;
    x[i] = v;
  }
}

// r64 = y64 - T x64: the forward apply from float64 data, its interpolation in
// double-float arithmetic (accurate to ~1e-13, far below what the refinement
// needs)
gs_status residual64(Plan* P, cudaStream_t st) {
  if (P->direct)
    GS_TRY(direct_T<double>(P, P->d, (const double2*)P->x64, P->d.vq, nullptr, st));
  else
    GS_TRY(nfft_T<double>(P, P->d, (const double2*)P->x64, P->d.vq, nullptr, st, nullptr, nullptr, true));
  GS_LAUNCH("solve_sub64", st, k_sub64<<<grid_for(P->M), 256, 0, st>>>((double2*)P->r64, (const double2*)P->y64, P->d.vq, P->M));
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

// stop-test value ||T^H r64||^2 into scal[S_TMP]; the adjoint in precision R,
// its result left in D.vs and the float32/64 copy of r64 in D.vr
template <typename R>
gs_status adjoint_of_residual(Plan* P, PrecData<R>& D, cudaStream_t st);
template <>
gs_status adjoint_of_residual<double>(Plan* P, PrecData<double>& D, cudaStream_t st) {
  GS_LAUNCH("solve_copy", st, k_copy<double><<<grid_for(P->M), 256, 0, st>>>(D.vr, (const double2*)P->r64, P->M));
  GS_TRY(apply_TH<double>(P, D, D.vr, D.vs, nullptr, st));
  return norm2_into<double>(P, D.vs, P->ncoef, S_TMP, nullptr, st);
}
template <>
gs_status adjoint_of_residual<float>(Plan* P, PrecData<float>& D, cudaStream_t st) {
  GS_LAUNCH("solve_to32", st, k_to32<<<grid_for(P->M), 256, 0, st>>>(D.vr, (const double2*)P->r64, P->M));
  GS_TRY(apply_TH<float>(P, D, D.vr, D.vs, nullptr, st));
  return norm2_into<float>(P, D.vs, P->ncoef, S_TMP, nullptr, st);
}

double read_scal(Plan* P, int slot, cudaStream_t st, gs_status* err) {
  double v = 0.0;
  cudaError_t e = cudaMemcpyAsync(&v, P->scal + slot, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) *err = cuda_fail(e, "reading a solver scalar");
  return v;
}

// ---------------------------------------------------------------- device-side mixed solve
// One CUDA graph per plan runs a whole GS_SOLVE_MIXED solve (float32 stop test):
//   setup -> [outer enter] -> while(outer) { pass init -> [inner enter] ->
//   while(inner) { CG iteration; inner cond } -> x += d, r = y - T x (float64),
//   s = T^H r (float32) -> outer cond } -> final
// Every condition kernel runs unconditionally once per loop body and counts the
// loop itself, so the inner loop ends after at most maxit - total iterations and
// the outer loop after at most max_outer passes, whatever the data.
__global__ void k_set_params(double* scal, double tol2, double maxit, double maxout, double irtol2) {
  scal[G_TOL2] = tol2;
  scal[G_MAXIT] = maxit;
  scal[G_MAXOUT] = maxout;
  scal[G_IRTOL2] = irtol2;
}
__global__ void k_solve_setup(double* scal, int* flag) {
  const double hb2 = scal[S_TMP];
  scal[G_HB2] = hb2;
  scal[G_NS2] = hb2;
  scal[G_THR2] = scal[G_TOL2] * hb2;
  scal[G_OUTER] = 0.0;
  scal[G_TOTAL] = 0.0;
  scal[G_STOP] = 0.0;
  scal[S_ITER] = 0.0;
  flag[0] = F_RUN;
}
__global__ void k_outer_enter(cudaGraphConditionalHandle h, const double* scal) {
  const bool go = scal[G_HB2] > 0.0 && scal[G_NS2] > scal[G_THR2] && scal[G_MAXOUT] >= 1.0 &&
                  scal[G_TOTAL] < scal[G_MAXIT];
  cudaGraphSetConditional(h, go ? 1u : 0u);
}
// Squared stop threshold of a refinement pass that starts at ||T^H r||^2 = ns2:
// a pass gains irtol (relative to its own start; a restart from the float64
// residual then removes the float32 drift), and never aims below tol / 2.  The
// first pass of a warm start instead ends at the first level irtol^k ||T^H y||
// below its start, the point where a zero start's pass ends, so that it joins
// that schedule rather than shifting it.
__host__ __device__ inline double pass_threshold(double ns2, double hb2, double tol2, double irtol2,
                                                 bool first_warm) {
  double t2 = irtol2 * ns2;
  if (first_warm) {
    double lev2 = irtol2;
    for (int k = 0; k < 64 && lev2 * hb2 >= ns2; ++k) lev2 *= irtol2;
    t2 = lev2 * hb2;
  }
  return fmax(0.25 * tol2 * hb2, t2);
}

__global__ void k_pass_init(double* scal, int* flag) {
  const double ns2 = scal[S_TMP];
  const double thr = pass_threshold(ns2, scal[G_HB2], scal[G_TOL2], scal[G_IRTOL2],
                                    scal[G_OUTER] == 0.0 && scal[G_WARM] != 0.0);
  scal[S_GAMMA] = ns2;
  scal[S_GNEW] = ns2;
  scal[S_BETA] = 0.0;  // the first direction of a pass is p = s
  flag[FL_ARRIVE] = 0;
  scal[S_S0] = ns2;
  scal[S_THR2] = thr;
  scal[S_ITER] = 0.0;
  scal[S_LOOP] = 0.0;
  scal[S_MAXIT] = scal[G_MAXIT] - scal[G_TOTAL];
  flag[0] = (ns2 <= thr) ? F_CONV : F_RUN;
}
__global__ void k_outer_cond(cudaGraphConditionalHandle h, const int* flag, double* scal) {
  const double outer = scal[G_OUTER] + 1.0;
  scal[G_OUTER] = outer;
  scal[G_TOTAL] += scal[S_ITER];
  scal[G_NS2] = scal[S_TMP];
  if (flag[0] == F_BREAK) scal[G_STOP] = (double)F_BREAK;
  const bool go = flag[0] != F_BREAK && scal[G_NS2] > scal[G_THR2] && outer < scal[G_MAXOUT] &&
                  scal[G_TOTAL] < scal[G_MAXIT];
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// capture the launches of `enq` into a child-graph node of `parent` after `dep`
template <typename F>
gs_status add_child(cudaGraph_t parent, cudaGraphNode_t* dep, cudaStream_t cs, F&& enq, cudaGraphNode_t* out) {
  GS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  gs_status s = enq(cs);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (s != GS_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "capturing a solve-graph segment");
  e = cudaGraphAddChildGraphNode(out, parent, dep, dep ? 1 : 0, g);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddChildGraphNode");
  return GS_OK;
}

gs_status add_kernel(cudaGraph_t parent, cudaGraphNode_t* dep, void* fn, void** args, cudaGraphNode_t* out) {
  cudaKernelNodeParams kp = {};
  kp.func = fn;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(1);
  kp.kernelParams = args;
  GS_CUDA(cudaGraphAddKernelNode(out, parent, dep, dep ? 1 : 0, &kp));
  return GS_OK;
}

gs_status add_while(cudaGraph_t parent, cudaGraphNode_t* dep, cudaGraphConditionalHandle h, cudaGraphNode_t* out,
                    cudaGraph_t* body) {
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  GS_CUDA(cudaGraphAddNode(out, parent, dep, nullptr, dep ? 1 : 0, &cp));
  *body = cp.conditional.phGraph_out[0];
  return GS_OK;
}

__global__ void k_set_scal(double* scal, int slot, double v) { scal[slot] = v; }

// warm start worse than zero (||T^H r0|| >= ||T^H y||): restart from x = 0, r = y,
// s = s_y (kept in vz), the plain method being the fallback
__global__ void k_fallback_zero(double* scal, double2* __restrict__ x, double2* __restrict__ r,
                                const double2* __restrict__ y, float2* __restrict__ s, const float2* __restrict__ sy,
                                int64_t nc, int64_t M) {
  if (!(scal[S_TMP] >= scal[G_HB2])) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc + M; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nc) {
      x[i] = make_double2(0.0, 0.0);
      s[i] = sy[i];
    } else {
      r[i - nc] = y[i - nc];
    }
  }
}
__global__ void k_fallback_scalars(double* scal) {
  if (scal[S_TMP] >= scal[G_HB2]) {
    scal[S_TMP] = scal[G_HB2];
    scal[G_WARM] = 0.0;
  } else {
    scal[G_WARM] = 1.0;
  }
  scal[G_NS2] = scal[S_TMP];
}

// eager applies on the plan's capture stream, so that kernel attributes (dynamic
// shared memory sizes) are set outside any capture
gs_status warm_solve_kernels(Plan* P, cudaStream_t st) {
  cudaStream_t cs = P->cap_stream;
  PrecData<float>& F = P->f;
  GS_CUDA(cudaStreamSynchronize(st));
  GS_TRY(apply_T<float>(P, F, F.vp, F.vq, nullptr, cs));
  GS_TRY(apply_TH<float>(P, F, F.vq, F.vz, nullptr, cs));
  GS_TRY(apply_T<double>(P, P->d, (const double2*)P->x64, P->d.vq, nullptr, cs));
  GS_CUDA(cudaStreamSynchronize(cs));
  return GS_OK;
}

// Adds the nodes of one whole mixed solve of plan P (data in P->y64, start in
// P->x64 when with_x0, parameters in P->scal) to graph G after node dep (NULL:
// no dependency); *last receives its final node.
gs_status add_solve_nodes(Plan* P, bool with_x0, cudaGraph_t G, cudaGraphNode_t dep, cudaGraphNode_t* last) {
  cudaStream_t cs = P->cap_stream;
  PrecData<float>& F = P->f;
  const int64_t nc = P->ncoef, M = P->M;
  cudaGraphConditionalHandle ho, hi;
  GS_CUDA(cudaGraphConditionalHandleCreate(&ho, G, 0, cudaGraphCondAssignDefault));
  cudaGraphNode_t n_setup, n_oenter, n_outer, n_final;
  GS_TRY(add_child(G, dep ? &dep : nullptr, cs, [&](cudaStream_t c) -> gs_status {
    GS_TRY(norm2_into<double>(P, (const double2*)P->y64, M, G_HY2, nullptr, c));
    if (!with_x0) GS_CUDA(cudaMemsetAsync(P->x64, 0, nc * sizeof(double2), c));
    k_copy<double><<<grid_for(M), 256, 0, c>>>((double2*)P->r64, (const double2*)P->y64, M);
    GS_TRY(adjoint_of_residual<float>(P, F, c));  // ||T^H y||^2, the scale of the stop test
    k_solve_setup<<<1, 1, 0, c>>>(P->scal, P->flag);
    if (with_x0) {  // r = y - T x0 (float64) and its stop-test value; zero start if not better
      k_copy<float><<<grid_for(nc), 256, 0, c>>>(F.vz, F.vs, nc);  // T^H y, for the fallback
      GS_TRY(residual64(P, c));
      GS_TRY(adjoint_of_residual<float>(P, F, c));
      k_fallback_zero<<<grid_for(nc + M), 256, 0, c>>>(P->scal, (double2*)P->x64, (double2*)P->r64,
                                                       (const double2*)P->y64, F.vs, F.vz, nc, M);
      k_fallback_scalars<<<1, 1, 0, c>>>(P->scal);
    }
    GS_CUDA(cudaGetLastError());
    return GS_OK;
  }, &n_setup));
  void* a_oenter[] = {&ho, &P->scal};
  GS_TRY(add_kernel(G, &n_setup, (void*)k_outer_enter, a_oenter, &n_oenter));
  cudaGraph_t outer_body = nullptr;
  GS_TRY(add_while(G, &n_oenter, ho, &n_outer, &outer_body));
  GS_CUDA(cudaGraphConditionalHandleCreate(&hi, outer_body, 0, cudaGraphCondAssignDefault));
  cudaGraphNode_t n_pinit, n_ienter, n_inner, n_post, n_ocond;
  GS_TRY(add_child(outer_body, nullptr, cs, [&](cudaStream_t c) -> gs_status {
    k_pass_init<<<1, 1, 0, c>>>(P->scal, P->flag);
    GS_CUDA(cudaMemsetAsync(F.vx, 0, nc * sizeof(float2), c));
    k_copy<float><<<grid_for(nc), 256, 0, c>>>(F.vp, F.vs, nc);
    if (!P->direct && P->dims == 2) GS_TRY(row_transform<float>(P, F, F.vs, F.hs, c));
    GS_CUDA(cudaGetLastError());
    return GS_OK;
  }, &n_pinit));
  void* a_ienter[] = {&hi, &P->flag, &P->scal};
  GS_TRY(add_kernel(outer_body, &n_pinit, (void*)k_loop_enter, a_ienter, &n_ienter));
  cudaGraph_t inner_body = nullptr;
  GS_TRY(add_while(outer_body, &n_ienter, hi, &n_inner, &inner_body));
  {
    GS_CUDA(cudaStreamBeginCaptureToGraph(cs, inner_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    gs_status sc = GS_OK;
    for (int u = 0; u < CG_UNROLL && sc == GS_OK; ++u) sc = cg_iteration<float>(P, F, true, cs);
    k_loop_cond<<<1, 1, 0, cs>>>(hi, P->flag, P->scal);
    cudaGraph_t bb = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &bb);
    if (sc != GS_OK) return sc;
    if (e != cudaSuccess) return cuda_fail(e, "capturing the CG iteration");
  }
  GS_TRY(add_child(outer_body, &n_inner, cs, [&](cudaStream_t c) -> gs_status {
    k_addto<float><<<grid_for(nc), 256, 0, c>>>((double2*)P->x64, F.vx, nc);
    GS_TRY(residual64(P, c));
    return adjoint_of_residual<float>(P, F, c);
  }, &n_post));
  void* a_ocond[] = {&ho, &P->flag, &P->scal};
  GS_TRY(add_kernel(outer_body, &n_post, (void*)k_outer_cond, a_ocond, &n_ocond));
  GS_TRY(add_child(G, &n_outer, cs, [&](cudaStream_t c) -> gs_status {
    return norm2_into<double>(P, (const double2*)P->r64, M, G_NR2, nullptr, c);
  }, &n_final));
  *last = n_final;
  return GS_OK;
}

gs_status build_solve_graph(Plan* P, bool with_x0, cudaStream_t st, cudaGraphExec_t* out) {
  GS_TRY(warm_solve_kernels(P, st));
  P->solve_kernels_warm = true;
  cudaGraph_t G = nullptr;
  GS_CUDA(cudaGraphCreate(&G, 0));
  struct Guard {
    cudaGraph_t g;
    ~Guard() {
      if (g) cudaGraphDestroy(g);
    }
  } guard{G};
  cudaGraphNode_t last = nullptr;
  GS_TRY(add_solve_nodes(P, with_x0, G, nullptr, &last));
  GS_CUDA(cudaGraphInstantiate(out, G, 0));
  return GS_OK;
}

// mixed solve through the cached solve graph; y_user and x_user as in gs_solve
gs_status launch_solve_graph(Plan* P, const double* y_user, double* x_user, const gs_solve_opts& o,
                             cudaStream_t st) {
  const int gi = o.x0_given ? 1 : 0;
  if (!P->solve_exec[gi]) {
    gs_status s = build_solve_graph(P, gi == 1, st, &P->solve_exec[gi]);
    if (s != GS_OK) {
      P->solve_exec[gi] = nullptr;
      P->solve_graph_failed = true;
      return s;
    }
  }
  if (o.x0_given) GS_CUDA(cudaMemcpyAsync(P->x64, x_user, P->ncoef * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  GS_TRY(gather_sorted<double>(P, (const double2*)y_user, (double2*)P->y64, st));
  k_set_params<<<1, 1, 0, st>>>(P->scal, o.tol * o.tol, (double)o.maxit, (double)o.max_outer,
                                o.inner_rtol * o.inner_rtol);
  GS_CUDA(cudaGetLastError());
  GS_CUDA(cudaGraphLaunch(P->solve_exec[gi], st));
  GS_CUDA(cudaMemcpyAsync(x_user, P->x64, P->ncoef * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  return GS_OK;
}

// info of a finished graph solve (host reads the plan's scalars)
gs_status graph_solve_info(Plan* P, const gs_solve_opts& o, gs_solve_info* info) {
  double sc[40];
  GS_CUDA(cudaMemcpy(sc, P->scal, sizeof(sc), cudaMemcpyDeviceToHost));
  gs_solve_info inf = {0, 0, 0.0, 0.0, GS_OK};
  const double hb2 = sc[G_HB2], hy2 = sc[G_HY2];
  inf.iterations = (int)sc[G_TOTAL];
  inf.outer = (int)sc[G_OUTER];
  P->last_iters = inf.iterations;
  inf.rel_normres = hb2 > 0 ? std::sqrt(sc[G_NS2] / hb2) : 0.0;
  inf.rel_res = hy2 > 0 ? std::sqrt((hb2 > 0 ? sc[G_NR2] : hy2) / hy2) : 0.0;
  gs_status rc = GS_OK;
  if (sc[G_STOP] == (double)F_BREAK) rc = GS_EBREAKDOWN;
  else if (hb2 > 0 && sc[G_NS2] > sc[G_THR2]) rc = GS_ENOTCONV;
  inf.status = rc;
  if (info) *info = inf;
  if (rc != GS_OK) set_error("solve stopped: relative normal-equation residual %.3e after %d iterations",
                             inf.rel_normres, inf.iterations);
  return rc;
}

bool graph_solve_ok(Plan* P, const gs_solve_opts& o) {
  static const bool no_graphs = std::getenv("GS_NO_GRAPHS") != nullptr;
  return o.mode == GS_SOLVE_MIXED && o.tol >= 1e-7 && !prof_on() && !no_graphs && !P->solve_graph_failed;
}

}  // namespace

gs_status solve(Plan* P, const double* y_user, double* x_user, const gs_solve_opts& o, gs_solve_info* info,
                cudaStream_t st) {
  if (graph_solve_ok(P, o)) {
    gs_status s = launch_solve_graph(P, y_user, x_user, o, st);
    if (s == GS_OK) {
      GS_CUDA(cudaStreamSynchronize(st));
      return graph_solve_info(P, o, info);
    }
    if (!P->solve_graph_failed) return s;
    cudaGetLastError();  // graph could not be built: fall through to host-driven passes
  }
  const int64_t nc = P->ncoef, M = P->M;
  double2* y64 = (double2*)P->y64;
  double2* x64 = (double2*)P->x64;
  gs_solve_info inf = {0, 0, 0.0, 0.0, GS_OK};
  gs_status err = GS_OK;
  GS_TRY(gather_sorted<double>(P, (const double2*)y_user, y64, st));
  GS_TRY(norm2_into<double>(P, y64, M, S_TMP, nullptr, st));
  const double hy2 = read_scal(P, S_TMP, st, &err);
  if (err != GS_OK) return err;
  // ||T^H y||^2, the scale of the stop test
  GS_CUDA(cudaMemsetAsync(x64, 0, nc * sizeof(double2), st));
  GS_LAUNCH("solve_copy", st, k_copy<double><<<grid_for(M), 256, 0, st>>>((double2*)P->r64, y64, M));
  if (o.mode == GS_SOLVE_FP64 || o.tol < 1e-7) GS_TRY(adjoint_of_residual<double>(P, P->d, st));
  else GS_TRY(adjoint_of_residual<float>(P, P->f, st));
  const double hb2 = read_scal(P, S_TMP, st, &err);
  if (err != GS_OK) return err;
  if (!(hb2 > 0.0)) {  // T^H y = 0: x = 0 is a least-squares solution
    GS_CUDA(cudaMemsetAsync(x_user, 0, nc * sizeof(double2), st));
    inf.rel_res = 1.0;
    inf.outer = 0;
    if (info) *info = inf;
    return GS_OK;
  }
  const double thr2 = o.tol * o.tol * hb2;
  if (o.x0_given) {
    GS_LAUNCH("solve_copy", st, k_copy<double><<<grid_for(nc), 256, 0, st>>>(x64, (const double2*)x_user, nc));
    GS_TRY(residual64(P, st));
  }
  const int check = 4;
  int total = 0, stop = F_RUN;
  double ns2 = hb2;
  GS_LAUNCH("solve_set_scal", st, k_set_scal<<<1, 1, 0, st>>>(P->scal, G_WARM, o.x0_given ? 1.0 : 0.0));
  if (o.mode == GS_SOLVE_FP64) {
    if (o.x0_given) {
      GS_TRY(adjoint_of_residual<double>(P, P->d, st));
      if (read_scal(P, S_TMP, st, &err) >= hb2) {  // warm start not better than zero: zero start
        GS_CUDA(cudaMemsetAsync(x64, 0, nc * sizeof(double2), st));
        GS_LAUNCH("solve_copy", st, k_copy<double><<<grid_for(M), 256, 0, st>>>((double2*)P->r64, y64, M));
        GS_TRY(adjoint_of_residual<double>(P, P->d, st));
        GS_LAUNCH("solve_set_scal", st, k_set_scal<<<1, 1, 0, st>>>(P->scal, G_WARM, 0.0));
      }
      if (err != GS_OK) return err;
    }
    // D.vr holds r, D.vs = T^H r, scal[S_TMP] = ||T^H r||^2
    GS_TRY(cgls_pass<double>(P, P->d, thr2, o.maxit, check, false, st, &total, &stop));
    GS_LAUNCH("solve_addto", st, k_addto<double><<<grid_for(nc), 256, 0, st>>>(x64, P->d.vx, nc));
    GS_TRY(residual64(P, st));
    GS_TRY(adjoint_of_residual<double>(P, P->d, st));
    ns2 = read_scal(P, S_TMP, st, &err);
    if (err != GS_OK) return err;
    inf.outer = 1;
  } else {
    // stop test (and pass rhs) T^H r in float64 when tol is below what a float32
    // adjoint of r can resolve (~1e-7 relative), else in float32
    const bool hi = o.tol < 1e-7;
    auto check_value = [&]() -> gs_status {
      if (hi) {
        GS_TRY(adjoint_of_residual<double>(P, P->d, st));
        ns2 = read_scal(P, S_TMP, st, &err);
        if (err != GS_OK) return err;
        GS_LAUNCH("solve_to32", st, k_to32<<<grid_for(nc), 256, 0, st>>>(P->f.vs, P->d.vs, nc));
        GS_CUDA(cudaGetLastError());
        return norm2_into<float>(P, P->f.vs, nc, S_TMP, nullptr, st);
      }
      GS_TRY(adjoint_of_residual<float>(P, P->f, st));
      ns2 = read_scal(P, S_TMP, st, &err);
      return err;
    };
    if (o.x0_given || hi) GS_TRY(check_value());
    bool warm = o.x0_given;
    if (o.x0_given && ns2 >= hb2) {  // warm start not better than zero: zero start
      GS_CUDA(cudaMemsetAsync(x64, 0, nc * sizeof(double2), st));
      GS_LAUNCH("solve_copy", st, k_copy<double><<<grid_for(M), 256, 0, st>>>((double2*)P->r64, y64, M));
      GS_TRY(check_value());
      GS_LAUNCH("solve_set_scal", st, k_set_scal<<<1, 1, 0, st>>>(P->scal, G_WARM, 0.0));
      warm = false;
    }
    for (int outer = 0; outer < o.max_outer; ++outer) {
      if (ns2 <= thr2 || total >= o.maxit) break;
      double thr_pass = pass_threshold(ns2, hb2, o.tol * o.tol, o.inner_rtol * o.inner_rtol, outer == 0 && warm);
      int it = 0;
      GS_TRY(cgls_pass<float>(P, P->f, thr_pass, o.maxit - total, check, true, st, &it, &stop));
      total += it;
      inf.outer = outer + 1;
      GS_LAUNCH("solve_addto", st, k_addto<float><<<grid_for(nc), 256, 0, st>>>(x64, P->f.vx, nc));
      GS_TRY(residual64(P, st));
      GS_TRY(check_value());
      if (stop == F_BREAK) break;
    }
  }
  GS_TRY(norm2_into<double>(P, (const double2*)P->r64, M, S_TMP, nullptr, st));
  const double nr2 = read_scal(P, S_TMP, st, &err);
  if (err != GS_OK) return err;
  GS_CUDA(cudaMemcpyAsync(x_user, x64, nc * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  inf.iterations = total;
  inf.rel_normres = std::sqrt(ns2 / hb2);
  inf.rel_res = hy2 > 0 ? std::sqrt(nr2 / hy2) : 0.0;
  gs_status rc = GS_OK;
  if (stop == F_BREAK) rc = GS_EBREAKDOWN;
  else if (ns2 > thr2) rc = GS_ENOTCONV;
  inf.status = rc;
  if (info) *info = inf;
  if (rc != GS_OK) set_error("solve stopped: relative normal-equation residual %.3e after %d iterations",
                             inf.rel_normres, total);
  return rc;
}

}  // namespace gs

// ---------------------------------------------------------------- batched solves
namespace gs {
namespace {
constexpr int POOL = 16;
struct StreamPool {
  int dev = -1;
  cudaStream_t s[POOL] = {};
  cudaEvent_t done[POOL] = {};
  cudaEvent_t start = nullptr;
};
StreamPool g_pools[64];
std::mutex g_pool_mu;

gs_status get_pool(StreamPool** out) {
  int dev = 0;
  GS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d unsupported", dev);
    return GS_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> g(g_pool_mu);
  StreamPool& p = g_pools[dev];
  if (p.dev < 0) {
    for (int i = 0; i < POOL; ++i) {
      GS_CUDA(cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking));
      GS_CUDA(cudaEventCreateWithFlags(&p.done[i], cudaEventDisableTiming));
    }
    GS_CUDA(cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming));
    p.dev = dev;
  }
  *out = &p;
  return GS_OK;
}
}  // namespace

// ---------------------------------------------------------------- batch schedule
// A batch of mixed solves: each problem's whole solve is one CUDA graph (nested
// while-conditional nodes), launched on one of POOL library-owned streams.  The
// problems are assigned to streams up front by longest-processing-time-first:
// sorted by estimated cost, each to the stream with the least work so far, so the
// host enqueues every launch at once and waits only at the end.  The cost of a
// solve is its CG iterations times a per-iteration time model (a fixed ~40 us of
// small kernels plus terms in M and the coefficient count); the iterations are
// those of the plan's previous solve when it has one (the schedule tunes itself
// on measured counts), else a common guess.  (One graph holding all solves as 16
// chains was measured and is slower: 23.6 against ~35 problems/s on the
// 512-problem batch, the chains' nested loops barely overlapping.)
double solve_cost(const Plan* P) {
  const double per_it = 40.0 + (double)P->M / 3000.0 + (double)P->ncoef / 1000.0;  // us
  return ((P->last_iters > 0) ? (double)P->last_iters + 1.0 : 100.0) * per_it;
}

gs_status solve_batch_graphs(Plan** plans, int B, const double* const* y, double* const* x,
                             const gs_solve_opts& o, gs_solve_info* infos, cudaStream_t st) {
  StreamPool* pool = nullptr;
  GS_TRY(get_pool(&pool));
  std::lock_guard<std::mutex> g(g_pool_mu);
  // graphs first (building one synchronises), then every launch
  const int gi = o.x0_given ? 1 : 0;
  for (int p = 0; p < B; ++p) {
    Plan* P = plans[p];
    if (P->solve_exec[gi]) continue;
    gs_status s = build_solve_graph(P, gi == 1, st, &P->solve_exec[gi]);
    if (s != GS_OK) {
      P->solve_exec[gi] = nullptr;
      P->solve_graph_failed = true;
      return s;
    }
  }
  std::vector<int> ord(B);
  std::vector<double> cost(B);
  for (int p = 0; p < B; ++p) {
    ord[p] = p;
    cost[p] = solve_cost(plans[p]);
  }
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  const int ns = B < POOL ? B : POOL;
  std::vector<std::vector<int>> lane(ns);
  std::vector<double> load(ns, 0.0);
  for (int p : ord) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lane[l].push_back(p);
    load[l] += cost[p];
  }
  GS_CUDA(cudaEventRecord(pool->start, st));
  for (int i = 0; i < ns; ++i) GS_CUDA(cudaStreamWaitEvent(pool->s[i], pool->start, 0));
  // round-robin over the streams, so that streams sharing a hardware queue
  // interleave their solves in schedule order instead of one stream's whole list
  // queueing ahead of the other's
  size_t depth = 0;
  for (int i = 0; i < ns; ++i) depth = std::max(depth, lane[i].size());
  for (size_t r = 0; r < depth; ++r)
    for (int i = 0; i < ns; ++i)
      if (r < lane[i].size()) GS_TRY(launch_solve_graph(plans[lane[i][r]], y[lane[i][r]], x[lane[i][r]], o, pool->s[i]));
  for (int i = 0; i < ns; ++i) {
    GS_CUDA(cudaEventRecord(pool->done[i], pool->s[i]));
    GS_CUDA(cudaStreamWaitEvent(st, pool->done[i], 0));
  }
  GS_CUDA(cudaStreamSynchronize(st));
  gs_status first = GS_OK;
  for (int p = 0; p < B; ++p) {
    gs_solve_info inf;
    gs_status r = graph_solve_info(plans[p], o, &inf);
    if (infos) infos[p] = inf;
    if (r != GS_OK && first == GS_OK) first = r;
  }
  return first;
}

// In a batch the problems' kernels run side by side, and CTAs launched early to
// wait for the kernel before them (the programmatic launches of the spread and the
// reductions) would only hold SM space that other problems' kernels could use:
// measured on the 512-problem bench batch, 39.4 problems/s with them against 41.2
// without.  So a plan solved in a batch launches without them from then on; its
// graphs, captured with them, are rebuilt once (after a device synchronisation,
// so that no launch of a destroyed graph is in flight).
static gs_status batch_launch_mode(Plan** plans, int B) {
  bool stale = false;
  for (int p = 0; p < B; ++p) stale = stale || plans[p]->pdl;
  if (!stale) return GS_OK;
  GS_CUDA(cudaDeviceSynchronize());
  for (int p = 0; p < B; ++p) {
    Plan* P = plans[p];
    if (!P->pdl) continue;
    P->pdl = false;
    for (int i = 0; i < 2; ++i) {
      if (P->solve_exec[i]) cudaGraphExecDestroy(P->solve_exec[i]);
      P->solve_exec[i] = nullptr;
      if (P->f.cg_exec[i]) cudaGraphExecDestroy(P->f.cg_exec[i]);
      P->f.cg_exec[i] = nullptr;
      if (P->d.cg_exec[i]) cudaGraphExecDestroy(P->d.cg_exec[i]);
      P->d.cg_exec[i] = nullptr;
    }
  }
  return GS_OK;
}

gs_status solve_batch(Plan** plans, int B, const double* const* y, double* const* x, const gs_solve_opts& o,
                      gs_solve_info* infos, cudaStream_t st) {
  GS_TRY(batch_launch_mode(plans, B));
  bool all_graph = true;
  for (int p = 0; p < B; ++p) all_graph = all_graph && graph_solve_ok(plans[p], o);
  if (all_graph) return solve_batch_graphs(plans, B, y, x, o, infos, st);
  // options without a device-side solve (float64 mode, tol < 1e-7, tracing): one
  // solve per problem, launched on 16 streams as they come free
  StreamPool* pool = nullptr;
  GS_TRY(get_pool(&pool));
  std::lock_guard<std::mutex> g(g_pool_mu);
  GS_CUDA(cudaEventRecord(pool->start, st));
  const int ns = B < POOL ? B : POOL;
  for (int i = 0; i < ns; ++i) GS_CUDA(cudaStreamWaitEvent(pool->s[i], pool->start, 0));
  std::vector<char> graphed(B, 0);
  gs_status first = GS_OK;
  // largest problems first (samples x coefficients), each on the first stream whose
  // previous solve has finished: the streams stay busy however the work is spread
  std::vector<int> ord(B);
  for (int p = 0; p < B; ++p) ord[p] = p;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    return (double)plans[a]->M * (double)plans[a]->ncoef > (double)plans[b]->M * (double)plans[b]->ncoef;
  });
  std::vector<char> busy(ns, 0);
  int next = 0;
  while (next < B) {
    bool launched = false;
    for (int i = 0; i < ns && next < B; ++i) {
      if (busy[i]) {
        const cudaError_t q = cudaEventQuery(pool->done[i]);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return cuda_fail(q, "waiting for a batch stream");
      }
      const int p = ord[next++];
      cudaStream_t s = pool->s[i];
      bool done_graph = false;
      if (graph_solve_ok(plans[p], o)) {
        gs_status r = launch_solve_graph(plans[p], y[p], x[p], o, s);
        if (r == GS_OK) {
          graphed[p] = 1;
          done_graph = true;
        } else {
          if (!plans[p]->solve_graph_failed) return r;
          cudaGetLastError();
        }
      }
      if (!done_graph) {
        gs_solve_info inf;
        gs_status r = solve(plans[p], y[p], x[p], o, &inf, s);  // host-driven fallback
        if (infos) infos[p] = inf;
        if (r != GS_OK && first == GS_OK) first = r;
      }
      GS_CUDA(cudaEventRecord(pool->done[i], s));
      busy[i] = 1;
      launched = true;
    }
    if (!launched) std::this_thread::yield();
  }
  for (int i = 0; i < ns; ++i) {
    GS_CUDA(cudaEventRecord(pool->done[i], pool->s[i]));
    GS_CUDA(cudaStreamWaitEvent(st, pool->done[i], 0));
  }
  GS_CUDA(cudaStreamSynchronize(st));
  for (int p = 0; p < B; ++p) {
    if (!graphed[p]) continue;
    gs_solve_info inf;
    gs_status r = graph_solve_info(plans[p], o, &inf);
    if (infos) infos[p] = inf;
    if (r != GS_OK && first == GS_OK) first = r;
  }
  return first;
}

}  // namespace gs
