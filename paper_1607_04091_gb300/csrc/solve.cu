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
#include <vector>

#include "gs_internal.h"

namespace gs {

namespace {

constexpr int RED_BLOCKS = 512;
enum { S_GAMMA = 0, S_DELTA, S_ALPHA, S_BETA, S_GNEW, S_THR2, S_S0, S_ITER, S_MAXIT, S_TMP, S_LOOP };
enum { F_RUN = 0, F_CONV = 1, F_BREAK = 2, F_MAXIT = 3 };

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

// alpha = gamma / ||q||^2
__global__ void k_alpha(const double* part, int np, double* scal, int* flag) {
  if (flag[0] != F_RUN) return;
  double d = block_sum(part, np);
  if (threadIdx.x == 0) {
    scal[S_DELTA] = d;
    double a = scal[S_GAMMA] / d;
    if (!(d > 0.0) || !isfinite(a)) flag[0] = F_BREAK;
    else scal[S_ALPHA] = a;
  }
}

// gamma' = ||s||^2, beta = gamma'/gamma, stop test
__global__ void k_beta(const double* part, int np, double* scal, int* flag) {
  if (flag[0] != F_RUN) return;
  double g = block_sum(part, np);
  if (threadIdx.x == 0) {
    double beta = g / scal[S_GAMMA];
    scal[S_BETA] = beta;
    scal[S_GAMMA] = g;
    scal[S_ITER] += 1.0;
    if (!isfinite(beta)) flag[0] = F_BREAK;
    else if (g <= scal[S_THR2]) flag[0] = F_CONV;
    else if (scal[S_ITER] >= scal[S_MAXIT]) flag[0] = F_MAXIT;
  }
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

// p = s + beta p
template <typename R>
__global__ void k_update_p(C<R>* __restrict__ p, const C<R>* __restrict__ s, int64_t n, const double* scal,
                           const int* flag) {
  if (flag[0] != F_RUN) return;
  const R bt = (R)scal[S_BETA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    C<R> v = p[i], sv = s[i];
    v.x = sv.x + bt * v.x;
    v.y = sv.y + bt * v.y;
    p[i] = v;
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
  gs_status s = apply_T<R>(P, D, D.vp, D.vq, nullptr, st);
  if (s != GS_OK) return s;
  GS_LAUNCH("cgls_norm2", st, k_norm2<R><<<RED_BLOCKS, 256, 0, st>>>(D.vq, M, P->red, P->flag));
  GS_LAUNCH("cgls_scalar", st, k_alpha<<<1, 256, 0, st>>>(P->red, RED_BLOCKS, P->scal, P->flag));
  if (normal_eq) {
    GS_LAUNCH("cgls_axpy", st,
              k_update_xr<R><<<grid_for(nc), 256, 0, st>>>(D.vx, D.vp, nc, nullptr, nullptr, 0, P->scal, P->flag));
    s = apply_TH<R>(P, D, D.vq, D.vz, nullptr, st);
    if (s != GS_OK) return s;
    GS_LAUNCH("cgls_axpy", st,
              k_update_xr<R><<<grid_for(nc), 256, 0, st>>>(nullptr, nullptr, 0, D.vs, D.vz, nc, P->scal, P->flag));
  } else {
    GS_LAUNCH("cgls_axpy", st,
              k_update_xr<R><<<grid_for(nc + M), 256, 0, st>>>(D.vx, D.vp, nc, D.vr, D.vq, M, P->scal, P->flag));
    s = apply_TH<R>(P, D, D.vr, D.vs, nullptr, st);
    if (s != GS_OK) return s;
  }
  GS_LAUNCH("cgls_norm2", st, k_norm2<R><<<RED_BLOCKS, 256, 0, st>>>(D.vs, nc, P->red, P->flag));
  GS_LAUNCH("cgls_scalar", st, k_beta<<<1, 256, 0, st>>>(P->red, RED_BLOCKS, P->scal, P->flag));
  GS_LAUNCH("cgls_axpy", st, k_update_p<R><<<grid_for(nc), 256, 0, st>>>(D.vp, D.vs, nc, P->scal, P->flag));
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

// Capture a whole CG pass as one graph: [enter kernel] -> while(cond) { iteration; cond kernel }.
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
      gs_status s = cg_iteration<R>(P, D, normal_eq, cs);
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

#define GS_TRY(x)               \
  do {                          \
    gs_status s_ = (x);         \
    if (s_ != GS_OK) return s_; \
  } while (0)

// r64 = y64 - T x64 (float64 forward apply)
gs_status residual64(Plan* P, cudaStream_t st) {
  GS_TRY(apply_T<double>(P, P->d, (const double2*)P->x64, P->d.vq, nullptr, st));
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

}  // namespace

gs_status solve(Plan* P, const double* y_user, double* x_user, const gs_solve_opts& o, gs_solve_info* info,
                cudaStream_t st) {
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
  if (o.mode == GS_SOLVE_FP64) {
    if (o.x0_given) GS_TRY(adjoint_of_residual<double>(P, P->d, st));
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
    for (int outer = 0; outer < o.max_outer; ++outer) {
      if (ns2 <= thr2 || total >= o.maxit) break;
      double thr_pass = std::max(0.25 * thr2, o.inner_rtol * o.inner_rtol * ns2);
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
