// Direct evaluation of T x and T^H y entry by entry (small problems, and a GPU
// cross-check of the NFFT path).  Interior entries are built on the fly as
// w_m exp(-2 pi i k eta'_m) (Sec. 4; eq. NDFT_def with the wrapped eta'), the
// boundary entries come from the plan's factor tables; 2D entries are products
// of the x and y factors (Sec. 5, App. C).
#include "gs_internal.h"

namespace gs {

namespace {

template <typename R> struct Tr;
template <> struct Tr<float> {
  static __device__ void sc(float a, float* s, float* c) { sincospif(a, s, c); }
};
template <> struct Tr<double> {
  static __device__ void sc(double a, double* s, double* c) { sincospi(a, s, c); }
};

template <typename T> __device__ inline T dmul(T a, T b) {
  T r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// t_{m,i} for dimension d (0 = x carries sqrt(mu) through the tables)
template <typename R>
__device__ inline C<R> factor(const double* xs, const C<R>* w, const C<R>* bf, int64_t M, int d, int64_t s,
                              int i, int N, int J, int b) {
  if (i < b) return bf[((int64_t)d * M + s) * 2 * b + i];
  if (i >= N - b) return bf[((int64_t)d * M + s) * 2 * b + b + (N - 1 - i)];
  double eta = ldexp(xs[(int64_t)d * M + s], -J);
  double ew = eta - rint(eta);
  R ph = (R)(2.0 * (double)(i - N / 2) * ew);  // exp(-2 pi i k eta') = exp(-i pi ph)
  R sn, cs;
  Tr<R>::sc(ph, &sn, &cs);
  C<R> e;
  e.x = cs;
  e.y = -sn;
  return dmul(w[(int64_t)d * M + s], e);
}

template <typename R>
__global__ void k_direct_T(const double* __restrict__ xs, const C<R>* __restrict__ w,
                           const C<R>* __restrict__ bf, int64_t M, int N, int J, int b, int dims,
                           const C<R>* __restrict__ x, const int32_t* __restrict__ perm, C<R>* __restrict__ y) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= M) return;
  C<R> out;
  out.x = 0;
  out.y = 0;
  if (dims == 1) {
    for (int i = 0; i < N; ++i) {
      C<R> t = dmul(factor<R>(xs, w, bf, M, 0, s, i, N, J, b), x[i]);
      out.x += t.x;
      out.y += t.y;
    }
  } else {
    for (int j = 0; j < N; ++j) {
      C<R> row;
      row.x = 0;
      row.y = 0;
      for (int i = 0; i < N; ++i) {
        C<R> t = dmul(factor<R>(xs, w, bf, M, 0, s, i, N, J, b), x[(int64_t)j * N + i]);
        row.x += t.x;
        row.y += t.y;
      }
      C<R> t = dmul(factor<R>(xs, w, bf, M, 1, s, j, N, J, b), row);
      out.x += t.x;
      out.y += t.y;
    }
  }
  y[perm ? perm[s] : s] = out;
}

template <typename R>
__global__ void k_direct_TH(const double* __restrict__ xs, const C<R>* __restrict__ w,
                            const C<R>* __restrict__ bf, int64_t M, int N, int J, int b, int dims,
                            const C<R>* __restrict__ u, const int32_t* __restrict__ perm, C<R>* __restrict__ z) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t nco = (dims == 1) ? N : (int64_t)N * N;
  if (q >= nco) return;
  int i = (int)(q % N), j = (int)(q / N);
  C<R> acc;
  acc.x = 0;
  acc.y = 0;
  for (int64_t s = 0; s < M; ++s) {
    C<R> t = factor<R>(xs, w, bf, M, 0, s, i, N, J, b);
    if (dims == 2) t = dmul(t, factor<R>(xs, w, bf, M, 1, s, j, N, J, b));
    C<R> us = u[perm ? perm[s] : s];
    acc.x += t.x * us.x + t.y * us.y;  // conj(t) u
    acc.y += t.x * us.y - t.y * us.x;
  }
  z[q] = acc;
}

}  // namespace

template <typename R>
gs_status direct_T(Plan* P, PrecData<R>& D, const C<R>* x, C<R>* y, const int32_t* perm, cudaStream_t st) {
  GS_LAUNCH(pname<R>("direct_T<f32>", "direct_T<f64>"), st, k_direct_T<R><<<(P->M + 127) / 128, 128, 0, st>>>(P->xi_sorted, D.w, D.bf, P->M, (int)P->N, P->J, P->b,
                                                    P->dims, x, perm, y));
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

template <typename R>
gs_status direct_TH(Plan* P, PrecData<R>& D, const C<R>* u, C<R>* z, const int32_t* perm, cudaStream_t st) {
  GS_LAUNCH(pname<R>("direct_TH<f32>", "direct_TH<f64>"), st, k_direct_TH<R><<<(P->ncoef + 127) / 128, 128, 0, st>>>(P->xi_sorted, D.w, D.bf, P->M, (int)P->N, P->J, P->b,
                                                         P->dims, u, perm, z));
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

template gs_status direct_T<float>(Plan*, PrecData<float>&, const float2*, float2*, const int32_t*, cudaStream_t);
template gs_status direct_T<double>(Plan*, PrecData<double>&, const double2*, double2*, const int32_t*,
                                    cudaStream_t);
template gs_status direct_TH<float>(Plan*, PrecData<float>&, const float2*, float2*, const int32_t*,
                                    cudaStream_t);
template gs_status direct_TH<double>(Plan*, PrecData<double>&, const double2*, double2*, const int32_t*,
                                     cudaStream_t);

}  // namespace gs
