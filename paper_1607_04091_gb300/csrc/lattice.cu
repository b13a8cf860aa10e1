// Exact lattice path of T and T^H (Sec. 3.2: on a uniform grid the NDFT is a
// phase-shifted DFT, no spreading).
//
// When every sampling frequency lies on the lattice (1/sigma) Z^d, the
// oversampled grid point of a sample is exact: n xi / 2^J = sigma xi is an
// integer j, and the interior sum
//     sum_k x_k e^{-2 pi i k xi / 2^J} = sum_k x_k e^{-2 pi i k j / n}
// is entry j (mod n) of the length-n DFT of the interior coefficients placed at
// (k mod n) -- the DFT of Sec. 3.2's zero-interleaved vector, with the index
// shift written as a wrap instead of the printed phase factors.  So the plan's
// FFT passes run with the deapodisation factors set to one, and
//   T   picks that one grid value per sample (no window), times the interior
//       factor, plus the boundary terms exactly as on the NFFT path;
//   T^H folds each sample's value into its one grid point (and, in 2D, into
//       the side lines and corner channels of the boundary terms), then runs the
//       inverse passes.
// The folds sum in a fixed order (no atomics): results are deterministic.  In 2D
// this also covers tensor grids (Table 1's "Uniform 2D"): the row and column
// transforms of the passes carry the shared per-row and per-column factors.
#include "device_common.cuh"

namespace gs {
namespace {
using namespace dev;

__device__ inline int bcol_l(int k, int b, int N) { return (k < b) ? k : N - 1 - (k - b); }

// ---------------------------------------------------------------- 1D
template <typename R>
__global__ void k_pick1d(const int32_t* __restrict__ fl, const C<R>* __restrict__ w, const C<R>* __restrict__ bf,
                         int b, const C<R>* __restrict__ grid, const C<R>* __restrict__ x, int64_t N, int64_t M,
                         const int32_t* __restrict__ perm, C<R>* __restrict__ y) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= M) return;
  C<R> out = cmul(w[s], grid[fl[s]]);
  for (int k = 0; k < b; ++k) {
    out = cadd(out, cmul(bf[s * 2 * b + k], x[k]));
    out = cadd(out, cmul(bf[s * 2 * b + b + k], x[N - 1 - k]));
  }
  y[perm ? perm[s] : s] = out;
}

// grid point j: the sum of u conj(w) over the samples at j (its bin's range)
template <typename R>
__global__ void k_fold1d(const int32_t* __restrict__ bin_start, int tile, const int32_t* __restrict__ fl,
                         const C<R>* __restrict__ w, const C<R>* __restrict__ u, const int32_t* __restrict__ perm,
                         int n, C<R>* __restrict__ grid) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int bin = j / tile;
  C<R> acc = mk<R>(0, 0);
  for (int s = bin_start[bin]; s < bin_start[bin + 1]; ++s)
    if (fl[s] == j) acc = cadd(acc, cmulc(u[perm ? perm[s] : s], w[s]));
  grid[j] = acc;
}

// boundary channel c (1D: 2b channels; 2D: (2b)^2 corners): fixed-order tree sum
// over all samples of u conj(f0[c]) conj(f1[c]) (f1 absent in 1D)
template <typename R>
__global__ void k_fold_chan(const C<R>* __restrict__ bf, int b2, int dims, const C<R>* __restrict__ u,
                            const int32_t* __restrict__ perm, int64_t M, C<R>* __restrict__ out) {
  __shared__ C<R> red[256];
  const int c = blockIdx.x;
  const int kx = (dims == 1) ? c : c % b2, ky = (dims == 1) ? 0 : c / b2;
  C<R> acc = mk<R>(0, 0);
  for (int64_t s = threadIdx.x; s < M; s += blockDim.x) {
    C<R> v = cmulc(u[perm ? perm[s] : s], bf[s * b2 + kx]);
    if (dims == 2) v = cmulc(v, bf[(M + s) * b2 + ky]);
    acc = cadd(acc, v);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}

// ---------------------------------------------------------------- 2D
// T: per work item (the NFFT path's launch shape), one thread per sample:
//   y = wx wy G[jx][jy] + wy sum_k bx_k S0[k][jy] + wx sum_k by_k S1[k][jx] + sum bx by X
// and, when norm_part is set, the item's sum of |y|^2 (lanes, then warps, in order)
template <typename R>
__global__ void __launch_bounds__(128) k_pick2d(const int32_t* __restrict__ work, const int32_t* __restrict__ order,
                                                const int32_t* __restrict__ fl, const C<R>* __restrict__ w,
                                                const C<R>* __restrict__ bf, int b, const C<R>* __restrict__ grid,
                                                const C<R>* __restrict__ hrows, const C<R>* __restrict__ side,
                                                int n, const C<R>* __restrict__ x, int N, int64_t M,
                                                const int32_t* __restrict__ perm, C<R>* __restrict__ y,
                                                double* __restrict__ norm_part) {
  __shared__ double wsum[4];
  const int b2 = 2 * b;
  const int it = order[blockIdx.x];
  const int s0 = work[3 * it + 1], s1 = work[3 * it + 2];
  double nacc = 0.0;
  for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    const int jx = fl[s], jy = fl[M + s];
    const C<R> wxs = w[s], wys = w[M + s];
    C<R> out = cmul(cmul(wxs, wys), grid[(int64_t)jx * n + jy]);
    if (b2 > 0) {
      const C<R>* bx = bf + (int64_t)s * b2;
      const C<R>* by = bf + (M + s) * b2;
      C<R> sx = mk<R>(0, 0), sy = mk<R>(0, 0), cc = mk<R>(0, 0);
      for (int k = 0; k < b2; ++k) {
        const C<R> bxk = bx[k], byk = by[k];
        sx = cadd(sx, cmul(bxk, side[(int64_t)k * n + jy]));
        sy = cadd(sy, cmul(byk, hrows[(int64_t)bcol_l(k, b, N) * n + jx]));
        C<R> rr = mk<R>(0, 0);
        for (int kx = 0; kx < b2; ++kx) rr = cadd(rr, cmul(bx[kx], x[(int64_t)bcol_l(k, b, N) * N + bcol_l(kx, b, N)]));
        cc = cadd(cc, cmul(byk, rr));
      }
      out = cadd(out, cmul(wys, sx));
      out = cadd(out, cmul(wxs, sy));
      out = cadd(out, cc);
    }
    y[perm ? perm[s] : s] = out;
    nacc += (double)out.x * out.x + (double)out.y * out.y;
  }
  if (norm_part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nacc += __shfl_down_sync(0xffffffffu, nacc, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = nacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += wsum[i];
      norm_part[it] = t;
    }
  }
}

// grid point (jx, jy) of bin (bx, by), one thread each (tile x tile CTA): the sum of
// u conj(wx wy) over the bin's samples at that point, staged in chunks
constexpr int FOLD_CHUNK = 256;
template <typename R>
__global__ void k_fold2d_grid(const int32_t* __restrict__ bin_start, int tile, int nbx,
                              const int32_t* __restrict__ fl, const C<R>* __restrict__ w,
                              const C<R>* __restrict__ u, const int32_t* __restrict__ perm, int64_t M, int n,
                              C<R>* __restrict__ grid) {
  __shared__ int pt[FOLD_CHUNK];
  __shared__ C<R> val[FOLD_CHUNK];
  const int bin = blockIdx.x, bx = bin % nbx, by = bin / nbx;
  const int t = threadIdx.x, tx = t / tile, ty = t - tx * tile;
  const int jx = bx * tile + tx, jy = by * tile + ty;
  const int me = tx * tile + ty;
  const int s0 = bin_start[bin], s1 = bin_start[bin + 1];
  C<R> acc = mk<R>(0, 0);
  for (int c0 = s0; c0 < s1; c0 += FOLD_CHUNK) {
    const int nc = min(FOLD_CHUNK, s1 - c0);
    __syncthreads();
    for (int i = t; i < nc; i += blockDim.x) {
      const int s = c0 + i;
      pt[i] = (fl[s] - bx * tile) * tile + (fl[M + s] - by * tile);
      val[i] = cmulc(cmulc(u[perm ? perm[s] : s], w[s]), w[M + s]);
    }
    __syncthreads();
    for (int i = 0; i < nc; ++i)
      if (pt[i] == me) acc = cadd(acc, val[i]);
  }
  grid[(int64_t)jx * n + jy] = acc;
}

// side lines, step 1: CTA per bin (bx, by), thread (dim, k, l): the bin's share of
// dim 0 (x-sides along y): u conj(wy) conj(bx_k) of its samples at jy = by tile + l;
// dim 1 (y-sides along x): u conj(wx) conj(by_k) of its samples at jx = bx tile + l
template <typename R>
__global__ void k_fold2d_side_part(const int32_t* __restrict__ bin_start, int tile, int nbx,
                                   const int32_t* __restrict__ fl, const C<R>* __restrict__ w,
                                   const C<R>* __restrict__ bf, int b2, const C<R>* __restrict__ u,
                                   const int32_t* __restrict__ perm, int64_t M, C<R>* __restrict__ lat) {
  extern __shared__ __align__(16) unsigned char smraw[];
  int* pos = reinterpret_cast<int*>(smraw);                               // [FOLD_CHUNK][2]
  C<R>* uw = reinterpret_cast<C<R>*>(smraw + 2 * FOLD_CHUNK * sizeof(C<R>));  // [FOLD_CHUNK][2]
  C<R>* fk = uw + 2 * FOLD_CHUNK;                                         // [FOLD_CHUNK][2][b2]
  const int bin = blockIdx.x, bx = bin % nbx, by = bin / nbx;
  const int t = threadIdx.x, dim = t / (b2 * tile), r = t - dim * b2 * tile, k = r / tile, l = r - k * tile;
  const bool active = dim < 2;
  const int s0 = bin_start[bin], s1 = bin_start[bin + 1];
  C<R> acc = mk<R>(0, 0);
  for (int c0 = s0; c0 < s1; c0 += FOLD_CHUNK) {
    const int nc = min(FOLD_CHUNK, s1 - c0);
    __syncthreads();
    for (int i = t; i < nc; i += blockDim.x) {
      const int s = c0 + i;
      const C<R> us = u[perm ? perm[s] : s];
      pos[2 * i] = fl[M + s] - by * tile;  // dim 0: position along y
      pos[2 * i + 1] = fl[s] - bx * tile;  // dim 1: position along x
      uw[2 * i] = cmulc(us, w[M + s]);
      uw[2 * i + 1] = cmulc(us, w[s]);
    }
    for (int i = t; i < nc * 2 * b2; i += blockDim.x) {
      const int q = i / (2 * b2), rr = i - q * 2 * b2, d = rr / b2, kk = rr - d * b2;
      fk[i] = bf[((int64_t)d * M + c0 + q) * b2 + kk];  // d = 0: bx, d = 1: by
    }
    __syncthreads();
    if (active)
      for (int i = 0; i < nc; ++i)
        if (pos[2 * i + dim] == l) acc = cadd(acc, cmulc(uw[2 * i + dim], fk[(i * 2 + dim) * b2 + k]));
  }
  if (active) lat[(((int64_t)bin * 2 + dim) * b2 + k) * tile + l] = acc;
}

// side lines, step 2: thread (dim, k, j): the bins' shares summed in bin order,
// over bx (dim 0, j = jy) or over by (dim 1, j = jx)
template <typename R>
__global__ void k_fold2d_side_sum(const C<R>* __restrict__ lat, int tile, int nbx, int b2, int n,
                                  C<R>* __restrict__ side) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)2 * b2 * n) return;
  const int dim = (int)(t / ((int64_t)b2 * n)), r = (int)(t - (int64_t)dim * b2 * n), k = r / n, j = r - k * n;
  const int jb = j / tile, l = j - jb * tile;
  C<R> acc = mk<R>(0, 0);
  for (int q = 0; q < nbx; ++q) {
    const int bin = (dim == 0) ? q + nbx * jb : jb + nbx * q;
    acc = cadd(acc, lat[(((int64_t)bin * 2 + dim) * b2 + k) * tile + l]);
  }
  side[((int64_t)dim * b2 + k) * n + j] = acc;
}

}  // namespace

template <typename R>
gs_status lattice_pick(Plan* P, PrecData<R>& D, const C<R>* x, C<R>* y, const int32_t* perm, cudaStream_t st,
                       double* norm_part, const C<R>* hrows) {
  const int64_t M = P->M;
  if (P->dims == 1) {
    GS_LAUNCH(pname<R>("pick1d<f32>", "pick1d<f64>"), st,
              k_pick1d<R><<<(M + 255) / 256, 256, 0, st>>>(P->fl, D.w, D.bf, P->b, D.grid, x, P->N, M, perm, y));
  } else {
    if (P->nwork == 0) return GS_OK;
    GS_LAUNCH(pname<R>("pick2d<f32>", "pick2d<f64>"), st,
              k_pick2d<R><<<P->nwork, 128, 0, st>>>(P->work, P->work_order, P->fl, D.w, D.bf, P->b, D.grid,
                                                   hrows ? hrows : D.hbuf, D.side, (int)P->n, x, (int)P->N, M, perm,
                                                   y, norm_part));
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

template <typename R>
gs_status lattice_fold(Plan* P, PrecData<R>& D, const C<R>* u, const int32_t* perm, cudaStream_t st) {
  const int64_t M = P->M;
  const int n = (int)P->n, b2 = 2 * P->b, tile = P->tile;
  if (P->dims == 1) {
    GS_LAUNCH(pname<R>("fold1d<f32>", "fold1d<f64>"), st,
              k_fold1d<R><<<(n + 255) / 256, 256, 0, st>>>(P->bin_start, tile, P->fl, D.w, u, perm, n, D.grid));
    if (b2 > 0)
      GS_LAUNCH(pname<R>("fold_chan<f32>", "fold_chan<f64>"), st,
                k_fold_chan<R><<<b2, 256, 0, st>>>(D.bf, b2, 1, u, perm, M, D.corner));
  } else {
    GS_LAUNCH(pname<R>("fold2d_grid<f32>", "fold2d_grid<f64>"), st,
              k_fold2d_grid<R><<<P->nbins, tile * tile, 0, st>>>(P->bin_start, tile, P->nbx, P->fl, D.w, u, perm, M,
                                                                  n, D.grid));
    if (b2 > 0) {
      const size_t sh = (size_t)FOLD_CHUNK * 2 * (2 + b2) * sizeof(C<R>);
      if (sh > 48 * 1024)
        GS_CUDA(cudaFuncSetAttribute((const void*)k_fold2d_side_part<R>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
      const int thr = ((2 * b2 * tile + 31) / 32) * 32;
      GS_LAUNCH(pname<R>("fold2d_side<f32>", "fold2d_side<f64>"), st,
                k_fold2d_side_part<R><<<P->nbins, thr, sh, st>>>(P->bin_start, tile, P->nbx, P->fl, D.w, D.bf, b2, u,
                                                                 perm, M, D.lat));
      const int64_t tot = (int64_t)2 * b2 * n;
      GS_LAUNCH(pname<R>("fold2d_side<f32>", "fold2d_side<f64>"), st,
                k_fold2d_side_sum<R><<<(tot + 255) / 256, 256, 0, st>>>(D.lat, tile, P->nbx, b2, n, D.side));
      GS_LAUNCH(pname<R>("fold_chan<f32>", "fold_chan<f64>"), st,
                k_fold_chan<R><<<b2 * b2, 256, 0, st>>>(D.bf, b2, 2, u, perm, M, D.corner));
    }
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

template gs_status lattice_pick<float>(Plan*, PrecData<float>&, const float2*, float2*, const int32_t*, cudaStream_t,
                                       double*, const float2*);
template gs_status lattice_pick<double>(Plan*, PrecData<double>&, const double2*, double2*, const int32_t*,
                                        cudaStream_t, double*, const double2*);
template gs_status lattice_fold<float>(Plan*, PrecData<float>&, const float2*, const int32_t*, cudaStream_t);
template gs_status lattice_fold<double>(Plan*, PrecData<double>&, const double2*, const int32_t*, cudaStream_t);

}  // namespace gs
