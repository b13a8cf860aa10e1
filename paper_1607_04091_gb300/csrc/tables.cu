// Plan construction: binning of the samples into grid tiles, density weights,
// and the per-sample factor tables of T (Sec. 4, Sec. 5; App. A, A.1).
//
// Tables per sample and dimension, built in float64 on the GPU:
//   w   = sqrt(mu) 2^-J/2 phi-hat(xi / 2^J)                       (interior, D of Sec. 4)
//   bf  = sqrt(mu) 2^-J/2 exp(+pi i xi) phi^L_k-hat(xi / 2^J)     (left, k < b)
//         sqrt(mu) 2^-J/2 exp(-pi i xi) phi^R_k-hat(xi / 2^J)     (right, k < b)
// (sqrt(mu) only on the x factor in 2D).  phi-hat is the product of App. A
// (from j = 1), cut at depth D with |xi/2^(J+D)| <= 2^-30 and closed by the
// second-order Taylor polynomial 1 - 2 pi i mu1 z - 2 pi^2 mu2 z^2 of phi-hat
// at that tiny argument (error below 1e-24).  The boundary transforms follow
// the recursion v1(eta) = U v1(eta/2) + V v2(eta/2) of App. A.1, unrolled D
// times from v1(0), evaluated innermost-first together with phi-hat at every
// level.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gs_internal.h"
#include "device_common.cuh"

namespace gs {

namespace {

__constant__ double c_h[2 * GS_MAX_P];
__constant__ double c_UL[GS_MAX_P * GS_MAX_P], c_VL[GS_MAX_P * (2 * GS_MAX_P - 1)], c_v0L[GS_MAX_P];
__constant__ double c_UR[GS_MAX_P * GS_MAX_P], c_VR[GS_MAX_P * (2 * GS_MAX_P - 1)], c_v0R[GS_MAX_P];

__device__ inline double2 cm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Grid coordinate of each sample: eta = xi / 2^J wrapped to [-1/2, 1/2]
// (the interior NDFT is 1-periodic in eta for integer k), u = n eta.
__global__ void k_coords(const double* __restrict__ xi, int64_t M, int dims, int J, int64_t n,
                         int tile, int nbx, int32_t* __restrict__ fl, int32_t* __restrict__ key) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= M) return;
  int kk = 0;
  for (int d = 0; d < dims; ++d) {
    double eta = ldexp(xi[d * M + s], -J);
    double ew = eta - rint(eta);
    double u = ew * (double)n;
    double f = floor(u);
    int64_t li = (int64_t)f;
    li = ((li % n) + n) % n;
    fl[d * M + s] = (int32_t)li;
    int b = (int)(li / tile);
    kk += (d == 0) ? b : b * nbx;
  }
  key[s] = kk;
}

// Stable counting sort by bin, step 1: histogram of each chunk of 1024 samples.
constexpr int SORT_CHUNK = 1024;
__global__ void k_chunk_hist(const int32_t* __restrict__ key, int64_t M, int nbins,
                             int32_t* __restrict__ counts) {
  extern __shared__ int32_t sh[];
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * SORT_CHUNK;
  for (int i = threadIdx.x; i < SORT_CHUNK; i += blockDim.x) {
    int64_t s = base + i;
    if (s < M) atomicAdd(&sh[key[s]], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) counts[(int64_t)blockIdx.x * nbins + i] = sh[i];
}

// step 2: per bin, exclusive scan over chunks (in place) and the bin total.
__global__ void k_scan_chunks(int32_t* counts, int nchunks, int nbins, int32_t* total) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  int32_t run = 0;
  for (int c = 0; c < nchunks; ++c) {
    int32_t v = counts[(int64_t)c * nbins + b];
    counts[(int64_t)c * nbins + b] = run;
    run += v;
  }
  total[b] = run;
}

// step 3: exclusive scan of the bin totals (one block).
__global__ void k_scan_bins(const int32_t* total, int nbins, int32_t* start) {
  __shared__ int32_t part[1024];
  int per = (nbins + blockDim.x - 1) / blockDim.x;
  int lo = threadIdx.x * per, hi = min(nbins, lo + per);
  int32_t s = 0;
  for (int i = lo; i < hi; ++i) s += total[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      int32_t v = part[i];
      part[i] = run;
      run += v;
    }
  }
  __syncthreads();
  int32_t run = part[threadIdx.x];
  for (int i = lo; i < hi; ++i) {
    start[i] = run;
    run += total[i];
  }
  if (threadIdx.x == blockDim.x - 1) start[nbins] = run;
}

// step 4: scatter; the rank inside a chunk counts earlier samples of the same bin.
__global__ void k_chunk_scatter(const int32_t* __restrict__ key, int64_t M, int nbins,
                                const int32_t* __restrict__ counts, const int32_t* __restrict__ start,
                                int32_t* __restrict__ perm) {
  __shared__ int32_t sk[SORT_CHUNK];
  int64_t base = (int64_t)blockIdx.x * SORT_CHUNK;
  for (int i = threadIdx.x; i < SORT_CHUNK; i += blockDim.x) sk[i] = (base + i < M) ? key[base + i] : -1;
  __syncthreads();
  for (int i = threadIdx.x; i < SORT_CHUNK; i += blockDim.x) {
    if (base + i >= M) continue;
    int k = sk[i], r = 0;
    for (int j = 0; j < i; ++j) r += (sk[j] == k);
    perm[start[k] + counts[(int64_t)blockIdx.x * nbins + k] + r] = (int32_t)(base + i);
  }
}

// ---------------------------------------------------------------- 1D Voronoi weights
// bitonic sort of (xi, index) pairs padded to a power of two with +inf keys
__global__ void k_bitonic(double* key, int32_t* val, int64_t P, int64_t j, int64_t k) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= P) return;
  int64_t l = i ^ j;
  if (l <= i) return;
  bool up = (i & k) == 0;
  double a = key[i], b = key[l];
  bool swap = up ? (a > b || (a == b && val[i] > val[l])) : (a < b || (a == b && val[i] < val[l]));
  if (swap) {
    key[i] = b;
    key[l] = a;
    int32_t t = val[i];
    val[i] = val[l];
    val[l] = t;
  }
}

// Sec. 4.1: mu = length of the Voronoi cell [(x_{i-1}+x_i)/2, (x_i+x_{i+1})/2], the
// outer cells closed by [-K, K], all clipped to [-K, K].
__global__ void k_voronoi(const double* skey, const int32_t* sval, int64_t M, double K, double* mu) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  double lo = (i == 0) ? -K : 0.5 * (skey[i - 1] + skey[i]);
  double hi = (i == M - 1) ? K : 0.5 * (skey[i] + skey[i + 1]);
  lo = fmin(fmax(lo, -K), K);
  hi = fmin(fmax(hi, -K), K);
  mu[sval[i]] = hi - lo;
}

__global__ void k_gather_xi(const double* __restrict__ xi, const double* __restrict__ mu,
                            const int32_t* __restrict__ perm, int64_t M, int dims,
                            double* __restrict__ xs, double* __restrict__ ms) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= M) return;
  int32_t o = perm[s];
  for (int d = 0; d < dims; ++d) xs[d * M + s] = xi[d * M + o];
  ms[s] = mu ? mu[o] : 1.0;
}

__global__ void k_gather_fl(const int32_t* __restrict__ flo, const int32_t* __restrict__ perm,
                            int64_t M, int dims, int32_t* __restrict__ fls) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= M) return;
  for (int d = 0; d < dims; ++d) fls[d * M + s] = flo[d * M + perm[s]];
}

// ---------------------------------------------------------------- K1: factor tables
// One thread per (sample, dimension).
__global__ void k_tables(const double* __restrict__ xs, const double* __restrict__ ms, int64_t M,
                         int dims, int J, int p, int b, double mu1, double mu2, int64_t n,
                         double2* __restrict__ w64, double2* __restrict__ bf64, double* __restrict__ fr64,
                         float2* __restrict__ w32, float2* __restrict__ bf32, float* __restrict__ fr32,
                         int m32, double beta32, float* __restrict__ win32) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= M * dims) return;
  int d = (int)(g / M);
  int64_t s = g - (int64_t)d * M;
  double xi = xs[d * M + s];
  double eta = ldexp(xi, -J);
  double aeta = fabs(eta);
  int D = 30 + (aeta > 1.0 ? (int)ceil(log2(aeta)) : 0);
  double z = ldexp(eta, -D);
  // phi-hat(z), Taylor: 1 - 2 pi i mu1 z - 2 pi^2 mu2 z^2
  double2 ph = make_double2(1.0 - 2.0 * M_PI * M_PI * mu2 * z * z, -2.0 * M_PI * mu1 * z);
  double2 vL[GS_MAX_P], vR[GS_MAX_P];
  for (int k = 0; k < b; ++k) {
    vL[k] = make_double2(c_v0L[k], 0.0);
    vR[k] = make_double2(c_v0R[k], 0.0);
  }
  const int nv = 2 * p - 1;
  for (int l = D - 1; l >= 0; --l) {
    double e = ldexp(eta, -(l + 1));  // ph = phi-hat(e) here
    double sn, cs;
    sincospi(2.0 * e, &sn, &cs);
    double2 c = make_double2(cs, -sn);  // exp(-2 pi i e)
    // powers E[q] = c^q, q = 0..3p
    double2 E[3 * GS_MAX_P + 1];
    E[0] = make_double2(1.0, 0.0);
    for (int q = 1; q <= 3 * p; ++q) E[q] = cm(E[q - 1], c);
    if (b > 0) {
      double2 nL[GS_MAX_P], nR[GS_MAX_P];
      for (int k = 0; k < p; ++k) {
        double2 aL = make_double2(0.0, 0.0), aR = make_double2(0.0, 0.0);
        for (int j = 0; j < p; ++j) {
          double uL = c_UL[k * GS_MAX_P + j], uR = c_UR[k * GS_MAX_P + j];
          aL.x += uL * vL[j].x; aL.y += uL * vL[j].y;
          aR.x += uR * vR[j].x; aR.y += uR * vR[j].y;
        }
        for (int mi = 0; mi < nv; ++mi) {
          // left v2 = ph exp(-2 pi i m e), right v2 = ph exp(+2 pi i (m+1) e), m = p + mi
          double2 tL = cm(ph, E[p + mi]);
          double2 eR = E[p + mi + 1];
          double2 tR = cm(ph, make_double2(eR.x, -eR.y));
          double qL = c_VL[k * (2 * GS_MAX_P - 1) + mi], qR = c_VR[k * (2 * GS_MAX_P - 1) + mi];
          aL.x += qL * tL.x; aL.y += qL * tL.y;
          aR.x += qR * tR.x; aR.y += qR * tR.y;
        }
        nL[k] = aL;
        nR[k] = aR;
      }
      for (int k = 0; k < p; ++k) {
        vL[k] = nL[k];
        vR[k] = nR[k];
      }
    }
    // m0(e) = sum_{k=-p+1}^{p} h_k c^k = conj(c)^(p-1) sum_j h[j] c^j
    double2 m = make_double2(0.0, 0.0);
    for (int j = 0; j < 2 * p; ++j) {
      m.x += c_h[j] * E[j].x;
      m.y += c_h[j] * E[j].y;
    }
    double2 cinv = make_double2(E[p - 1].x, -E[p - 1].y);
    m = cm(m, cinv);
    ph = cm(m, ph);  // phi-hat(2e) = m0(e) phi-hat(e)
  }
  double sc = ldexp(1.0, 0) / sqrt(ldexp(1.0, J));
  if (d == 0) sc *= sqrt(ms[s]);
  double2 wv = make_double2(sc * ph.x, sc * ph.y);
  w64[d * M + s] = wv;
  w32[d * M + s] = make_float2((float)wv.x, (float)wv.y);
  if (b > 0) {
    double sn, cs;
    sincospi(xi, &sn, &cs);
    double2 pl = make_double2(sc * cs, sc * sn);   // sc exp(+pi i xi)
    double2 pr = make_double2(sc * cs, -sc * sn);  // sc exp(-pi i xi)
    int64_t base = ((int64_t)d * M + s) * (2 * b);
    for (int k = 0; k < b; ++k) {
      double2 L = cm(pl, vL[k]), R = cm(pr, vR[k]);
      bf64[base + k] = L;
      bf64[base + b + k] = R;
      bf32[base + k] = make_float2((float)L.x, (float)L.y);
      bf32[base + b + k] = make_float2((float)R.x, (float)R.y);
    }
  }
  // fractional grid coordinate
  double ew = eta - rint(eta);
  double u = ew * (double)n;
  double fr = u - floor(u);
  fr64[d * M + s] = fr;
  float f32 = (float)fr;
  if (f32 >= 1.0f) f32 = 0.99999994f;
  fr32[d * M + s] = f32;
  // float32 window values of the 2m taps, evaluated in float64 at the float64
  // coordinate: phi(dist) = sinh(beta sqrt(m^2 - dist^2)) / (pi sqrt(m^2 - dist^2))
  for (int a = 0; a < 2 * m32; ++a) {
    double dist = fr + (double)(m32 - 1 - a);
    double s2 = (double)(m32 * m32) - dist * dist;
    double v = (s2 <= 0.0) ? beta32 / M_PI : sinh(beta32 * sqrt(s2)) / (M_PI * sqrt(s2));
    win32[((int64_t)s * dims + d) * (2 * m32) + a] = (float)v;
  }
}

// deapodisation 1/psi(k), psi(k) = I0(m sqrt(beta^2 - (2 pi k/n)^2)), interior
// indices only (boundary indices get 0 so the NFFT ignores them)
// 1 / psi(k) of the interior coefficients (0 at the boundary indices); unit: 1
// instead (the exact lattice path has no window to divide out)
__global__ void k_deap(int64_t N, int b, int64_t n, int m, double beta, double* d64, float* d32,
                       int which, int unit) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double v = 0.0;
  if (unit) {
    v = (i >= b && i < N - b) ? 1.0 : 0.0;
  } else if (i >= b && i < N - b) {
    double k = (double)(i - N / 2);
    double a = 2.0 * M_PI * k / (double)n;
    double arg = (double)m * sqrt(beta * beta - a * a);
    v = 1.0 / cyl_bessel_i0(arg);
  }
  if (which == 0) d64[i] = v;
  else d32[i] = (float)v;
}

__global__ void k_twiddle(int64_t n, double2* t64, float2* t32) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n / 2) return;
  double sn, cs;
  sincospi(2.0 * (double)k / (double)n, &sn, &cs);
  t64[k] = make_double2(cs, -sn);
  t32[k] = make_float2((float)cs, (float)-sn);
}

template <typename T>
gs_status dalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    return GS_ENOMEM;
  }
  return GS_OK;
}

// float64 window values phi(frac + m - 1 - a) of the 2m taps of every sample and
// dimension, [s][d][a], by the same function the kernels use without a table
__global__ void k_win64(const double* __restrict__ frac, int64_t M, int dims, int m, double beta,
                        double* __restrict__ win) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= M * dims) return;
  const int d = (int)(g / M);
  const int64_t s = g - (int64_t)d * M;
  const double t = frac[g];
  double* out = win + (s * dims + d) * (2 * m);
  for (int a = 0; a < 2 * m; ++a) out[a] = dev::kb_window(t + (double)(m - 1 - a), m, beta);
}

template <typename R>
gs_status alloc_prec(Plan* P, PrecData<R>& D, int m) {
  D.m = m;
  D.beta = M_PI * (2.0 - 1.0 / (double)P->sigma);
  const int64_t M = P->M, n = P->n, N = P->N;
  const int dims = P->dims, b = P->b, b2 = 2 * b;
  GS_TRY(dalloc(&D.frac, (size_t)dims * M));
  // window values of every tap: float32 always; float64 while the table stays
  // within WIN64_BYTES (else the kernels evaluate the window per tap)
  if (sizeof(R) == 4 || (double)dims * M * 2 * m * sizeof(double) <= (double)WIN64_BYTES)
    GS_TRY(dalloc(&D.win, (size_t)dims * M * 2 * m));
  GS_TRY(dalloc(&D.w, (size_t)dims * M));
  GS_TRY(dalloc(&D.bf, (size_t)dims * M * (b2 > 0 ? b2 : 1)));
  GS_TRY(dalloc(&D.deap, (size_t)N));
  GS_TRY(dalloc(&D.tw, (size_t)(n / 2)));
  if (!P->direct) {
    if (dims == 1) {
      GS_TRY(dalloc(&D.grid, (size_t)n));
      if (n >= 4096) GS_TRY(dalloc(&D.ftmp, (size_t)n));
      D.part_stride = TILE1 + 2 * m + b2;
    } else {
      GS_TRY(dalloc(&D.grid, (size_t)n * n));
      GS_TRY(dalloc(&D.hbuf, (size_t)N * n));
      GS_TRY(dalloc(&D.side, (size_t)2 * (b2 > 0 ? b2 : 1) * n));
      GS_TRY(dalloc(&D.hs, (size_t)N * n));
      GS_TRY(dalloc(&D.hp, (size_t)N * n));
      if (P->lattice && b2 > 0)
        GS_TRY(dalloc(&D.lat, (size_t)P->nbins * 2 * b2 * P->tile));
      int pw = TILE2 + 2 * m;
      D.part_stride = (int64_t)pw * pw + 2 * b2 * pw + b2 * b2;
    }
  }
  GS_TRY(dalloc(&D.corner, (size_t)(b2 * b2 > 0 ? b2 * b2 : 1)));
  GS_TRY(dalloc(&D.vx, (size_t)P->ncoef));
  GS_TRY(dalloc(&D.vs, (size_t)P->ncoef));
  GS_TRY(dalloc(&D.vp, (size_t)P->ncoef));
  GS_TRY(dalloc(&D.vr, (size_t)M));
  GS_TRY(dalloc(&D.vq, (size_t)M));
  GS_TRY(dalloc(&D.vz, (size_t)P->ncoef));
  return GS_OK;
}

}  // namespace

template <typename R>
static gs_status grow_part(PrecData<R>& D, int nwork) {
  if (D.part) cudaFree(D.part);
  D.part = nullptr;
  return dalloc(&D.part, (size_t)nwork * D.part_stride);
}

gs_status set_work(Plan* P, int chunk, cudaStream_t st) {
  if (chunk < 1) {
    set_error("work item size %d < 1", chunk);
    return GS_EINVAL;
  }
  const std::vector<int32_t>& hstart = P->bin_start_h;
  // a bin of c samples gives ceil(c / chunk) items of near-equal size, so that
  // no item is much smaller than its siblings (600 at chunk 512: 300 + 300)
  std::vector<int32_t> work, wstart(P->nbins + 1);
  for (int bn = 0; bn < P->nbins; ++bn) {
    wstart[bn] = (int32_t)(work.size() / 3);
    const int64_t s0 = hstart[bn], c = hstart[bn + 1] - s0;
    const int64_t k = (c + chunk - 1) / chunk;
    for (int64_t i = 0; i < k; ++i) {
      work.push_back(bn);
      work.push_back((int32_t)(s0 + c * i / k));
      work.push_back((int32_t)(s0 + c * (i + 1) / k));
    }
  }
  wstart[P->nbins] = (int32_t)(work.size() / 3);
  void* old[] = {P->work, P->work_start, P->work_order, P->wcol, P->wcol_start};
  GS_CUDA(cudaStreamSynchronize(st));
  for (void* p : old)
    if (p) cudaFree(p);
  P->work = P->work_start = P->work_order = P->wcol = P->wcol_start = nullptr;
  P->nwork = (int)(work.size() / 3);
  P->chunk = chunk;
  GS_TRY(dalloc(&P->work, work.size() > 0 ? work.size() : 3));
  GS_TRY(dalloc(&P->work_start, wstart.size()));
  if (!work.empty())
    GS_CUDA(cudaMemcpyAsync(P->work, work.data(), work.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemcpyAsync(P->work_start, wstart.data(), wstart.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice, st));
  // launch order: larger items first, so that the last wave holds the short ones
  std::vector<int32_t> order(P->nwork);
  for (int i = 0; i < P->nwork; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return work[3 * a + 2] - work[3 * a + 1] > work[3 * b + 2] - work[3 * b + 1];
  });
  GS_TRY(dalloc(&P->work_order, order.size() > 0 ? order.size() : 1));
  if (!order.empty())
    GS_CUDA(cudaMemcpyAsync(P->work_order, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                            st));
  // the same work items grouped by bin column (for reductions along x)
  std::vector<int32_t> wcol, wcs(P->nbx + 1);
  for (int bx = 0; bx < P->nbx; ++bx) {
    wcs[bx] = (int32_t)wcol.size();
    for (int by = 0; by < P->nby; ++by)
      for (int32_t wi = wstart[by * P->nbx + bx]; wi < wstart[by * P->nbx + bx + 1]; ++wi) wcol.push_back(wi);
  }
  wcs[P->nbx] = (int32_t)wcol.size();
  GS_TRY(dalloc(&P->wcol, wcol.size() > 0 ? wcol.size() : 1));
  GS_TRY(dalloc(&P->wcol_start, wcs.size()));
  if (!wcol.empty())
    GS_CUDA(cudaMemcpyAsync(P->wcol, wcol.data(), wcol.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemcpyAsync(P->wcol_start, wcs.data(), wcs.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  // per-item partial sums of the spread, and the reduction partials (per work
  // item or 512 blocks, then up to 1184 blocks)
  if (P->nwork > P->work_cap || !P->red) {
    const int cap = std::max(P->nwork, 1);
    if (!P->direct) {
      GS_TRY(grow_part(P->d, cap));
      GS_TRY(grow_part(P->f, cap));
    }
    if (P->red) cudaFree(P->red);
    P->red = nullptr;
    GS_TRY(dalloc(&P->red, (size_t)std::max(8192, cap + 2048)));
    P->work_cap = cap;
  }
  GS_CUDA(cudaStreamSynchronize(st));
  return GS_OK;
}

gs_status build_plan(Plan* P, const double* xi_host, const double* mu_host, cudaStream_t st) {
  const int64_t M = P->M;
  const int dims = P->dims;
  const int T = (dims == 1) ? TILE1 : TILE2;
  P->tile = T;
  P->tile = (int)std::min<int64_t>(T, P->n);
  P->nbx = (int)(P->n / P->tile);
  P->nby = (dims == 2) ? P->nbx : 1;
  P->nbins = P->nbx * P->nby;

  // constants to the GPU
  const Constants& K = P->k;
  double UL[GS_MAX_P * GS_MAX_P] = {0}, UR[GS_MAX_P * GS_MAX_P] = {0};
  double VL[GS_MAX_P * (2 * GS_MAX_P - 1)] = {0}, VR[GS_MAX_P * (2 * GS_MAX_P - 1)] = {0};
  for (int i = 0; i < GS_MAX_P; ++i)
    for (int j = 0; j < GS_MAX_P; ++j) {
      UL[i * GS_MAX_P + j] = K.left.U[i][j];
      UR[i * GS_MAX_P + j] = K.right.U[i][j];
    }
  for (int i = 0; i < GS_MAX_P; ++i)
    for (int j = 0; j < 2 * GS_MAX_P - 1; ++j) {
      VL[i * (2 * GS_MAX_P - 1) + j] = K.left.V[i][j];
      VR[i * (2 * GS_MAX_P - 1) + j] = K.right.V[i][j];
    }
  GS_CUDA(cudaMemcpyToSymbolAsync(c_h, K.h, sizeof(K.h), 0, cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemcpyToSymbolAsync(c_UL, UL, sizeof(UL), 0, cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemcpyToSymbolAsync(c_UR, UR, sizeof(UR), 0, cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemcpyToSymbolAsync(c_VL, VL, sizeof(VL), 0, cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemcpyToSymbolAsync(c_VR, VR, sizeof(VR), 0, cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemcpyToSymbolAsync(c_v0L, K.left.v10, sizeof(K.left.v10), 0, cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemcpyToSymbolAsync(c_v0R, K.right.v10, sizeof(K.right.v10), 0, cudaMemcpyHostToDevice, st));

  // upload xi (dimension-major) and weights
  std::vector<double> xd((size_t)dims * M);
  for (int64_t s = 0; s < M; ++s)
    for (int d = 0; d < dims; ++d) xd[(size_t)d * M + s] = xi_host[s * dims + d];
  double *xi_d = nullptr, *mu_d = nullptr, *ms = nullptr;
  int32_t *fl_o = nullptr, *key = nullptr, *counts = nullptr, *total = nullptr;
  GS_TRY(dalloc(&xi_d, xd.size()));
  GS_CUDA(cudaMemcpyAsync(xi_d, xd.data(), xd.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  if (mu_host) {
    GS_TRY(dalloc(&mu_d, (size_t)M));
    GS_CUDA(cudaMemcpyAsync(mu_d, mu_host, M * sizeof(double), cudaMemcpyHostToDevice, st));
  } else if (P->bandwidth > 0 && dims == 1) {
    int64_t Pp = 1;
    while (Pp < M) Pp <<= 1;
    double* skey;
    int32_t* sval;
    GS_TRY(dalloc(&skey, (size_t)Pp));
    GS_TRY(dalloc(&sval, (size_t)Pp));
    std::vector<double> hk(Pp, INFINITY);
    std::vector<int32_t> hv(Pp);
    for (int64_t i = 0; i < Pp; ++i) hv[i] = (int32_t)i;
    for (int64_t i = 0; i < M; ++i) hk[i] = xi_host[i];
    GS_CUDA(cudaMemcpyAsync(skey, hk.data(), Pp * sizeof(double), cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemcpyAsync(sval, hv.data(), Pp * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    int thr = 256;
    int64_t blk = (Pp + thr - 1) / thr;
    for (int64_t k = 2; k <= Pp; k <<= 1)
      for (int64_t j = k >> 1; j > 0; j >>= 1) k_bitonic<<<blk, thr, 0, st>>>(skey, sval, Pp, j, k);
    GS_TRY(dalloc(&mu_d, (size_t)M));
    k_voronoi<<<(M + 255) / 256, 256, 0, st>>>(skey, sval, M, P->bandwidth, mu_d);
    GS_CUDA(cudaGetLastError());
    GS_CUDA(cudaStreamSynchronize(st));
    cudaFree(skey);
    cudaFree(sval);
  }

  // coordinates and stable counting sort by tile
  GS_TRY(dalloc(&fl_o, (size_t)dims * M));
  GS_TRY(dalloc(&key, (size_t)M));
  GS_TRY(dalloc(&P->perm, (size_t)M));
  GS_TRY(dalloc(&P->fl, (size_t)dims * M));
  GS_TRY(dalloc(&P->xi_sorted, (size_t)dims * M));
  GS_TRY(dalloc(&ms, (size_t)M));
  GS_TRY(dalloc(&P->bin_start, (size_t)P->nbins + 1));
  const int nchunks = (int)((M + SORT_CHUNK - 1) / SORT_CHUNK);
  GS_TRY(dalloc(&counts, (size_t)nchunks * P->nbins));
  GS_TRY(dalloc(&total, (size_t)P->nbins));
  k_coords<<<(M + 255) / 256, 256, 0, st>>>(xi_d, M, dims, P->J, P->n, P->tile, P->nbx, fl_o, key);
  size_t shb = (size_t)P->nbins * sizeof(int32_t);
  if (shb > 48 * 1024) GS_CUDA(cudaFuncSetAttribute(k_chunk_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb));
  k_chunk_hist<<<nchunks, 256, shb, st>>>(key, M, P->nbins, counts);
  k_scan_chunks<<<(P->nbins + 255) / 256, 256, 0, st>>>(counts, nchunks, P->nbins, total);
  k_scan_bins<<<1, 1024, 0, st>>>(total, P->nbins, P->bin_start);
  k_chunk_scatter<<<nchunks, 256, 0, st>>>(key, M, P->nbins, counts, P->bin_start, P->perm);
  k_gather_xi<<<(M + 255) / 256, 256, 0, st>>>(xi_d, mu_d, P->perm, M, dims, P->xi_sorted, ms);
  k_gather_fl<<<(M + 255) / 256, 256, 0, st>>>(fl_o, P->perm, M, dims, P->fl);
  GS_CUDA(cudaGetLastError());

  // work items: each bin's sample range split into chunks (set_work)
  P->bin_start_h.assign(P->nbins + 1, 0);
  GS_CUDA(cudaMemcpyAsync(P->bin_start_h.data(), P->bin_start, (P->nbins + 1) * sizeof(int32_t),
                          cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));

  // per-precision tables and workspaces
  GS_TRY(alloc_prec(P, P->d, P->m_hi));
  GS_TRY(alloc_prec(P, P->f, P->m_lo));
  int64_t tot = M * dims;
  k_tables<<<(tot + 127) / 128, 128, 0, st>>>(P->xi_sorted, ms, M, dims, P->J, P->p, P->b, K.mu1, K.mu2,
                                             P->n, P->d.w, P->d.bf, P->d.frac, P->f.w, P->f.bf, P->f.frac,
                                             P->f.m, P->f.beta, P->f.win);
  if (P->d.win)
    k_win64<<<(tot + 127) / 128, 128, 0, st>>>(P->d.frac, M, dims, P->d.m, P->d.beta, P->d.win);
  k_deap<<<(P->N + 255) / 256, 256, 0, st>>>(P->N, P->b, P->n, P->d.m, P->d.beta, P->d.deap, nullptr, 0,
                                             P->lattice);
  k_deap<<<(P->N + 255) / 256, 256, 0, st>>>(P->N, P->b, P->n, P->f.m, P->f.beta, nullptr, P->f.deap, 1,
                                             P->lattice);
  k_twiddle<<<(P->n / 2 + 255) / 256, 256, 0, st>>>(P->n, P->d.tw, P->f.tw);
  GS_CUDA(cudaGetLastError());

  GS_TRY(set_work(P, P->chunk > 0 ? P->chunk : (dims == 1 ? CHUNK1 : CHUNK2), st));
  GS_TRY(dalloc(&P->scal, 64));
  GS_TRY(dalloc(&P->flag, 16));
  GS_CUDA(cudaMemsetAsync(P->flag, 0, 16 * sizeof(int), st));
  GS_TRY(dalloc(&P->y64, (size_t)2 * M));
  GS_TRY(dalloc(&P->r64, (size_t)2 * M));
  GS_TRY(dalloc(&P->x64, (size_t)2 * P->ncoef));
  GS_CUDA(cudaStreamSynchronize(st));
  cudaFree(xi_d);
  if (mu_d) cudaFree(mu_d);
  cudaFree(ms);
  cudaFree(fl_o);
  cudaFree(key);
  cudaFree(counts);
  cudaFree(total);
  return GS_OK;
}

}  // namespace gs
