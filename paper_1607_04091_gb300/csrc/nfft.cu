// T x and T^H y through the Kaiser-Bessel NFFT plus the boundary factors.
//
// Sec. 4: T = [L I R] with I = D F, F the NDFT of eq. NDFT_def on the wrapped
// frequencies eta' = xi/2^J - round(xi/2^J); Sec. 3.2 / NFFT.jl approximate F x
// by an NFFT.  Here (window of Kaiser 1974 as used by Keiner-Kunis-Potts):
//   grid n = sigma N, beta = pi (2 - 1/sigma), half-width m,
//   g_l   = sum_k c_k / psi(k) exp(-2 pi i k l / n),   psi(k) = I0(m sqrt(beta^2 - (2 pi k/n)^2)),
//   F c (eta') ~= sum_{|u - l| < m} g_l phi(u - l),   u = n eta',
//   phi(d) = sinh(beta sqrt(m^2 - d^2)) / (pi sqrt(m^2 - d^2)).
// The adjoint is the exact transpose: spread with the same window, inverse DFT,
// divide by psi.  2D (Sec. 5, App. C): separable window and deapodisation;
// interior x interior through a 2D grid, sides (boundary x interior) through 1D
// grids of the boundary rows / columns, corners directly.
//
// Data layout on the device (per precision R):
//   grid  [lx][ly]     n x n (2D) or n (1D) oversampled grid
//   hbuf  [j][lx]      N x n: x-transform of every coefficient row j (2D)
//   side  [2][2b][n]   forward: x-side grids along y; adjoint: both side grids
//   part  per spread work item: padded tile, side segments, corner sums
// The grid size n = sigma 2^J and the bin count n / tile are powers of two, so
// periodic indices wrap with the mask n - 1.
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "gs_internal.h"
#include "device_common.cuh"

namespace gs {

namespace {
using namespace dev;

// ---------------------------------------------------------------- shared-memory FFT
// In-place DFT of nb rows of length n (a power of two) held contiguously in
// shared memory: F[q] = sum_l f[l] e^{-+2 pi i l q / n} (+ for the inverse, no
// scaling), natural order in and out.  Stockham's autosort form with radix-8
// passes and, for the remaining factor, one radix-4 or radix-2 pass: the pass of
// radix R after sub-transforms of length Ns (Ns = product of the earlier radices)
// reads f[j + r n/R], r < R, multiplies by e^{-+2 pi i r (j mod Ns) / (Ns R)},
// takes the R-point DFT in registers and writes it to (j div Ns) Ns R + (j mod Ns)
// + r Ns.  Every thread holds PPT points per pass (the caller launches at least
// nb n / PPT threads); a pass is load, barrier, compute and store, barrier.
// Twiddles: the base e^{-+2 pi i (j mod Ns) / (Ns R)} from the plan's table
// tw[k tws] = e^{-2 pi i k / n}, k < n/2, and its powers by multiplication.
template <typename R> __device__ inline C<R> csub(C<R> a, C<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
// a (-i), or a i for the inverse
template <typename R> __device__ inline C<R> rot_q(C<R> a, bool inv) { return inv ? mk<R>(-a.y, a.x) : mk<R>(a.y, -a.x); }

template <typename R> __device__ inline void dft_reg2(C<R>* v, bool) {
  const C<R> a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub<R>(a, b);
}
template <typename R> __device__ inline void dft4(C<R>& v0, C<R>& v1, C<R>& v2, C<R>& v3, bool inv) {
  const C<R> a0 = cadd(v0, v2), a1 = csub<R>(v0, v2), a2 = cadd(v1, v3), w = rot_q<R>(csub<R>(v1, v3), inv);
  v0 = cadd(a0, a2);
  v2 = csub<R>(a0, a2);
  v1 = cadd(a1, w);
  v3 = csub<R>(a1, w);
}
template <typename R> __device__ inline void dft_reg4(C<R>* v, bool inv) { dft4<R>(v[0], v[1], v[2], v[3], inv); }
// 8 points: two 4-point DFTs of the even and odd samples, combined with e^{-+i pi q/4}
template <typename R> __device__ inline void dft_reg8(C<R>* v, bool inv) {
  C<R> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<R>(e0, e1, e2, e3, inv);
  dft4<R>(o0, o1, o2, o3, inv);
  const R h = (R)0.70710678118654752440;  // 1/sqrt(2)
  const C<R> t1 = inv ? mk<R>((o1.x - o1.y) * h, (o1.x + o1.y) * h) : mk<R>((o1.x + o1.y) * h, (o1.y - o1.x) * h);
  const C<R> t2 = rot_q<R>(o2, inv);
  const C<R> t3 = inv ? mk<R>((-o3.x - o3.y) * h, (o3.x - o3.y) * h) : mk<R>((o3.y - o3.x) * h, (-o3.x - o3.y) * h);
  v[0] = cadd(e0, o0);
  v[4] = csub<R>(e0, o0);
  v[1] = cadd(e1, t1);
  v[5] = csub<R>(e1, t1);
  v[2] = cadd(e2, t2);
  v[6] = csub<R>(e2, t2);
  v[3] = cadd(e3, t3);
  v[7] = csub<R>(e3, t3);
}
template <typename R, int RAD> __device__ inline void dft_reg(C<R>* v, bool inv) {
  if constexpr (RAD == 8) dft_reg8<R>(v, inv);
  else if constexpr (RAD == 4) dft_reg4<R>(v, inv);
  else dft_reg2<R>(v, inv);
}

// one pass: radix RAD = 2^lr, n / RAD = 2^lgq butterflies per row, Ns = 2^lgNs
template <typename R, int RAD, int PPT>
__device__ inline void fft_pass(C<R>* buf, int nb, int n, int lgq, int lgNs, const C<R>* __restrict__ tw, int tws,
                                bool inv) {
  constexpr int NB = PPT / RAD;  // butterflies per thread
  constexpr int lr = (RAD == 8) ? 3 : (RAD == 4) ? 2 : 1;
  const int q = 1 << lgq, Ns = 1 << lgNs;
  const int nbf = nb << lgq;
  C<R> v[NB][RAD];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int bi = threadIdx.x + k * blockDim.x;
    if (bi < nbf) {
      const C<R>* src = buf + (bi >> lgq) * n + (bi & (q - 1));
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[k][r] = src[r * q];
    }
  }
  // base twiddle e^{-+2 pi i jm / (Ns RAD)} = table entry jm (n / (Ns RAD)) tws (below n tws / 2);
  // it does not depend on the data, so its load overlaps the barrier
  C<R> wb[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int bi = threadIdx.x + k * blockDim.x;
    wb[k] = mk<R>(1, 0);
    if (bi < nbf && lgNs > 0) {
      const int jm = (bi & (q - 1)) & (Ns - 1);
      wb[k] = tw[(jm << (lgq - lgNs)) * tws];
      if (inv) wb[k].y = -wb[k].y;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int bi = threadIdx.x + k * blockDim.x;
    if (bi < nbf) {
      const int row = bi >> lgq, j = bi & (q - 1), jm = j & (Ns - 1);
      if (lgNs > 0) {  // twiddle r = base^r (rounding error <= r ulp)
        C<R> w = wb[k];
        v[k][1] = cmul(v[k][1], w);
#pragma unroll
        for (int r = 2; r < RAD; ++r) {
          w = cmul(w, wb[k]);
          v[k][r] = cmul(v[k][r], w);
        }
      }
      dft_reg<R, RAD>(v[k], inv);
      C<R>* dst = buf + row * n + ((j >> lgNs) << (lgNs + lr)) + jm;
#pragma unroll
      for (int r = 0; r < RAD; ++r) dst[r * Ns] = v[k][r];
    }
  }
  __syncthreads();
}

template <typename R, int PPT>
__device__ void fft_smem(C<R>* buf, int nb, int n, int logn, const C<R>* __restrict__ tw, bool inverse, int tws = 1) {
  int lgNs = 0;
  while (lgNs < logn) {
    const int left = logn - lgNs;
    if (left >= 3) {
      fft_pass<R, 8, PPT>(buf, nb, n, logn - 3, lgNs, tw, tws, inverse);
      lgNs += 3;
    } else if (left == 2) {
      fft_pass<R, 4, PPT>(buf, nb, n, logn - 2, lgNs, tw, tws, inverse);
      lgNs += 2;
    } else {
      fft_pass<R, 2, PPT>(buf, nb, n, logn - 1, lgNs, tw, tws, inverse);
      lgNs += 1;
    }
  }
}
constexpr int PPT_ROW = 8;  // points per thread and pass
// threads of an FFT CTA: PPT_ROW points each for its nb rows of length n (at most
// 1024 threads: n <= 8192 per CTA, which covers the single-CTA 1D transforms,
// n < FOUR_STEP_N, the four-step rows and the 2D passes, n <= 1024)
inline int fft_threads(int nb, int n) {
  const int t = ((nb * n / PPT_ROW + 31) / 32) * 32;
  return t < 64 ? 64 : (t > 1024 ? 1024 : t);
}

// the adjoint's last pass also updates a coefficient row per CTA in the CG solver:
// at least 128 threads
inline int adj1_threads(int nb, int n) { return std::max(128, fft_threads(nb, n)); }

// for t = threadIdx.x, + blockDim.x, ... < total: v = load(t), then store(t, v), in
// groups of LB per thread whose loads are all issued before the group's stores
// (the pass kernels have few warps, so memory latency is hidden by batching)
template <typename R> struct Cv {  // a value and whether to store it
  C<R> v;
  bool ok;
};
template <int LB, typename T, typename L, typename S>
__device__ inline void batched(int total, L load, S store) {
  for (int base = threadIdx.x; base < total; base += LB * blockDim.x) {
    T v[LB];
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int t = base + u * blockDim.x;
      if (t < total) v[u] = load(t);
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int t = base + u * blockDim.x;
      if (t < total) store(t, v[u]);
    }
  }
}

// The n/2 twiddles of a 2D pass into shared memory: fetched into registers
// before the pass issues its row or column loads and stored after them, so that
// both share one round trip; the radix passes then read their twiddles from
// shared memory instead of waiting on a global load before each barrier.
template <typename R> struct TwStage {
  C<R> v[4];
  __device__ inline void fetch(const C<R>* __restrict__ tw, int nh) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = threadIdx.x + u * blockDim.x;
      if (i < nh) v[u] = tw[i];
    }
  }
  __device__ inline void store(const C<R>* __restrict__ tw, C<R>* tws, int nh) const {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = threadIdx.x + u * blockDim.x;
      if (i < nh) tws[i] = v[u];
    }
    for (int i = threadIdx.x + 4 * blockDim.x; i < nh; i += blockDim.x) tws[i] = tw[i];
  }
};

// ---------------------------------------------------------------- 1D forward
// deapodise + zero-pad + FFT: one CTA, n <= 16384 (float) / 8192 (double)
template <typename R>
__global__ void k_fwd1d_fft(const C<R>* __restrict__ x, const R* __restrict__ deap, int64_t N, int n,
                            int logn, const C<R>* __restrict__ tw, C<R>* __restrict__ grid) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C<R>* buf = reinterpret_cast<C<R>*>(smraw);
  for (int i = threadIdx.x; i < n; i += blockDim.x) buf[i] = mk<R>(0, 0);
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    R dv = deap[i];
    if (dv != (R)0) {
      int idx = (int)((i - N / 2) & (n - 1));
      buf[idx] = cscale(x[i], dv);
    }
  }
  __syncthreads();
  fft_smem<R, PPT_ROW>(buf, 1, n, logn, tw, false);
  for (int i = threadIdx.x; i < n; i += blockDim.x) grid[i] = buf[i];
}

// ---------------------------------------------------------------- 1D four-step FFT (large n)
// n = n1 n2, l = j1 + n1 j2, l' = k2 + n2 k1:
//   G[l'] = sum_j1 e^{-2 pi i j1 k1/n1} [ e^{-2 pi i j1 k2/n} sum_j2 a[j1 + n1 j2] e^{-2 pi i j2 k2/n2} ]
// tw holds e^{-2 pi i k/n}, k < n/2 (sub-FFTs of length L use stride n/L).
template <typename R>
__device__ inline C<R> tw_full(const C<R>* tw, int64_t k, int64_t n, bool inverse) {
  k %= n;
  C<R> w = (k < n / 2) ? tw[k] : tw[k - n / 2];
  if (k >= n / 2) {
    w.x = -w.x;
    w.y = -w.y;
  }
  if (inverse) w.y = -w.y;
  return w;
}

// forward step 1: CTA per j1; deapodised, zero-padded input column -> B[j1][k2]
template <typename R>
__global__ void k_fwd1d_cols(const C<R>* __restrict__ x, const R* __restrict__ deap, int64_t N, int n, int n1,
                             int n2, int logn2, const C<R>* __restrict__ tw, C<R>* __restrict__ B) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C<R>* buf = reinterpret_cast<C<R>*>(smraw);
  const int j1 = blockIdx.x;
  for (int j2 = threadIdx.x; j2 < n2; j2 += blockDim.x) {
    const int l = j1 + n1 * j2;
    const int64_t k = (l < n / 2) ? l : (int64_t)l - n;
    const int64_t i = k + N / 2;
    C<R> v = mk<R>(0, 0);
    if (i >= 0 && i < N) {
      const R dv = deap[i];
      if (dv != (R)0) v = cscale(x[i], dv);
    }
    buf[j2] = v;
  }
  __syncthreads();
  fft_smem<R, PPT_ROW>(buf, 1, n2, logn2, tw, false, n / n2);
  for (int k2 = threadIdx.x; k2 < n2; k2 += blockDim.x)
    B[(int64_t)j1 * n2 + k2] = cmul(buf[k2], tw_full<R>(tw, (int64_t)j1 * k2, n, false));
}

// forward step 2: CTA per k2; FFT over j1 -> grid[k2 + n2 k1]
template <typename R>
__global__ void k_fwd1d_rows(const C<R>* __restrict__ B, int n, int n1, int logn1, int n2,
                             const C<R>* __restrict__ tw, C<R>* __restrict__ grid) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C<R>* buf = reinterpret_cast<C<R>*>(smraw);
  const int k2 = blockIdx.x;
  for (int j1 = threadIdx.x; j1 < n1; j1 += blockDim.x) buf[j1] = B[(int64_t)j1 * n2 + k2];
  __syncthreads();
  fft_smem<R, PPT_ROW>(buf, 1, n1, logn1, tw, false, n / n1);
  for (int k1 = threadIdx.x; k1 < n1; k1 += blockDim.x) grid[k2 + (int64_t)n2 * k1] = buf[k1];
}

// adjoint step 1: CTA per k2; inverse FFT over k1 of grid[k2 + n2 k1], twiddle -> Cb[k2][j1]
template <typename R>
__global__ void k_adj1d_rows(const C<R>* __restrict__ grid, int n, int n1, int logn1, int n2,
                             const C<R>* __restrict__ tw, C<R>* __restrict__ Cb) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C<R>* buf = reinterpret_cast<C<R>*>(smraw);
  const int k2 = blockIdx.x;
  for (int k1 = threadIdx.x; k1 < n1; k1 += blockDim.x) buf[k1] = grid[k2 + (int64_t)n2 * k1];
  __syncthreads();
  fft_smem<R, PPT_ROW>(buf, 1, n1, logn1, tw, true, n / n1);
  for (int j1 = threadIdx.x; j1 < n1; j1 += blockDim.x)
    Cb[(int64_t)k2 * n1 + j1] = cmul(buf[j1], tw_full<R>(tw, (int64_t)j1 * k2, n, true));
}

// adjoint step 2: CTA per j1; inverse FFT over k2 -> z at l = j1 + n1 j2, cropped and
// deapodised; boundary coefficients from the channel sums
template <typename R>
__global__ void k_adj1d_cols(const C<R>* __restrict__ Cb, const R* __restrict__ deap, int64_t N, int n, int n1,
                             int n2, int logn2, const C<R>* __restrict__ tw, const C<R>* __restrict__ bsum, int b,
                             C<R>* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C<R>* buf = reinterpret_cast<C<R>*>(smraw);
  const int j1 = blockIdx.x;
  for (int k2 = threadIdx.x; k2 < n2; k2 += blockDim.x) buf[k2] = Cb[(int64_t)k2 * n1 + j1];
  __syncthreads();
  fft_smem<R, PPT_ROW>(buf, 1, n2, logn2, tw, true, n / n2);
  for (int j2 = threadIdx.x; j2 < n2; j2 += blockDim.x) {
    const int l = j1 + n1 * j2;
    const int64_t k = (l < n / 2) ? l : (int64_t)l - n;
    const int64_t i = k + N / 2;
    if (i < 0 || i >= N) continue;
    if (i >= b && i < N - b) z[i] = cscale(buf[j2], deap[i]);
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < 2 * b; i += blockDim.x) z[i < b ? i : N - 1 - (i - b)] = bsum[i];
}

// KB interpolation + weights + boundary block, one thread per sorted sample
template <typename R>
__global__ void k_interp1d(const int32_t* __restrict__ fl, const R* __restrict__ frac,
                           const C<R>* __restrict__ w, const C<R>* __restrict__ bf, int b,
                           const C<R>* __restrict__ grid, int n, int m, R beta,
                           const C<R>* __restrict__ x, int64_t N, int64_t M,
                           const int32_t* __restrict__ perm, C<R>* __restrict__ y) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= M) return;
  int f = fl[s];
  R t = frac[s];
  C<R> v = mk<R>(0, 0);
  for (int a = 0; a < 2 * m; ++a) {
    int l = f - m + 1 + a;
    l &= n - 1;
    R d = t + (R)(m - 1 - a);
    R wv = kb_window(d, m, beta);
    C<R> g = grid[l];
    v.x += wv * g.x;
    v.y += wv * g.y;
  }
  C<R> out = cmul(w[s], v);
  for (int k = 0; k < b; ++k) {
    out = cadd(out, cmul(bf[s * 2 * b + k], x[k]));
    out = cadd(out, cmul(bf[s * 2 * b + b + k], x[N - 1 - k]));
  }
  y[perm ? perm[s] : s] = out;
}

// ---------------------------------------------------------------- 1D adjoint
// CTA per work item; one warp per sample at a time, lanes over the taps, each
// warp with a private padded tile (no atomics, fixed summation order).
template <typename R>
__global__ void k_spread1d(const int32_t* __restrict__ work, const int32_t* __restrict__ fl,
                           const R* __restrict__ frac, const C<R>* __restrict__ w,
                           const C<R>* __restrict__ bf, int b, const C<R>* __restrict__ u,
                           const int32_t* __restrict__ perm, int tile, int m, R beta,
                           C<R>* __restrict__ part, int64_t stride) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C<R>* tiles = reinterpret_cast<C<R>*>(smraw);
  const int PW = tile + 2 * m;
  const int nw = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  C<R>* my = tiles + wid * (PW + 2 * b);
  for (int i = lane; i < PW + 2 * b; i += 32) my[i] = mk<R>(0, 0);
  __syncwarp();
  const int bin = work[3 * blockIdx.x], s0 = work[3 * blockIdx.x + 1], s1 = work[3 * blockIdx.x + 2];
  const int ox = bin * tile;
  for (int s = s0 + wid; s < s1; s += nw) {
    C<R> us = u[perm ? perm[s] : s];
    C<R> val = cmulc(us, w[s]);
    int base = fl[s] - ox + 1;  // padded index of tap 0
    R t = frac[s];
    for (int a = lane; a < 2 * m; a += 32) {
      R wv = kb_window(t + (R)(m - 1 - a), m, beta);
      C<R> c = my[base + a];
      c.x += wv * val.x;
      c.y += wv * val.y;
      my[base + a] = c;
    }
    for (int k = lane; k < 2 * b; k += 32) my[PW + k] = cadd(my[PW + k], cmulc(us, bf[(int64_t)s * 2 * b + k]));
    __syncwarp();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < PW + 2 * b; i += blockDim.x) {
    C<R> acc = mk<R>(0, 0);
    for (int q = 0; q < nw; ++q) acc = cadd(acc, tiles[q * (PW + 2 * b) + i]);
    part[blockIdx.x * stride + i] = acc;
  }
}

// grid point gx: sum of all padded tiles that cover it (neighbour bins, wrap)
template <typename R>
__global__ void k_reduce1d(const int32_t* __restrict__ work_start, const C<R>* __restrict__ part,
                           int64_t stride, int nbx, int tile, int m, int n, C<R>* __restrict__ grid) {
  int gx = blockIdx.x * blockDim.x + threadIdx.x;
  if (gx >= n) return;
  const int bx = gx / tile, PW = tile + 2 * m;
  int cand[3], nc = 0;
  for (int dx = -1; dx <= 1; ++dx) {
    int nb = (bx + dx) & (nbx - 1);
    bool dup = false;
    for (int q = 0; q < nc; ++q) dup |= (cand[q] == nb);
    if (!dup) cand[nc++] = nb;
  }
  C<R> acc = mk<R>(0, 0);
  for (int c = 0; c < nc; ++c) {
    int nb = cand[c];
    int q0 = (gx - nb * tile + m) & (n - 1);
    for (int wi = work_start[nb]; wi < work_start[nb + 1]; ++wi)
      for (int q = q0; q < PW; q += n) acc = cadd(acc, part[wi * stride + q]);
  }
  grid[gx] = acc;
}

// boundary (or corner) channel sums over all work items: one CTA per channel,
// threads stride over the work items, fixed-order tree sum
template <typename R>
__device__ __forceinline__ void reduce_chan_one(int c, const C<R>* __restrict__ part, int64_t stride, int64_t off,
                                                int nwork, C<R>* __restrict__ out) {
  __shared__ C<R> red[256];
  C<R> acc = mk<R>(0, 0);
  for (int wi = threadIdx.x; wi < nwork; wi += blockDim.x) acc = cadd(acc, part[wi * stride + off + c]);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}
template <typename R>
__global__ void k_reduce_chan(const C<R>* __restrict__ part, int64_t stride, int64_t off, int nch,
                              int nwork, C<R>* __restrict__ out) {
  reduce_chan_one<R>(blockIdx.x, part, stride, off, nwork, out);
}

// inverse FFT + crop + deapodise + boundary adjoint
template <typename R>
__global__ void k_adj1d_fft(const C<R>* __restrict__ grid, const R* __restrict__ deap, int64_t N, int n,
                            int logn, const C<R>* __restrict__ tw, const C<R>* __restrict__ bsum, int b,
                            C<R>* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C<R>* buf = reinterpret_cast<C<R>*>(smraw);
  for (int i = threadIdx.x; i < n; i += blockDim.x) buf[i] = grid[i];
  __syncthreads();
  fft_smem<R, PPT_ROW>(buf, 1, n, logn, tw, true);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    C<R> v;
    if (i < b) v = bsum[i];
    else if (i >= N - b) v = bsum[b + (N - 1 - i)];
    else v = cscale(buf[(i - N / 2) & (n - 1)], deap[i]);
    z[i] = v;
  }
}

// ---------------------------------------------------------------- 2D forward
// pass 1: x-transform of every coefficient row j -> hbuf[j][:]
template <typename R>
__global__ void k_fwd2d_pass1(const C<R>* __restrict__ x, const R* __restrict__ deap, int N, int n,
                              int logn, int rows, const C<R>* __restrict__ tw, C<R>* __restrict__ hbuf) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C<R>* buf = reinterpret_cast<C<R>*>(smraw);
  C<R>* tws = buf + (size_t)rows * n;
  const int j0 = blockIdx.x * rows;
  const int nr = min(rows, N - j0);
  TwStage<R> tp;
  tp.fetch(tw, n / 2);
  // grid point l of row r holds coefficient i = l + N/2 (mod n), deapodised, or 0
  batched<PPT_ROW, C<R>>(
      nr * n,
      [&](int t) {
        const int r = t >> logn, l = t & (n - 1);
        const int i = (l + N / 2) & (n - 1);
        C<R> v = mk<R>(0, 0);
        if (i < N) {
          const R dv = deap[i];
          if (dv != (R)0) v = cscale(x[(int64_t)(j0 + r) * N + i], dv);
        }
        return v;
      },
      [&](int t, C<R> v) { buf[t] = v; });
  tp.store(tw, tws, n / 2);
  __syncthreads();
  fft_smem<R, PPT_ROW>(buf, nr, n, logn, tws, false);
  for (int t = threadIdx.x; t < nr * n; t += blockDim.x) hbuf[(int64_t)j0 * n + t] = buf[t];
}

// pass 2: y-transform of hbuf columns (interior rows) -> grid[lx][:], and of the
// x-boundary coefficient rows i in B -> side[0][k][:]
template <typename R>
__global__ void k_fwd2d_pass2(const C<R>* __restrict__ hbuf, const C<R>* __restrict__ x,
                              const R* __restrict__ deap, int N, int n, int logn, int b, int cols,
                              const C<R>* __restrict__ tw, C<R>* __restrict__ grid, C<R>* __restrict__ side,
                              PComb<R> pc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C<R>* buf = reinterpret_cast<C<R>*>(smraw);
  C<R>* tws = buf + (size_t)cols * n;
  const int c0 = blockIdx.x * cols;
  const int ntot = n + 2 * b;
  const int nc = min(cols, ntot - c0);
  TwStage<R> tp;
  tp.fetch(tw, n / 2);
  // CG direction update (PComb): every row j < N of each column is visited once
  // below, the x-boundary rows (deap = 0) included, so that hp and the boundary
  // columns of p are complete for the interpolation
  const bool comb = pc.hs != nullptr;
  const bool wr = comb && pc.flag[0] == F_RUN;
  const double bd = comb ? pc.beta[0] : 0.0;
  const bool b0 = bd == 0.0;
  const R bt = (R)bd;
  // position l of column c holds row j = l + N/2 (mod n) of the column, deapodised, or 0
  batched<PPT_ROW, C<R>>(
      nc * n,
      [&](int t) {
        const int c = t >> logn, l = t & (n - 1);
        const int j = (l + N / 2) & (n - 1);
        C<R> v = mk<R>(0, 0);
        if (j < N) {
          const R dv = deap[j];
          const int col = c0 + c;
          C<R> u;
          if (col < n) {
            const int64_t e = (int64_t)j * n + col;
            if (comb) {
              u = pc.hs[e];
              if (!b0) {
                const C<R> h = pc.hp[e];
                u = mk<R>(u.x + bt * h.x, u.y + bt * h.y);
              }
              if (wr) pc.hp[e] = u;
            } else {
              u = hbuf[e];
            }
          } else {
            const int k = col - n;
            const int64_t e = (int64_t)j * N + ((k < b) ? k : (N - 1 - (k - b)));
            if (comb) {
              u = pc.s[e];
              if (!b0) {
                const C<R> q = pc.p[e];
                u = mk<R>(u.x + bt * q.x, u.y + bt * q.y);
              }
              if (wr) pc.p[e] = u;
            } else {
              u = x[e];
            }
          }
          if (dv != (R)0) v = cscale(u, dv);
        }
        return v;
      },
      [&](int t, C<R> v) { buf[t] = v; });
  tp.store(tw, tws, n / 2);
  __syncthreads();
  fft_smem<R, PPT_ROW>(buf, nc, n, logn, tws, false);
  for (int t = threadIdx.x; t < nc * n; t += blockDim.x) {
    int c = t / n, l = t - c * n;
    int col = c0 + c;
    if (col < n) grid[(int64_t)col * n + l] = buf[t];
    else side[(int64_t)(col - n) * n + l] = buf[t];
  }
}

// ---------------------------------------------------------------- 2D adjoint
// Spread of one work item (tile (bx, by), samples s0..s1): per warp a private
// padded tile P[(T+2m)^2] ([px][py]), x-side segments S0[2b][T+2m] (along y),
// y-side segments S1[2b][T+2m] (along x), corner sums in registers.
__device__ inline int neighbours(int bx, int nbx, int* cand) {
  int nc = 0;
  for (int dx = -1; dx <= 1; ++dx) {
    int nb = (bx + dx) & (nbx - 1);
    bool dup = false;
    for (int q = 0; q < nc; ++q) dup |= (cand[q] == nb);
    if (!dup) cand[nc++] = nb;
  }
  return nc;
}

// 2D grid point (gx, gy): sum of the padded tiles of the neighbouring bins
template <typename R>
__global__ void k_reduce2d_grid(const int32_t* __restrict__ work_start, const C<R>* __restrict__ part,
                                int64_t stride, int nbx, int tile, int m, int n, C<R>* __restrict__ grid) {
  const int gx = blockIdx.x * tile + threadIdx.y;
  const int gy = blockIdx.y * tile + threadIdx.x;
  if (gx >= n || gy >= n) return;
  const int PW = tile + 2 * m;
  // neighbour bins along each axis in the order -1, 0, +1, each bin once (as neighbours())
  const int bx = gx / tile, by = gy / tile;
  int cx[3], cy[3];
  bool vx[3], vy[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    cx[d] = (bx + d - 1) & (nbx - 1);
    cy[d] = (by + d - 1) & (nbx - 1);
  }
  vx[0] = vy[0] = true;
  vx[1] = cx[1] != cx[0];
  vy[1] = cy[1] != cy[0];
  vx[2] = cx[2] != cx[0] && cx[2] != cx[1];
  vy[2] = cy[2] != cy[0] && cy[2] != cy[1];
  C<R> acc = mk<R>(0, 0);
#pragma unroll
  for (int iy = 0; iy < 3; ++iy)
#pragma unroll
    for (int ix = 0; ix < 3; ++ix) {
      if (!vx[ix] || !vy[iy]) continue;
      const int nb = cy[iy] * nbx + cx[ix];
      const int qx0 = (gx - cx[ix] * tile + m) & (n - 1);
      const int qy0 = (gy - cy[iy] * tile + m) & (n - 1);
      if (qx0 >= PW || qy0 >= PW) continue;  // this bin's tiles do not reach (gx, gy)
      for (int wi = work_start[nb]; wi < work_start[nb + 1]; ++wi)
        for (int qx = qx0; qx < PW; qx += n)
          for (int qy = qy0; qy < PW; qy += n) acc = cadd(acc, part[wi * stride + qx * PW + qy]);
    }
  grid[(int64_t)gx * n + gy] = acc;
}

// The same sum for 16 x 16 tiles and at least 3 bins per axis (no bin is its own
// neighbour): CTA per tile, thread per point; the item ranges of the 3 x 3
// neighbour bins are read once per CTA.  Bins and items are visited in the order
// of k_reduce2d_grid, so the sums are identical.
template <typename R>
__device__ __forceinline__ void reduce_grid16_tile(int bx, int by, const int32_t* __restrict__ work_start,
                                                   const C<R>* __restrict__ part, int64_t stride, int nbx, int m,
                                                   int n, C<R>* __restrict__ grid) {
  constexpr int T = 16;
  __shared__ int rng[9][2];  // [iy * 3 + ix] -> first, end item
  if (threadIdx.x < 9) {
    const int iy = threadIdx.x / 3, ix = threadIdx.x - 3 * iy;
    const int nb = ((by + iy - 1) & (nbx - 1)) * nbx + ((bx + ix - 1) & (nbx - 1));
    rng[threadIdx.x][0] = work_start[nb];
    rng[threadIdx.x][1] = work_start[nb + 1];
  }
  __syncthreads();
  const int lx = threadIdx.x >> 4, ly = threadIdx.x & 15;
  const int PW = T + 2 * m;
  // A point takes its own bin and, within m of a tile edge, the neighbour across
  // that edge (m <= 8 < T: one per axis at most).  Slots in the order of
  // k_reduce2d_grid: (ya, xa), (ya, xb), (yb, xa), (yb, xb) with ya < yb, xa < xb.
  const int ya = (ly < m) ? 0 : 1, yb = (ly < m) ? 1 : (ly >= T - m) ? 2 : -1;
  const int xa = (lx < m) ? 0 : 1, xb = (lx < m) ? 1 : (lx >= T - m) ? 2 : -1;
  int beg[4], c[4], off[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int iy = (s < 2) ? ya : yb, ix = (s & 1) ? xb : xa;
    const bool ok = iy >= 0 && ix >= 0;
    const int j = ok ? iy * 3 + ix : 0;
    beg[s] = rng[j][0];
    c[s] = ok ? rng[j][1] - rng[j][0] : 0;
    off[s] = (lx - T * (ix - 1) + m) * PW + (ly - T * (iy - 1) + m);
  }
  const int c01 = c[0] + c[1], c012 = c01 + c[2], K = c012 + c[3];
  // the contributions k = 0..K-1 in slot order, items ascending: eight loads in
  // flight, then the adds in k order (the sum of k_reduce2d_grid, bit for bit)
  C<R> acc = mk<R>(0, 0);
  for (int k0 = 0; k0 < K; k0 += 8) {
    C<R> v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = k0 + u;
      const int s = (k >= c[0]) + (k >= c01) + (k >= c012);
      const int cs = (s == 0) ? 0 : (s == 1) ? c[0] : (s == 2) ? c01 : c012;
      const int bs = (s == 0) ? beg[0] : (s == 1) ? beg[1] : (s == 2) ? beg[2] : beg[3];
      const int os = (s == 0) ? off[0] : (s == 1) ? off[1] : (s == 2) ? off[2] : off[3];
      v[u] = (k < K) ? part[(int64_t)(bs + k - cs) * stride + os] : mk<R>(0, 0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k0 + u < K) acc = cadd(acc, v[u]);
  }
  grid[(int64_t)(bx * T + lx) * n + by * T + ly] = acc;
}
template <typename R>
__global__ void __launch_bounds__(256) k_reduce2d_grid16(const int32_t* __restrict__ work_start,
                                                         const C<R>* __restrict__ part, int64_t stride, int nbx,
                                                         int m, int n, C<R>* __restrict__ grid) {
  reduce_grid16_tile<R>(blockIdx.x, blockIdx.y, work_start, part, stride, nbx, m, n, grid);
}

// side grids: which = 0 -> x-side k along y (segments S0; the work items of
// the neighbouring bin rows are contiguous), which = 1 -> y-side k along x
// (segments S1; work items of the neighbouring bin columns from the column
// list).  One CTA per (tile of output points, k, which); threads split the
// contributing work items, fixed-order tree sum.
template <typename R>
__device__ __forceinline__ void reduce_side_seg(int gb, int k, int which, const int32_t* __restrict__ work_start,
                                                const int32_t* __restrict__ wcol,
                                                const int32_t* __restrict__ wcol_start, const C<R>* __restrict__ part,
                                                int64_t stride, int nbx, int tile, int m, int n, int b2,
                                                C<R>* __restrict__ side) {
  __shared__ C<R> red[256];
  const int pt = threadIdx.x % tile, wl = threadIdx.x / tile, nl = blockDim.x / tile;
  const int g = gb * tile + pt;
  const int PW = tile + 2 * m;
  const int64_t off = (int64_t)PW * PW + (int64_t)which * b2 * PW + (int64_t)k * PW;
  int cn[3];
  const int nc = neighbours(gb, nbx, cn);
  C<R> acc = mk<R>(0, 0);
  for (int ci = 0; ci < nc; ++ci) {
    const int q0 = (g - cn[ci] * tile + m) & (n - 1);
    const int r0 = (which == 0) ? work_start[cn[ci] * nbx] : wcol_start[cn[ci]];
    const int r1 = (which == 0) ? work_start[(cn[ci] + 1) * nbx] : wcol_start[cn[ci] + 1];
    if (q0 >= PW) continue;  // this bin's segments do not reach g
    // items r0 + wl, + nl, ...: loads issued four at a time, summed in item order
    for (int r = r0 + wl; r < r1; r += 4 * nl) {
      C<R> v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int rr = r + u * nl;
        v[u] = mk<R>(0, 0);
        if (rr < r1) {
          const int wi = (which == 0) ? rr : wcol[rr];
          v[u] = part[wi * stride + off + q0];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc = cadd(acc, v[u]);
      for (int u = 0; u < 4; ++u)  // further periods (grids shorter than a padded tile)
        for (int q = q0 + n; q < PW; q += n) {
          const int rr = r + u * nl;
          if (rr < r1) acc = cadd(acc, part[((which == 0) ? rr : wcol[rr]) * stride + off + q]);
        }
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (wl == 0) {
    C<R> t = mk<R>(0, 0);
    for (int l = 0; l < nl; ++l) t = cadd(t, red[l * tile + pt]);
    side[((int64_t)which * b2 + k) * n + g] = t;
  }
}
template <typename R>
__global__ void k_reduce2d_side(const int32_t* __restrict__ work_start, const int32_t* __restrict__ wcol,
                                const int32_t* __restrict__ wcol_start, const C<R>* __restrict__ part,
                                int64_t stride, int nbx, int tile, int m, int n, int b2, int which0,
                                C<R>* __restrict__ side) {
  reduce_side_seg<R>(blockIdx.x, blockIdx.y, which0 + (int)blockIdx.z, work_start, wcol, wcol_start, part, stride,
                     nbx, tile, m, n, b2, side);
}

// All reductions of the 2D spread's partial tiles in one launch (16 x 16 tiles,
// 256 threads): CTAs [0, nbx^2) sum grid tiles, the next 2 nbx b2 the x- and
// y-side segments, the last b2^2 the corner channels.  Each CTA computes what the
// separate kernels compute, in the same order; one launch on the adjoint's own
// stream replaces three on two side branches.
template <typename R>
__global__ void __launch_bounds__(256) k_reduce2d_all(const int32_t* __restrict__ work_start,
                                                      const int32_t* __restrict__ wcol,
                                                      const int32_t* __restrict__ wcol_start,
                                                      const C<R>* __restrict__ part, int64_t stride, int nbx, int m,
                                                      int n, int b2, int nwork, int64_t coff, C<R>* __restrict__ grid,
                                                      C<R>* __restrict__ side, C<R>* __restrict__ corner) {
  const int ng = nbx * nbx, ns = nbx * b2;
  int id = blockIdx.x;
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the partial tiles of the spread before it
  if (id < ng) {
    reduce_grid16_tile<R>(id % nbx, id / nbx, work_start, part, stride, nbx, m, n, grid);
    return;
  }
  id -= ng;
  if (id < 2 * ns) {
    const int which = id / ns, r = id - which * ns;
    reduce_side_seg<R>(r % nbx, r / nbx, which, work_start, wcol, wcol_start, part, stride, nbx, 16, m, n, b2, side);
    return;
  }
  reduce_chan_one<R>(id - 2 * ns, part, stride, coff, nwork, corner);
}

// adjoint pass 2: inverse y-transform of grid columns -> hbuf[j][lx] (interior j),
// and of the x-side grids -> z[i + N j] for i in B, j interior
template <typename R>
__global__ void k_adj2d_pass2(const C<R>* __restrict__ grid, const C<R>* __restrict__ side,
                              const R* __restrict__ deap, int N, int n, int logn, int b, int cols,
                              const C<R>* __restrict__ tw, C<R>* __restrict__ hbuf, C<R>* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C<R>* buf = reinterpret_cast<C<R>*>(smraw);
  C<R>* tws = buf + (size_t)cols * n;
  const int c0 = blockIdx.x * cols;
  const int ntot = n + 2 * b;
  const int nc = min(cols, ntot - c0);
  TwStage<R> tp;
  tp.fetch(tw, n / 2);
  batched<PPT_ROW, C<R>>(
      nc * n,
      [&](int t) {
        const int c = t >> logn, l = t & (n - 1), col = c0 + c;
        return (col < n) ? grid[(int64_t)col * n + l] : side[(int64_t)(col - n) * n + l];
      },
      [&](int t, C<R> v) { buf[t] = v; });
  tp.store(tw, tws, n / 2);
  __syncthreads();
  fft_smem<R, PPT_ROW>(buf, nc, n, logn, tws, true);
  // t = c + nc j: column c of row j, so that consecutive threads write neighbouring columns
  batched<PPT_ROW, Cv<R>>(
      nc * N,
      [&](int t) {
        const int j = t / nc, c = t - j * nc;
        const R dv = deap[j];
        return Cv<R>{cscale(buf[c * n + ((j - N / 2) & (n - 1))], dv), dv != (R)0};
      },
      [&](int t, Cv<R> o) {
        if (!o.ok) return;
        const int j = t / nc, col = c0 + t - j * nc;
        if (col < n) {
          hbuf[(int64_t)j * n + col] = o.v;
        } else {
          const int k = col - n;
          z[(int64_t)j * N + ((k < b) ? k : (N - 1 - (k - b)))] = o.v;
        }
      });
}

// adjoint pass 1: inverse x-transform of hbuf rows (interior j) or of the y-side
// grids (boundary j) -> z[i + N j] for interior i; corners for boundary i and j
template <typename R>
__global__ void k_adj2d_pass1(const C<R>* __restrict__ hbuf, const C<R>* __restrict__ side1,
                              const C<R>* __restrict__ corner, const R* __restrict__ deap, int N,
                              int n, int logn, int b, int rows, const C<R>* __restrict__ tw,
                              C<R>* __restrict__ z, CgStep<R> cg) {
  extern __shared__ __align__(16) unsigned char smraw[];
  C<R>* buf = reinterpret_cast<C<R>*>(smraw);
  C<R>* tws = buf + (size_t)rows * n;
  const int j0 = blockIdx.x * rows;
  const int nr = min(rows, N - j0);
  const int b2 = 2 * b;
  const int cnt = nr * N;  // entries t = r N + i of these rows
  // entry t of z: from the inverse transform (interior i), a corner (boundary i
  // and j), or not written here (boundary i, interior j: pass 2 wrote it)
  auto zval = [&](int t, R dv) -> Cv<R> {
    const int r = t / N, i = t - r * N, j = j0 + r;
    if (dv != (R)0) return Cv<R>{cscale(buf[r * n + ((i - N / 2) & (n - 1))], dv), true};
    if (j >= b && j < N - b) return Cv<R>{mk<R>(0, 0), false};
    const int kx = (i < b) ? i : b + (N - 1 - i);
    const int ky = (j < b) ? j : b + (N - 1 - j);
    return Cv<R>{corner[ky * b2 + kx], true};
  };
  TwStage<R> tp;
  tp.fetch(tw, n / 2);
  // Fused CG step: its operands (x, p, s, the deapodisation factors and the
  // boundary-column entries of z) are fetched together with the row, so that
  // their loads overlap it; CPT entries per thread are held in registers, any
  // further ones are read in place.  The stop flag is read by every thread: it
  // changes only in the last CTA of this grid, after every CTA has read it.
  constexpr int CPT = 4;
  const bool fused = cg.x != nullptr;
  bool run = false;
  R a = (R)0;
  double bd = 0.0;
  C<R> xv[CPT], pv[CPT], sv[CPT], zb[CPT];
  R dvv[CPT];
  if (fused) {
    run = cg.flag[0] == F_RUN;
    a = (R)cg.alpha[0];
    bd = cg.hs ? cg.beta[0] : 0.0;
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const int t = threadIdx.x + u * blockDim.x;
      zb[u] = mk<R>(0, 0);
      if (t < cnt) {
        const int r = t / N, i = t - r * N, j = j0 + r;
        const int64_t k = (int64_t)j0 * N + t;
        dvv[u] = deap[i];
        xv[u] = cg.x[k];
        pv[u] = cg.p[k];
        sv[u] = cg.s[k];
        if (i < b || i >= N - b) {
          if (j >= b && j < N - b) {
            zb[u] = z[k];
          } else {
            const int kx = (i < b) ? i : b + (N - 1 - i);
            const int ky = (j < b) ? j : b + (N - 1 - j);
            zb[u] = corner[ky * b2 + kx];
          }
        }
      }
    }
  }
  batched<PPT_ROW, C<R>>(
      nr * n,
      [&](int t) {
        const int r = t >> logn, l = t & (n - 1), j = j0 + r;
        if (j >= b && j < N - b) return hbuf[(int64_t)j * n + l];
        const int k = (j < b) ? j : b + (N - 1 - j);
        return side1[(int64_t)k * n + l];
      },
      [&](int t, C<R> v) { buf[t] = v; });
  tp.store(tw, tws, n / 2);
  __syncthreads();
  fft_smem<R, PPT_ROW>(buf, nr, n, logn, tws, true);
  if (!fused) {
    batched<PPT_ROW, Cv<R>>(
        cnt, [&](int t) { return zval(t, deap[t % N]); },
        [&](int t, Cv<R> o) {
          if (o.ok) z[(int64_t)j0 * N + t] = o.v;
        });
    return;
  }
  // z of the held entries (each thread reads only the transform positions of its
  // own entries, which only it overwrites below)
#pragma unroll
  for (int u = 0; u < CPT; ++u) {
    const int t = threadIdx.x + u * blockDim.x;
    if (t < cnt) {
      const Cv<R> o = zval(t, dvv[u]);
      if (o.ok) {
        z[(int64_t)j0 * N + t] = o.v;
        zb[u] = o.v;
      }
    }
  }
  if (!run) {  // the solve has stopped: z only (the remaining entries too)
    for (int t = threadIdx.x + CPT * blockDim.x; t < cnt; t += blockDim.x) {
      const Cv<R> o = zval(t, deap[t % N]);
      if (o.ok) z[(int64_t)j0 * N + t] = o.v;
    }
    return;
  }
  // direction of this step (CgStep::hs): p = s + beta p on the interior columns,
  // with the beta of the previous step (beta = 0: p = s)
  const bool dir = cg.hs != nullptr;
  const bool b0 = bd == 0.0;
  const R bt = (R)bd;
  double acc = 0.0;
  // x += alpha p, s -= alpha z, ||s||^2, and the new s into this row's x-transform
  // input (as k_fwd2d_pass1 lays it out)
  auto step = [&](int t, C<R> xo, C<R> po, C<R> so, C<R> zo, R dv) {
    const int r = t / N, i = t - r * N;
    const int64_t k = (int64_t)j0 * N + t;
    if (dir && i >= b && i < N - b) {
      po = b0 ? so : mk<R>(so.x + bt * po.x, so.y + bt * po.y);
      cg.p[k] = po;
    }
    xo.x += a * po.x;
    xo.y += a * po.y;
    so.x -= a * zo.x;
    so.y -= a * zo.y;
    cg.x[k] = xo;
    cg.s[k] = so;
    acc += (double)so.x * so.x + (double)so.y * so.y;
    if (dir) {
      const int l = (i - N / 2) & (n - 1);
      buf[r * n + l] = (dv != (R)0) ? cscale(so, dv) : mk<R>(0, 0);
      for (int q = N; q < n; q += N) buf[r * n + ((l + q) & (n - 1))] = mk<R>(0, 0);
    }
  };
#pragma unroll
  for (int u = 0; u < CPT; ++u) {
    const int t = threadIdx.x + u * blockDim.x;
    if (t < cnt) step(t, xv[u], pv[u], sv[u], zb[u], dvv[u]);
  }
  for (int t = threadIdx.x + CPT * blockDim.x; t < cnt; t += blockDim.x) {
    const int64_t k = (int64_t)j0 * N + t;
    const R dv = deap[t % N];
    const Cv<R> o = zval(t, dv);
    if (o.ok) z[k] = o.v;
    step(t, cg.x[k], cg.p[k], cg.s[k], o.ok ? o.v : z[k], dv);
  }
  __shared__ double wsum[32];
  __shared__ int last;
  if (dir) {
    __syncthreads();
    fft_smem<R, PPT_ROW>(buf, nr, n, logn, tws, false);
    for (int t = threadIdx.x; t < nr * n; t += blockDim.x) cg.hs[(int64_t)j0 * n + t] = buf[t];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tsum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tsum += wsum[w];
    cg.part[blockIdx.x] = tsum;
    last = 0;
    if (cg.scal) {  // publish the partial, then count this CTA in
      __threadfence();
      last = (atomicAdd(cg.flag + FL_ARRIVE, 1) == (int)gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!last) return;
  // the last CTA: gamma' = sum of the partials in row order, beta, stop test
  __threadfence();
  double g = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) g += __ldcg(cg.part + i);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g += __shfl_down_sync(0xffffffffu, g, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = g;
  __syncthreads();
  if (threadIdx.x == 0) {
    double gs = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) gs += wsum[w];
    double* sc = cg.scal;
    const double beta = gs / sc[S_GAMMA];
    sc[S_BETA] = beta;
    sc[S_GNEW] = gs;
    sc[S_ITER] += 1.0;
    if (!isfinite(beta)) cg.flag[0] = F_BREAK;
    else if (gs <= sc[S_THR2]) cg.flag[0] = F_CONV;
    else if (sc[S_ITER] >= sc[S_MAXIT]) cg.flag[0] = F_MAXIT;
    cg.flag[FL_ARRIVE] = 0;
  }
}

template <typename R>
__global__ void k_gather(const C<R>* __restrict__ in, const int32_t* __restrict__ perm, int64_t M,
                         C<R>* __restrict__ out) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s < M) out[s] = in[perm[s]];
}
template <typename R>
__global__ void k_scatter(const C<R>* __restrict__ in, const int32_t* __restrict__ perm, int64_t M,
                          C<R>* __restrict__ out) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s < M) out[perm[s]] = in[s];
}

template <typename R>
gs_status set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) GS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return GS_OK;
}

template <typename R> constexpr int pass_cols() { return 2; }
constexpr int FOUR_STEP_N = 4096;  // 1D grids from this size use the two-pass FFT

}  // namespace

// ---------------------------------------------------------------- host drivers
template <typename R>
gs_status row_transform(Plan* P, PrecData<R>& D, const C<R>* v, C<R>* out, cudaStream_t st) {
  const int n = (int)P->n, logn = ilog2(P->n), N = (int)P->N;
  const int rows = 1;
  size_t sh1 = ((size_t)rows * n + n / 2) * sizeof(C<R>);
  gs_status s = set_smem<R>((const void*)k_fwd2d_pass1<R>, sh1);
  if (s != GS_OK) return s;
  GS_LAUNCH(pname<R>("fwd2d_pass1<f32>", "fwd2d_pass1<f64>"), st,
            k_fwd2d_pass1<R><<<(N + rows - 1) / rows, fft_threads(rows, n), sh1, st>>>(v, D.deap, N, n, logn, rows,
                                                                                      D.tw, out));
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

template <typename R>
gs_status nfft_T(Plan* P, PrecData<R>& D, const C<R>* x, C<R>* y, const int32_t* perm, cudaStream_t st,
                 double* norm_part, const PComb<R>* pc, bool df) {
  const int n = (int)P->n, logn = ilog2(P->n), N = (int)P->N, b = P->b;
  const int64_t M = P->M;
  const R beta = (R)D.beta;
  if (P->dims == 1) {
    if (n >= FOUR_STEP_N) {
      const int logn1 = logn / 2, logn2 = logn - logn1, n1 = 1 << logn1, n2 = 1 << logn2;
      GS_LAUNCH(pname<R>("fwd1d_cols<f32>", "fwd1d_cols<f64>"), st,
                k_fwd1d_cols<R><<<n1, 256, n2 * sizeof(C<R>), st>>>(x, D.deap, N, n, n1, n2, logn2, D.tw, D.ftmp));
      GS_LAUNCH(pname<R>("fwd1d_rows<f32>", "fwd1d_rows<f64>"), st,
                k_fwd1d_rows<R><<<n2, 256, n1 * sizeof(C<R>), st>>>(D.ftmp, n, n1, logn1, n2, D.tw, D.grid));
    } else {
      size_t sh = (size_t)n * sizeof(C<R>);
      gs_status s = set_smem<R>((const void*)k_fwd1d_fft<R>, sh);
      if (s != GS_OK) return s;
      GS_LAUNCH(pname<R>("fwd1d_fft<f32>", "fwd1d_fft<f64>"), st,
                k_fwd1d_fft<R><<<1, fft_threads(1, n), sh, st>>>(x, D.deap, N, n, logn, D.tw, D.grid));
    }
    if (P->lattice) GS_TRY(lattice_pick<R>(P, D, x, y, perm, st, nullptr, nullptr));
    else
      GS_LAUNCH(pname<R>("interp1d<f32>", "interp1d<f64>"), st,
                k_interp1d<R><<<(M + 255) / 256, 256, 0, st>>>(P->fl, D.frac, D.w, D.bf, b, D.grid, n, D.m, beta,
                                                               x, N, M, perm, y));
  } else {
    // pass 1 (the x transforms of the rows), unless a CG direction update forms
    // them from those of s and of the previous p in pass 2
    if (!pc) GS_TRY(row_transform<R>(P, D, x, D.hbuf, st));
    const int cols = pass_cols<R>();
    size_t sh2 = ((size_t)cols * n + n / 2) * sizeof(C<R>);
    gs_status s = set_smem<R>((const void*)k_fwd2d_pass2<R>, sh2);
    if (s != GS_OK) return s;
    GS_LAUNCH(pname<R>("fwd2d_pass2<f32>", "fwd2d_pass2<f64>"), st,
              k_fwd2d_pass2<R><<<(n + 2 * b + cols - 1) / cols, fft_threads(cols, n), sh2, st>>>(
                  D.hbuf, x, D.deap, N, n, logn, b, cols, D.tw, D.grid, D.side,
                  pc ? *pc : PComb<R>{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr}));
    gs_status si = launch_interp2d<R>(P, D, x, y, perm, st, norm_part, pc ? pc->hp : nullptr, df);
    if (si != GS_OK) return si;
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

// The adjoint with the spread's per-work-item partial sums (nwork x part_stride)
// in `part`: the plan's own buffer (nfft_TH) or a caller-given one
// (nfft_TH_scratch, which allocates nothing).
template <typename R>
static gs_status nfft_TH_part(Plan* P, PrecData<R>& D, const C<R>* y, C<R>* z, const int32_t* perm, C<R>* part,
                              cudaStream_t st, const CgStep<R>* cg) {
  const int n = (int)P->n, logn = ilog2(P->n), N = (int)P->N, b = P->b, b2 = 2 * b;
  const R beta = (R)D.beta;
  const int m = D.m, tile = P->tile;
  if (P->nwork == 0) {
    GS_CUDA(cudaMemsetAsync(z, 0, P->ncoef * sizeof(C<R>), st));
    return GS_OK;
  }
  if (P->dims == 1) {
    const int warps = 4;
    size_t sh = (size_t)warps * (tile + 2 * m + b2) * sizeof(C<R>);
    if (P->lattice) {
      GS_TRY(lattice_fold<R>(P, D, y, perm, st));
    } else {
    GS_LAUNCH(pname<R>("spread1d<f32>", "spread1d<f64>"), st,
              k_spread1d<R><<<P->nwork, warps * 32, sh, st>>>(P->work, P->fl, D.frac, D.w, D.bf, b, y, perm, tile,
                                                              m, beta, part, D.part_stride));
    GS_LAUNCH(pname<R>("reduce1d<f32>", "reduce1d<f64>"), st,
              k_reduce1d<R><<<(n + 127) / 128, 128, 0, st>>>(P->work_start, part, D.part_stride, P->nbx, tile, m,
                                                             n, D.grid));
    if (b2 > 0)
      GS_LAUNCH(pname<R>("reduce_chan<f32>", "reduce_chan<f64>"), st,
                k_reduce_chan<R><<<b2, 256, 0, st>>>(part, D.part_stride, tile + 2 * m, b2, P->nwork, D.corner));
    }
    if (n >= FOUR_STEP_N) {
      const int logn1 = logn / 2, logn2 = logn - logn1, n1 = 1 << logn1, n2 = 1 << logn2;
      GS_LAUNCH(pname<R>("adj1d_rows<f32>", "adj1d_rows<f64>"), st,
                k_adj1d_rows<R><<<n2, 256, n1 * sizeof(C<R>), st>>>(D.grid, n, n1, logn1, n2, D.tw, D.ftmp));
      GS_LAUNCH(pname<R>("adj1d_cols<f32>", "adj1d_cols<f64>"), st,
                k_adj1d_cols<R><<<n1, 256, n2 * sizeof(C<R>), st>>>(D.ftmp, D.deap, N, n, n1, n2, logn2, D.tw,
                                                                    D.corner, b, z));
    } else {
      size_t shf = (size_t)n * sizeof(C<R>);
      gs_status s = set_smem<R>((const void*)k_adj1d_fft<R>, shf);
      if (s != GS_OK) return s;
      GS_LAUNCH(pname<R>("adj1d_fft<f32>", "adj1d_fft<f64>"), st,
                k_adj1d_fft<R><<<1, fft_threads(1, n), shf, st>>>(D.grid, D.deap, N, n, logn, D.tw, D.corner, b, z));
    }
  } else {
    const int PW = tile + 2 * m;
    const int wsz = PW * PW + 2 * b2 * PW;
    const bool lat = P->lattice != 0;
    gs_status s = lat ? lattice_fold<R>(P, D, y, perm, st) : launch_spread2d<R>(P, D, y, perm, part, st);
    if (s != GS_OK) return s;
    // 16 x 16 tiles with boundary columns: every reduction of the partials in one launch
    const bool all1 = !lat && b2 > 0 && tile == 16 && P->nbx >= 3;
    if (all1) {
      const int nb = (int)(P->nbx * P->nbx + 2 * P->nbx * b2 + b2 * b2);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)nb);
      cfg.blockDim = dim3(256);
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = P->pdl ? 1 : 0;  // a programmatic dependent of the spread
      GS_LAUNCH(pname<R>("reduce2d_all<f32>", "reduce2d_all<f64>"), st,
                GS_CUDA(cudaLaunchKernelEx(&cfg, k_reduce2d_all<R>, P->work_start, P->wcol, P->wcol_start,
                                           (const C<R>*)part, D.part_stride, (int)P->nbx, m, n, b2, (int)P->nwork,
                                           (int64_t)wsz, D.grid, D.side, D.corner)));
    }
    // otherwise the three reductions read the same input: side segments and
    // corners on two side branches, the grid on st
    if (b2 > 0 && !lat && !all1) {
      GS_TRY(fork_aux(P, st, 0));
      GS_TRY(fork_aux(P, st, 1));
      cudaStream_t a0 = side_stream(P, st, 0), a1 = side_stream(P, st, 1);
      // x-side grids (pass 2) on branch 0; y-side grids and corners (pass 1) on branch 1
      dim3 sg(P->nbx, b2, 1);
      GS_LAUNCH(pname<R>("reduce2d_side<f32>", "reduce2d_side<f64>"), a0,
                k_reduce2d_side<R><<<sg, 256, 0, a0>>>(P->work_start, P->wcol, P->wcol_start, part,
                                                        D.part_stride, P->nbx, tile, m, n, b2, 0, D.side));
      GS_LAUNCH(pname<R>("reduce2d_side<f32>", "reduce2d_side<f64>"), a1,
                k_reduce2d_side<R><<<sg, 256, 0, a1>>>(P->work_start, P->wcol, P->wcol_start, part,
                                                        D.part_stride, P->nbx, tile, m, n, b2, 1, D.side));
      GS_LAUNCH(pname<R>("reduce_chan<f32>", "reduce_chan<f64>"), a1,
                k_reduce_chan<R><<<b2 * b2, 256, 0, a1>>>(part, D.part_stride, wsz, b2 * b2, P->nwork,
                                                           D.corner));
    }
    dim3 rg(P->nbx, P->nby), rb(tile, tile);
    if (lat || all1) {
    } else if (tile == 16 && P->nbx >= 3)
      GS_LAUNCH(pname<R>("reduce2d_grid<f32>", "reduce2d_grid<f64>"), st,
                k_reduce2d_grid16<R><<<rg, 256, 0, st>>>(P->work_start, part, D.part_stride, P->nbx, m, n,
                                                         D.grid));
    else
      GS_LAUNCH(pname<R>("reduce2d_grid<f32>", "reduce2d_grid<f64>"), st,
                k_reduce2d_grid<R><<<rg, rb, 0, st>>>(P->work_start, part, D.part_stride, P->nbx, tile, m, n,
                                                      D.grid));
    if (b2 > 0 && !lat && !all1) {
      GS_CUDA(cudaGetLastError());
      GS_TRY(join_aux(P, st, 0));  // x-side grids: the last columns of pass 2
    }
    const int cols = pass_cols<R>();
    size_t sh2 = ((size_t)cols * n + n / 2) * sizeof(C<R>);
    s = set_smem<R>((const void*)k_adj2d_pass2<R>, sh2);
    if (s != GS_OK) return s;
    GS_LAUNCH(pname<R>("adj2d_pass2<f32>", "adj2d_pass2<f64>"), st,
              k_adj2d_pass2<R><<<(n + b2 + cols - 1) / cols, fft_threads(cols, n), sh2, st>>>(D.grid, D.side, D.deap, N, n, logn, b,
                                                                              cols, D.tw, D.hbuf, z));
    const int rows = 1;
    size_t sh1 = ((size_t)rows * n + n / 2) * sizeof(C<R>);
    s = set_smem<R>((const void*)k_adj2d_pass1<R>, sh1);
    if (s != GS_OK) return s;
    if (b2 > 0 && !lat && !all1) GS_TRY(join_aux(P, st, 1));  // corner sums: pass 1
    if (cg && cg->join_branch >= 0) GS_TRY(join_aux(P, st, cg->join_branch));
    const CgStep<R> cgv =
        cg ? *cg : CgStep<R>{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, -1, nullptr, nullptr, nullptr};
    GS_LAUNCH(pname<R>("adj2d_pass1<f32>", "adj2d_pass1<f64>"), st,
              k_adj2d_pass1<R><<<(N + rows - 1) / rows, adj1_threads(rows, n), sh1, st>>>(D.hbuf, D.side + (int64_t)b2 * n,
                                                                         D.corner, D.deap, N, n, logn, b, rows,
                                                                         D.tw, z, cgv));
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

template <typename R>
gs_status nfft_TH(Plan* P, PrecData<R>& D, const C<R>* y, C<R>* z, const int32_t* perm, cudaStream_t st,
                  const CgStep<R>* cg) {
  return nfft_TH_part<R>(P, D, y, z, perm, D.part, st, cg);
}
template <typename R>
gs_status nfft_TH_scratch(Plan* P, PrecData<R>& D, const C<R>* y, C<R>* z, const int32_t* perm, C<R>* part,
                          cudaStream_t st) {
  return nfft_TH_part<R>(P, D, y, z, perm, part, st, nullptr);
}

template <typename R>
gs_status gather_sorted(Plan* P, const C<R>* y_user, C<R>* y_sorted, cudaStream_t st) {
  GS_LAUNCH(pname<R>("gather<f32>", "gather<f64>"), st, k_gather<R><<<(P->M + 255) / 256, 256, 0, st>>>(y_user, P->perm, P->M, y_sorted));
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}
template <typename R>
gs_status scatter_user(Plan* P, const C<R>* y_sorted, C<R>* y_user, cudaStream_t st) {
  GS_LAUNCH(pname<R>("scatter<f32>", "scatter<f64>"), st, k_scatter<R><<<(P->M + 255) / 256, 256, 0, st>>>(y_sorted, P->perm, P->M, y_user));
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

template gs_status nfft_T<float>(Plan*, PrecData<float>&, const float2*, float2*, const int32_t*, cudaStream_t,
                                 double*, const PComb<float>*, bool);
template gs_status nfft_T<double>(Plan*, PrecData<double>&, const double2*, double2*, const int32_t*, cudaStream_t,
                                  double*, const PComb<double>*, bool);
template gs_status row_transform<float>(Plan*, PrecData<float>&, const float2*, float2*, cudaStream_t);
template gs_status row_transform<double>(Plan*, PrecData<double>&, const double2*, double2*, cudaStream_t);
template gs_status nfft_TH<float>(Plan*, PrecData<float>&, const float2*, float2*, const int32_t*, cudaStream_t,
                                  const CgStep<float>*);
template gs_status nfft_TH<double>(Plan*, PrecData<double>&, const double2*, double2*, const int32_t*,
                                   cudaStream_t, const CgStep<double>*);
template gs_status nfft_TH_scratch<float>(Plan*, PrecData<float>&, const float2*, float2*, const int32_t*, float2*,
                                          cudaStream_t);
template gs_status nfft_TH_scratch<double>(Plan*, PrecData<double>&, const double2*, double2*, const int32_t*,
                                           double2*, cudaStream_t);
template gs_status gather_sorted<float>(Plan*, const float2*, float2*, cudaStream_t);
template gs_status gather_sorted<double>(Plan*, const double2*, double2*, cudaStream_t);
template gs_status scatter_user<float>(Plan*, const float2*, float2*, cudaStream_t);
template gs_status scatter_user<double>(Plan*, const double2*, double2*, cudaStream_t);

}  // namespace gs
