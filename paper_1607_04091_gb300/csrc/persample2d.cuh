// Per-sample 2D kernels of T and T^H: Kaiser-Bessel interpolation and spreading
// with the boundary factors (Sec. 5, App. C), specialised at compile time on the
// taps per dimension W = 2m and the boundary columns per dimension B2 = 2b
// (B2 = -1: any b, read at run time).  Compiled once per precision
// (persample2d_f32.cu, persample2d_f64.cu).
#pragma once

#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "device_common.cuh"

namespace gs {
namespace dev {

constexpr int NCQ = (GS_MAX_B * GS_MAX_B + 31) / 32;  // corner channels per lane

// window values of the W taps of sample s along dimension d: from the plan's
// table (float32 always, float64 when the plan holds one), else evaluated
template <typename R, int W> struct WinEval;
template <int W> struct WinEval<float, W> {
  static __device__ inline void get(const float* __restrict__ win, int64_t s, int d, float, float, float* out) {
    const float* p = win + ((int64_t)s * 2 + d) * W;
#pragma unroll
    for (int a = 0; a < W; ++a) out[a] = __ldg(p + a);
  }
};
template <int W> struct WinEval<double, W> {
  static __device__ inline void get(const double* win, int64_t s, int d, double t, double beta, double* out) {
    if (win) {  // the plan's table
      const double* p = win + ((int64_t)s * 2 + d) * W;
#pragma unroll
      for (int a = 0; a < W; ++a) out[a] = __ldg(p + a);
    } else {
#pragma unroll
      for (int a = 0; a < W; ++a) out[a] = kb_window(t + (double)(W / 2 - 1 - a), W / 2, beta);
    }
  }
};

__device__ inline int bcol(int k, int b, int N) { return (k < b) ? k : N - 1 - (k - b); }

// Interpolation for the samples of one work item (tile (bx, by)).  The CTA
// stages in shared memory the grid points, x-side and y-side grid segments its
// samples touch and the corner coefficients; one thread per sample gathers its
// W x W interior taps, B2 x W taps of each side and B2^2 corner terms:
//   y = wx wy v_int + wy sum_k bx_k v_xside_k + wx sum_k by_k v_yside_k + sum bx by X
template <typename R, int W, int B2>
__global__ void __launch_bounds__(128, (sizeof(R) == 4 ? 8 : 2)) k_interp2d(
    const int32_t* __restrict__ work, const int32_t* __restrict__ order, const int32_t* __restrict__ fl, const R* __restrict__ frac,
    const R* __restrict__ win, const C<R>* __restrict__ w, const C<R>* __restrict__ bf, int b_rt,
    const C<R>* __restrict__ grid, const C<R>* __restrict__ hbuf, const C<R>* __restrict__ side, int n, R beta,
    const C<R>* __restrict__ x, int N, int64_t M, int nbx, int tile, const int32_t* __restrict__ perm,
    C<R>* __restrict__ y, double* __restrict__ norm_part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int m = W / 2;
  const int b2 = (B2 >= 0) ? B2 : 2 * b_rt;
  const int b2m = b2 > 0 ? b2 : 1;  // divisor for corner indices (no corners when b2 = 0)
  const int b = b2 / 2;
  const int PW = tile + W;  // staged row i <-> grid point o - m + 1 + i
  const int nm = n - 1;
  C<R>* G = reinterpret_cast<C<R>*>(smraw);
  C<R>* S0 = G + PW * PW;   // x-side k along y
  C<R>* S1 = S0 + b2 * PW;  // y-side k along x
  C<R>* XC = S1 + b2 * PW;  // corner coefficients [ky][kx]
  const int it = order[blockIdx.x];  // work item (larger items launch first)
  const int bin = work[3 * it], s0 = work[3 * it + 1], s1 = work[3 * it + 2];
  const int ox = (bin % nbx) * tile, oy = (bin / nbx) * tile;
  const int gx0 = ox - m + 1, gy0 = oy - m + 1;
  for (int i = threadIdx.x; i < PW * PW; i += blockDim.x) {
    const int r = i / PW, c = i - r * PW;
    G[i] = grid[(int64_t)((gx0 + r) & nm) * n + ((gy0 + c) & nm)];
  }
  for (int i = threadIdx.x; i < b2 * PW; i += blockDim.x) {
    const int k = i / PW, c = i - k * PW;
    S0[i] = side[(int64_t)k * n + ((gy0 + c) & nm)];
    S1[i] = hbuf[(int64_t)bcol(k, b, N) * n + ((gx0 + c) & nm)];
  }
  for (int t = threadIdx.x; t < b2 * b2; t += blockDim.x) {
    const int kx = t % b2m, ky = t / b2m;
    XC[t] = x[(int64_t)bcol(ky, b, N) * N + bcol(kx, b, N)];
  }
  __syncthreads();
  double nacc = 0.0;
  for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    const int px = fl[s] - ox, py = fl[M + s] - oy;
    R wx[W], wy[W];
    WinEval<R, W>::get(win, s, 0, frac[s], beta, wx);
    WinEval<R, W>::get(win, s, 1, frac[M + s], beta, wy);
    C<R> vi = mk<R>(0, 0);
#pragma unroll
    for (int a = 0; a < W; ++a) {
      const C<R>* row = G + (px + a) * PW + py;
      C<R> acc = mk<R>(0, 0);
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const C<R> g = row[c];
        acc.x += wy[c] * g.x;
        acc.y += wy[c] * g.y;
      }
      vi.x += wx[a] * acc.x;
      vi.y += wx[a] * acc.y;
    }
    const C<R> wxs = w[s], wys = w[M + s];
    C<R> out = cmul(cmul(wxs, wys), vi);
    if (b2 > 0) {
      const C<R>* bx = bf + (int64_t)s * b2;
      const C<R>* by = bf + (M + s) * b2;
      C<R> sx = mk<R>(0, 0), sy = mk<R>(0, 0), cc = mk<R>(0, 0);
#pragma unroll
      for (int k = 0; k < (B2 >= 0 ? B2 : GS_MAX_B); ++k) {
        if (B2 < 0 && k >= b2) break;
        const C<R>* r0 = S0 + k * PW + py;
        const C<R>* r1 = S1 + k * PW + px;
        C<R> a0 = mk<R>(0, 0), a1 = mk<R>(0, 0);
#pragma unroll
        for (int c = 0; c < W; ++c) {
          const C<R> g0 = r0[c], g1 = r1[c];
          a0.x += wy[c] * g0.x;
          a0.y += wy[c] * g0.y;
          a1.x += wx[c] * g1.x;
          a1.y += wx[c] * g1.y;
        }
        const C<R> bxk = bx[k], byk = by[k];
        sx = cadd(sx, cmul(bxk, a0));
        sy = cadd(sy, cmul(byk, a1));
        C<R> rr = mk<R>(0, 0);  // corner row ky = k: sum_kx bx[kx] X[kx, k]
#pragma unroll
        for (int kx = 0; kx < (B2 >= 0 ? B2 : GS_MAX_B); ++kx) {
          if (B2 < 0 && kx >= b2) break;
          rr = cadd(rr, cmul(bx[kx], XC[k * b2 + kx]));
        }
        cc = cadd(cc, cmul(byk, rr));
      }
      out = cadd(out, cmul(wys, sx));
      out = cadd(out, cmul(wxs, sy));
      out = cadd(out, cc);
    }
    y[perm ? perm[s] : s] = out;
    nacc += (double)out.x * out.x + (double)out.y * out.y;
  }
  if (norm_part) {  // ||y||^2 over this item's samples: lanes, then warps, in a fixed order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nacc += __shfl_down_sync(0xffffffffu, nacc, o);
    __syncthreads();  // the staged tile is no longer read
    double* wsum = reinterpret_cast<double*>(smraw);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = nacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += wsum[i];
      norm_part[it] = t;
    }
  }
}

// ---------------------------------------------------------------- double-float interpolation
// The interpolation of k_interp2d<double> on the float32 units: every float64
// input becomes an unevaluated pair hi + lo of floats (about 48 significant
// bits), and each dot product runs as Dot2 (Ogita, Rump and Oishi, "Accurate sum
// and dot product", SIAM J. Sci. Comput. 26 (2005)): the rounding error of every
// product (TwoProd by FMA) and of every addition (Knuth's TwoSum) is gathered in
// a second float and added back at the end, so the result is about as accurate
// as if computed with twice the float32 precision.  On a part whose float64
// rate is 1/60 of its float32 rate this evaluates the float64 forward apply of
// the refinement residual several times faster, at relative accuracy ~1e-13,
// where the refinement needs far less than float64 precision.
namespace dfa {
struct df {
  float hi, lo;
};
__device__ inline df from(double v) {
  const float h = __double2float_rn(v);
  return df{h, __double2float_rn(v - (double)h)};
}
__device__ inline void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ inline df norm(float s, float c) {  // s + c as a normalised pair (|c| small against |s|)
  const float h = __fadd_rn(s, c);
  return df{h, __fsub_rn(c, __fsub_rn(h, s))};
}
// Dot2 accumulator: value s + c
struct acc {
  float s = 0.0f, c = 0.0f;
  __device__ inline void mac(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);  // exact: a.hi b.hi = p + e
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float q;
    two_sum(s, p, s, q);
    c = __fadd_rn(c, __fadd_rn(q, e));
  }
  __device__ inline void add(df a) {
    float q;
    two_sum(s, a.hi, s, q);
    c = __fadd_rn(c, __fadd_rn(q, a.lo));
  }
  __device__ inline void merge(const acc& o) {  // this += o
    float q;
    two_sum(s, o.s, s, q);
    c = __fadd_rn(c, __fadd_rn(q, o.c));
  }
  __device__ inline df get() const { return norm(s, c); }
};
struct cdf {
  df re, im;
};
__device__ inline cdf cfrom(double2 v) { return cdf{from(v.x), from(v.y)}; }
__device__ inline df neg(df a) { return df{-a.hi, -a.lo}; }
// a * b (complex)
__device__ inline cdf cmul(cdf a, cdf b) {
  acc r, i;
  r.mac(a.re, b.re);
  r.mac(neg(a.im), b.im);
  i.mac(a.re, b.im);
  i.mac(a.im, b.re);
  return cdf{r.get(), i.get()};
}
// r += a * b (complex)
__device__ inline void cmac(acc& r, acc& i, cdf a, cdf b) {
  r.mac(a.re, b.re);
  r.mac(neg(a.im), b.im);
  i.mac(a.re, b.im);
  i.mac(a.im, b.re);
}
}  // namespace dfa

// k_interp2d<double, W, B2> in double-float arithmetic (same staging, one thread
// per sample); the staged grid values are (re hi, re lo, im hi, im lo) float4s.
template <int W, int B2>
__global__ void __launch_bounds__(128, 2) k_interp2d_df(
    const int32_t* __restrict__ work, const int32_t* __restrict__ order, const int32_t* __restrict__ fl,
    const double* __restrict__ win, const double2* __restrict__ w, const double2* __restrict__ bf,
    const double2* __restrict__ grid, const double2* __restrict__ hbuf, const double2* __restrict__ side, int n,
    const double2* __restrict__ x, int N, int64_t M, int nbx, int tile, const int32_t* __restrict__ perm,
    double2* __restrict__ y) {
  using namespace dfa;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int m = W / 2, b = B2 / 2;
  const int PW = tile + W;
  const int nm = n - 1;
  float4* G = reinterpret_cast<float4*>(smraw);
  float4* S0 = G + PW * PW;
  float4* S1 = S0 + B2 * PW;
  float4* XC = S1 + B2 * PW;
  auto put = [](float4* d, double2 v) {
    const df r = from(v.x), i = from(v.y);
    *d = make_float4(r.hi, r.lo, i.hi, i.lo);
  };
  auto get = [](const float4& v) { return cdf{df{v.x, v.y}, df{v.z, v.w}}; };
  const int it = order[blockIdx.x];
  const int bin = work[3 * it], s0 = work[3 * it + 1], s1 = work[3 * it + 2];
  const int ox = (bin % nbx) * tile, oy = (bin / nbx) * tile;
  const int gx0 = ox - m + 1, gy0 = oy - m + 1;
  for (int i = threadIdx.x; i < PW * PW; i += blockDim.x) {
    const int r = i / PW, c = i - r * PW;
    put(G + i, grid[(int64_t)((gx0 + r) & nm) * n + ((gy0 + c) & nm)]);
  }
  for (int i = threadIdx.x; i < B2 * PW; i += blockDim.x) {
    const int k = i / PW, c = i - k * PW;
    put(S0 + i, side[(int64_t)k * n + ((gy0 + c) & nm)]);
    put(S1 + i, hbuf[(int64_t)bcol(k, b, N) * n + ((gx0 + c) & nm)]);
  }
  for (int t = threadIdx.x; t < B2 * B2; t += blockDim.x) {
    const int kx = t % B2, ky = t / B2;
    put(XC + t, x[(int64_t)bcol(ky, b, N) * N + bcol(kx, b, N)]);
  }
  __syncthreads();
  for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    const int px = fl[s] - ox, py = fl[M + s] - oy;
    df wx[W], wy[W];
    const double* pwx = win + ((int64_t)s * 2) * W;
#pragma unroll
    for (int a = 0; a < W; ++a) {
      wx[a] = from(__ldg(pwx + a));
      wy[a] = from(__ldg(pwx + W + a));
    }
    acc vr, vi;
#pragma unroll 2
    for (int a = 0; a < W; ++a) {
      const float4* row = G + (px + a) * PW + py;
      acc r0, r1, i0, i1;  // even and odd taps: four independent chains
#pragma unroll
      for (int c = 0; c < W; c += 2) {
        const cdf g0 = get(row[c]), g1 = get(row[c + 1]);
        r0.mac(wy[c], g0.re);
        i0.mac(wy[c], g0.im);
        r1.mac(wy[c + 1], g1.re);
        i1.mac(wy[c + 1], g1.im);
      }
      r0.merge(r1);
      i0.merge(i1);
      const df wxa = from(__ldg(pwx + a));
      vr.mac(wxa, r0.get());
      vi.mac(wxa, i0.get());
    }
    const cdf wxs = cfrom(w[s]), wys = cfrom(w[M + s]);
    acc orr, oi;
    cmac(orr, oi, cmul(wxs, wys), cdf{vr.get(), vi.get()});
    if (B2 > 0) {
      const double2* bx = bf + (int64_t)s * B2;
      const double2* by = bf + (M + s) * B2;
      acc sxr, sxi, syr, syi, ccr, cci;
#pragma unroll 2
      for (int k = 0; k < B2; ++k) {
        const float4* r0 = S0 + k * PW + py;
        const float4* r1 = S1 + k * PW + px;
        acc a0r, a0i, a1r, a1i;
#pragma unroll
        for (int c = 0; c < W; ++c) {
          const cdf g0 = get(r0[c]), g1 = get(r1[c]);
          a0r.mac(wy[c], g0.re);
          a0i.mac(wy[c], g0.im);
          a1r.mac(wx[c], g1.re);
          a1i.mac(wx[c], g1.im);
        }
        const cdf bxk = cfrom(bx[k]), byk = cfrom(by[k]);
        cmac(sxr, sxi, bxk, cdf{a0r.get(), a0i.get()});
        cmac(syr, syi, byk, cdf{a1r.get(), a1i.get()});
        acc rrr, rri;  // corner row ky = k: sum_kx bx[kx] X[kx, k]
#pragma unroll
        for (int kx = 0; kx < B2; ++kx) cmac(rrr, rri, cfrom(bx[kx]), get(XC[k * B2 + kx]));
        cmac(ccr, cci, byk, cdf{rrr.get(), rri.get()});
      }
      cmac(orr, oi, wys, cdf{sxr.get(), sxi.get()});
      cmac(orr, oi, wxs, cdf{syr.get(), syi.get()});
      orr.add(ccr.get());
      oi.add(cci.get());
    }
    const df o_r = orr.get(), o_i = oi.get();
    y[perm ? perm[s] : s] = make_double2((double)o_r.hi + (double)o_r.lo, (double)o_i.hi + (double)o_i.lo);
  }
}

// Spread of one work item (tile (bx, by), samples s0..s1) in batches.  Phase 1,
// one thread per sample: window values and the per-sample coefficients
// (u conj(wx wy); A_k = u conj(bx_k); conj(by_k); conj(wy); u conj(wx)) into
// shared memory (row strides padded against bank conflicts).  Phase 2, one warp
// per sample, lanes over the taps: read-modify-write into the warp's private
// padded tile P [(T+2m)^2], x-side segments S0 [2b][T+2m] and y-side segments
// S1 [2b][T+2m]; corner channel kx + 2b ky accumulates in a register of a fixed
// lane.  No atomics: each address is written by one lane of one warp per step.
template <typename R, int W, int B2>
__global__ void __launch_bounds__(256) k_spread2d(
    const int32_t* __restrict__ work, const int32_t* __restrict__ order, const int32_t* __restrict__ fl, const R* __restrict__ frac,
    const R* __restrict__ win, const C<R>* __restrict__ w, const C<R>* __restrict__ bf, int b_rt,
    const C<R>* __restrict__ u, const int32_t* __restrict__ perm, int64_t M, int nbx, int tile, R beta, int batch,
    C<R>* __restrict__ part, int64_t stride) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int b2 = (B2 >= 0) ? B2 : 2 * b_rt;
  const int b2m = b2 > 0 ? b2 : 1;  // divisor for corner indices (no corners when b2 = 0)
  const int PW = tile + W;
  const int wsz = PW * PW + 2 * b2 * PW;
  const int nw = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int vst = 3 + 2 * b2;      // complex values staged per sample
  const int wst = 2 * W + 1;       // window values staged per sample (padded)
  C<R>* base = reinterpret_cast<C<R>*>(smraw);
  C<R>* P = base + (int64_t)wid * wsz;
  C<R>* S0 = P + PW * PW;
  C<R>* S1 = S0 + b2 * PW;
  C<R>* CS = base + (int64_t)nw * wsz;        // [nw][b2*b2]
  C<R>* sv = CS + (int64_t)nw * b2 * b2;      // [batch][vst]
  R* swin = reinterpret_cast<R*>(sv + (int64_t)batch * vst);        // [batch][wst]
  int* spos = reinterpret_cast<int*>(swin + (int64_t)batch * wst);  // [batch][2]
  for (int i = lane; i < wsz; i += 32) P[i] = mk<R>(0, 0);
  C<R> cc[NCQ];
  int cka[NCQ], ckb[NCQ];
#pragma unroll
  for (int q = 0; q < NCQ; ++q) {
    const int ch = lane + 32 * q;
    cc[q] = mk<R>(0, 0);
    cka[q] = (ch < b2 * b2) ? 3 + ch % b2m : 0;       // A[kx]
    ckb[q] = (ch < b2 * b2) ? 3 + b2 + ch / b2m : 0;  // conj(by[ky])
  }
  const int it = order[blockIdx.x];  // work item (larger items launch first)
  const int bin = work[3 * it], s0 = work[3 * it + 1], s1 = work[3 * it + 2];
  const int ox = (bin % nbx) * tile, oy = (bin / nbx) * tile;
  for (int sb = s0; sb < s1; sb += batch) {
    const int nb = min(batch, s1 - sb);
    if (threadIdx.x < nb) {
      const int j = threadIdx.x, s = sb + j;
      const C<R> us = u[perm ? perm[s] : s];
      spos[2 * j] = fl[s] - ox + 1;
      spos[2 * j + 1] = fl[M + s] - oy + 1;
      R wv[W];
      WinEval<R, W>::get(win, s, 0, frac[s], beta, wv);
#pragma unroll
      for (int a = 0; a < W; ++a) swin[j * wst + a] = wv[a];
      WinEval<R, W>::get(win, s, 1, frac[M + s], beta, wv);
#pragma unroll
      for (int a = 0; a < W; ++a) swin[j * wst + W + a] = wv[a];
      const C<R> wxs = w[s], wys = w[M + s];
      C<R>* v = sv + (int64_t)j * vst;
      v[0] = cmulc(cmulc(us, wxs), wys);
      v[1] = mk<R>(wys.x, -wys.y);
      v[2] = cmulc(us, wxs);
#pragma unroll
      for (int k = 0; k < (B2 >= 0 ? B2 : GS_MAX_B); ++k) {
        if (B2 < 0 && k >= b2) break;
        const C<R> bxk = bf[(int64_t)s * b2 + k], byk = bf[(M + s) * b2 + k];
        v[3 + k] = cmulc(us, bxk);
        v[3 + b2 + k] = mk<R>(byk.x, -byk.y);
      }
    }
    __syncthreads();
    for (int j = wid; j < nb; j += nw) {
      const int px = spos[2 * j], py = spos[2 * j + 1];
      const R* wx = swin + j * wst;
      const R* wy = wx + W;
      const C<R>* v = sv + (int64_t)j * vst;
      const C<R> vi = v[0];
#pragma unroll
      for (int q = 0; q < (W * W + 31) / 32; ++q) {
        const int t = lane + 32 * q;
        if (t < W * W) {
          const int a = t / W, c = t % W;
          const R f = wx[a] * wy[c];
          C<R>& d = P[(px + a) * PW + (py + c)];
          d.x += f * vi.x;
          d.y += f * vi.y;
        }
      }
      if (b2 > 0) {
        const C<R> cwy = v[1], uwx = v[2];
#pragma unroll
        for (int q = 0; q < (B2 >= 0 ? (B2 * W + 31) / 32 : (GS_MAX_B * W + 31) / 32); ++q) {
          const int t = lane + 32 * q;
          if (t < b2 * W) {
            const int k = t / W, c = t % W;
            const C<R> v0 = cmul(v[3 + k], cwy);       // x-side k, along y
            C<R>& d0 = S0[k * PW + py + c];
            d0.x += wy[c] * v0.x;
            d0.y += wy[c] * v0.y;
            const C<R> v1 = cmul(uwx, v[3 + b2 + k]);  // y-side k, along x
            C<R>& d1 = S1[k * PW + px + c];
            d1.x += wx[c] * v1.x;
            d1.y += wx[c] * v1.y;
          }
        }
#pragma unroll
        for (int q = 0; q < NCQ; ++q)
          if (lane + 32 * q < b2 * b2) cc[q] = cadd(cc[q], cmul(v[cka[q]], v[ckb[q]]));
      }
      __syncwarp();
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NCQ; ++q)
    if (lane + 32 * q < b2 * b2) CS[wid * b2 * b2 + lane + 32 * q] = cc[q];
  __syncthreads();
  C<R>* out = part + it * stride;
  for (int i = threadIdx.x; i < wsz; i += blockDim.x) {
    C<R> acc = mk<R>(0, 0);
    for (int q = 0; q < nw; ++q) acc = cadd(acc, base[(int64_t)q * wsz + i]);
    out[i] = acc;
  }
  for (int i = threadIdx.x; i < b2 * b2; i += blockDim.x) {
    C<R> acc = mk<R>(0, 0);
    for (int q = 0; q < nw; ++q) acc = cadd(acc, CS[q * b2 * b2 + i]);
    out[wsz + i] = acc;
  }
}

// ---------------------------------------------------------------- warp-level tensor-core helpers
// (mma.sync TF32 with the 3xTF32 split and cp.async staging; used by the
// tensor-core interpolation below)
namespace tc {
// x = hi + lo with hi = x rounded to the 10 explicit mantissa bits of TF32 (add half
// an ulp of TF32 to the bit pattern, then clear the 13 low bits: round to nearest,
// ties away from zero) and lo = x - hi exact in float32, |lo| <= 2^-11 |x|.  lo goes
// to the tensor core as it is; TF32 uses its 10 leading mantissa bits, so the
// split keeps about 21 bits of x.
__device__ inline void split(float x, uint32_t& hi, uint32_t& lo) {
  hi = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
  lo = __float_as_uint(x - __uint_as_float(hi));
}
__device__ inline void mma(float* c, const uint32_t* a, const uint32_t* b) {
  asm(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// B fragment (8 x 8, k-rows k0.., columns n0..) from an operand stored [n][k]
__device__ inline void load_bT(const float* B, int ld, int n0, int k0, int lane, uint32_t* hi, uint32_t* lo) {
  const int g = lane >> 2, t = lane & 3;
  split(B[(n0 + g) * ld + k0 + t], hi[0], lo[0]);
  split(B[(n0 + g) * ld + k0 + t + 4], hi[1], lo[1]);
}
__device__ inline void cp_async16(float* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src));
}
__device__ inline void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src));
}
__device__ inline void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src));
}
__device__ inline void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ inline void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
}  // namespace tc

}  // namespace dev
}  // namespace gs
#include "spread2d_tcgen05.cuh"
namespace gs {
namespace dev {

// ---------------------------------------------------------------- tensor-core interpolation
// float32, W = 8 taps, 2b = 8 boundary columns, 16 x 16 tiles.  With the staged
// grid tile G[x][y], side segments S0[k][y], S1[k][x] and corner coefficients
// X[ky][kx] of one work item, a batch of 32 samples needs
//   H[s][x]  = sum_y wy_s[y - py_s] G[x][y]        (interior, then sum_a wx_s[a] H[s][px_s + a])
//   Q0[s][k] = sum_y wy_s[y - py_s] S0[k][y]       (x-sides, then sum_k bx_s[k] Q0[s][k])
//   Q1[s][k] = sum_x wx_s[x - px_s] S1[k][x]       (y-sides, then sum_k by_s[k] Q1[s][k])
//   RR[s][ky] = sum_kx bx_s[kx] X[ky][kx]          (corners, then sum_ky by_s[ky] RR[s][ky])
// i.e. GEMMs with M = samples, on mma.sync m16n8k8 TF32 with the 3xTF32 split.
// The window operand is never written out: a lane's fragment rows are fixed
// samples, and its element (row s, column k0 + c) is tap k0 + c - pos_s of s,
// nonzero in exactly one of the three k-steps; each lane loads and splits its
// taps once per batch and selects them per step.  The item operands G, S0, S1
// stay plain floats, split at each fragment load (a 64-bit pair load would take
// two shared-memory wavefronts).  Per batch: cp.async stages the
// next batch's inputs; warps 0-1 form H (one 16-sample block each, real and
// imaginary part), warp 2 Q0 and half of RR, warp 3 Q1 and the other half; then
// four threads per sample combine
//   y = wx wy sum_a wx_a H[px + a] + wy sum_k bx_k Q0_k + wx sum_k by_k Q1_k + sum_k by_k RR_k.
namespace tci {
using tc::split;
using tc::mma;
using tc::cp_async16;
using tc::cp_async8;
using tc::cp_async4;
using tc::cp_commit;
using tc::cp_wait_all;
constexpr int SBT = 32, W = 8, B2 = 8, TILE = 16, PW = TILE + W;
constexpr int LDQ = 28;  // rows of the item operands [n][k]: conflict-free fragment loads
constexpr int LDX = 20;  // rows of the corner operands (K = 16), stored [ky][k]
constexpr int LDS = 20;  // staged rows of 16 floats
// item operands (floats)
constexpr int I_GR = 0, I_GI = I_GR + PW * LDQ;  // [x][y]
constexpr int I_S0R = I_GI + PW * LDQ, I_S0I = I_S0R + B2 * LDQ;  // [k][y]
constexpr int I_S1R = I_S0I + B2 * LDQ, I_S1I = I_S1R + B2 * LDQ;  // [k][x]
constexpr int I_XR = I_S1I + B2 * LDQ;  // [ky][k]: k < 8 Re X[ky][k], k >= 8 -Im X[ky][k - 8]
constexpr int I_XI = I_XR + B2 * LDX;       // [ky][k]: k < 8 Im X[ky][k], k >= 8  Re X[ky][k - 8]
constexpr int N_ITEM = I_XI + B2 * LDX;
// the four terms of each sample (interior, x-sides, y-sides, corners), complex
// [buffer][term][sample]: batch b's terms are summed during batch b + 1
constexpr int O_T = N_ITEM;
constexpr int T_SIZE = 4 * 2 * SBT;
// staged inputs, two buffers: taps wx | wy, bx, by (complex), phases wx wy, grid indices
constexpr int ST_WIN = 0, ST_BX = ST_WIN + SBT * LDS, ST_BY = ST_BX + SBT * LDS, ST_W = ST_BY + SBT * LDS;
constexpr int ST_FL = ST_W + 4 * SBT;
constexpr int ST_SIZE = ST_FL + 2 * SBT;
constexpr int S_STAGE = O_T + 2 * T_SIZE;
constexpr int N_SMEM = S_STAGE + 2 * ST_SIZE;
static_assert(S_STAGE % 4 == 0 && ST_SIZE % 4 == 0 && O_T % 2 == 0, "16-byte staging, 8-byte terms");

__device__ inline void stage(float* st, int wid, int lane, int sb, int nb, const float* __restrict__ win,
                             const float2* __restrict__ w, const float2* __restrict__ bf,
                             const int32_t* __restrict__ fl, int64_t M) {
  if (lane >= nb) return;
  const int64_t s = sb + lane;
  if (wid == 0) {
    const float* src = win + s * (2 * W);
#pragma unroll
    for (int c = 0; c < 4; ++c) cp_async16(st + ST_WIN + lane * LDS + 4 * c, src + 4 * c);
  } else if (wid < 3) {
    const float2* src = bf + (s + (wid == 2 ? M : 0)) * B2;
    float* dst = st + (wid == 1 ? ST_BX : ST_BY) + lane * LDS;
#pragma unroll
    for (int c = 0; c < 4; ++c) cp_async16(dst + 4 * c, src + 2 * c);
  } else {
    cp_async8(st + ST_W + 4 * lane, w + s);
    cp_async8(st + ST_W + 4 * lane + 2, w + M + s);
    cp_async4(st + ST_FL + 2 * lane, fl + s);
    cp_async4(st + ST_FL + 2 * lane + 1, fl + M + s);
  }
}
// The lane's window elements of one batch: for fragment rows h (samples rs0 + g +
// 8h, window start pos[h]; pos < -W for an empty row) and column halves e
// (columns t + 4e + 8 step), the step at which tap t + 4e + 8 step - pos is in
// range and that tap, split
template <int NH>
__device__ inline void win_elems(const float* taps, const int* pos, int rs0, int lane, int* ks, uint32_t* hi,
                                 uint32_t* lo) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int h = 0; h < NH; ++h)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int c0 = t + 4 * e - pos[h];      // column offset at step 0, in [-15, 7] or >= 16
      const int step = (7 - c0) >> 3;         // 0..2 for a sample, negative for an empty row
      float v = 0.0f;
      if (step >= 0) v = taps[(rs0 + g + 8 * (h & 1) + 16 * (h >> 1)) * LDS + c0 + 8 * step];
      ks[2 * h + e] = step;
      split(v, hi[2 * h + e], lo[2 * h + e]);
    }
}
}  // namespace tci

static __global__ void __launch_bounds__(128, 7) k_interp2d_tc(
    const int32_t* __restrict__ work, const int32_t* __restrict__ order, const int32_t* __restrict__ fl,
    const float* __restrict__ win, const float2* __restrict__ w, const float2* __restrict__ bf,
    const float2* __restrict__ grid, const float2* __restrict__ hbuf, const float2* __restrict__ side, int n,
    const float2* __restrict__ x, int N, int64_t M, int nbx, const int32_t* __restrict__ perm,
    float2* __restrict__ y, double* __restrict__ norm_part) {
  using namespace tci;
  extern __shared__ __align__(16) float sm[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  // a kernel launched as this one's programmatic dependent (the spread of a CG
  // step) may start its set-up now; it waits for this grid before reading y
  asm volatile("griddepcontrol.launch_dependents;");
  const int it = order[blockIdx.x];  // work item (larger items launch first)
  const int bin = work[3 * it], s0 = work[3 * it + 1], s1 = work[3 * it + 2];
  const int ox = (bin % nbx) * TILE, oy = (bin / nbx) * TILE;
  constexpr int m = W / 2, b = B2 / 2;
  const int nm = n - 1, gx0 = ox - m + 1, gy0 = oy - m + 1;
  stage(sm + S_STAGE, wid, lane, s0, min(SBT, s1 - s0), win, w, bf, fl, M);
  cp_commit();
  // item operands (staged row i <-> grid point o - m + 1 + i)
  for (int i = threadIdx.x; i < PW * PW; i += blockDim.x) {
    const int r = i / PW, c = i - r * PW;
    const float2 v = grid[(int64_t)((gx0 + r) & nm) * n + ((gy0 + c) & nm)];
    sm[I_GR + r * LDQ + c] = v.x;
    sm[I_GI + r * LDQ + c] = v.y;
  }
  for (int i = threadIdx.x; i < B2 * PW; i += blockDim.x) {
    const int k = i / PW, c = i - k * PW;
    const float2 a = side[(int64_t)k * n + ((gy0 + c) & nm)];
    const float2 e = hbuf[(int64_t)bcol(k, b, N) * n + ((gx0 + c) & nm)];
    sm[I_S0R + k * LDQ + c] = a.x;
    sm[I_S0I + k * LDQ + c] = a.y;
    sm[I_S1R + k * LDQ + c] = e.x;
    sm[I_S1I + k * LDQ + c] = e.y;
  }
  if (threadIdx.x < B2 * B2) {
    const int kx = threadIdx.x % B2, ky = threadIdx.x / B2;
    const float2 X = x[(int64_t)bcol(ky, b, N) * N + bcol(kx, b, N)];
    sm[I_XR + ky * LDX + kx] = X.x;
    sm[I_XR + ky * LDX + B2 + kx] = -X.y;
    sm[I_XI + ky * LDX + kx] = X.y;
    sm[I_XI + ky * LDX + B2 + kx] = X.x;
  }
  double nacc = 0.0;
  // y = (interior + x-sides) + (y-sides + corners) for the samples of a finished batch
  auto finish = [&](const float* tb, int sbp, int nbp) {
    if (wid == 0 && lane < nbp) {
      const float2* tm = reinterpret_cast<const float2*>(tb);
      const float2 c = cadd(cadd(tm[lane], tm[SBT + lane]), cadd(tm[2 * SBT + lane], tm[3 * SBT + lane]));
      const int s = sbp + lane;
      y[perm ? perm[s] : s] = c;
      nacc += (double)c.x * c.x + (double)c.y * c.y;
    }
  };
  int buf = 0, sb_prev = 0, nb_prev = 0;
  for (int sb = s0; sb < s1; sb += SBT, buf ^= 1) {
    const int nb = min(SBT, s1 - sb);
    cp_wait_all();
    __syncthreads();  // this batch staged, item operands written; the last batch's terms written
    if (sb + SBT < s1)
      stage(sm + S_STAGE + (buf ^ 1) * ST_SIZE, wid, lane, sb + SBT, min(SBT, s1 - sb - SBT), win, w, bf, fl, M);
    cp_commit();
    if (sb > s0) finish(sm + O_T + (buf ^ 1) * T_SIZE, sb_prev, nb_prev);
    sb_prev = sb;
    nb_prev = nb;
    float* tbuf = sm + O_T + buf * T_SIZE;
    const float* st = sm + S_STAGE + buf * ST_SIZE;
    const int* sfl = reinterpret_cast<const int*>(st + ST_FL);
    float acc[6][4];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][q] = 0.0f;
    if (wid < 2) {
      // H for samples m0 .. m0+15: tiles [re: 0-2 | im: 3-5][x block]
      const int m0 = 16 * wid;
      int pos[2], ks[4];
      uint32_t th[4], tl[4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int s = m0 + g + 8 * h;
        pos[h] = (s < nb) ? sfl[2 * s + 1] - oy : -2 * W;
      }
      win_elems<2>(st + ST_WIN + W, pos, m0, lane, ks, th, tl);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        uint32_t ah[4], al[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // fragment element q = row half + 2 column half
          const int i = 2 * (q & 1) + (q >> 1);
          ah[q] = (ks[i] == k) ? th[i] : 0u;
          al[q] = (ks[i] == k) ? tl[i] : 0u;
        }
#pragma unroll
        for (int ri = 0; ri < 2; ++ri) {  // real, then imaginary part of G: 12 fragment registers live
          uint32_t bh[3][2], bl[3][2];
#pragma unroll
          for (int nbk = 0; nbk < 3; ++nbk)
            tc::load_bT(sm + (ri ? I_GI : I_GR), LDQ, 8 * nbk, 8 * k, lane, bh[nbk], bl[nbk]);
#pragma unroll
          for (int term = 0; term < 3; ++term)
#pragma unroll
            for (int nbk = 0; nbk < 3; ++nbk)
              mma(acc[3 * ri + nbk], term == 2 ? al : ah, term == 1 ? bl[nbk] : bh[nbk]);
        }
      }
      // interior term: the lane holds H[s][x] for its two samples and six columns x;
      // sum wx_s[x - px_s] H[s][x] over them, then over the quad's four lanes
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int s = m0 + g + 8 * h;
        const int px = (s < nb) ? sfl[2 * s] - ox : -2 * W;
        float2 v = make_float2(0.0f, 0.0f);
        // the lane's columns 8 nbk + 2t + e (nbk = 0..2) are 8 apart, so at most one
        // of them falls in the window [px, px + 8): block nb_e, tap a_e
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int c0 = 2 * t + e - px;   // tap index in block 0, in [-15, 7] or <= -9 for an empty row
          const int nbe = (7 - c0) >> 3;   // block whose tap index is in [0, 8)
          if (nbe >= 0 && nbe < 3) {
            const float tap = st[ST_WIN + s * LDS + c0 + 8 * nbe];
            const float hr = (nbe == 0) ? acc[0][2 * h + e] : (nbe == 1) ? acc[1][2 * h + e] : acc[2][2 * h + e];
            const float hi = (nbe == 0) ? acc[3][2 * h + e] : (nbe == 1) ? acc[4][2 * h + e] : acc[5][2 * h + e];
            v.x += tap * hr;
            v.y += tap * hi;
          }
        }
        v.x += __shfl_xor_sync(0xffffffffu, v.x, 1);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, 1);
        v.x += __shfl_xor_sync(0xffffffffu, v.x, 2);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, 2);
        if (t == 0 && s < nb) {
          const float4 ww = *reinterpret_cast<const float4*>(st + ST_W + 4 * s);
          *reinterpret_cast<float2*>(tbuf + 2 * s) = cmul(cmul(make_float2(ww.x, ww.y), make_float2(ww.z, ww.w)), v);
        }
      }
    } else {
      // warp 2: Q0 (wy, S0), warp 3: Q1 (wx, S1); tiles [block][re | im]; corners in 4, 5
      const bool xs = (wid == 2);
      int pos[4], ks[8];
      uint32_t th[8], tl[8];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int s = g + 8 * h;
        pos[h] = (s < nb) ? sfl[2 * s + (xs ? 1 : 0)] - (xs ? oy : ox) : -2 * W;
      }
      win_elems<4>(st + ST_WIN + (xs ? W : 0), pos, 0, lane, ks, th, tl);
      const float* Sr = sm + (xs ? I_S0R : I_S1R);
      const float* Si = sm + (xs ? I_S0I : I_S1I);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        uint32_t ah[2][4], al[2][4], bh[2][2], bl[2][2];
#pragma unroll
        for (int mb = 0; mb < 2; ++mb)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int i = 2 * (2 * mb + (q & 1)) + (q >> 1);
            ah[mb][q] = (ks[i] == k) ? th[i] : 0u;
            al[mb][q] = (ks[i] == k) ? tl[i] : 0u;
          }
        tc::load_bT(Sr, LDQ, 0, 8 * k, lane, bh[0], bl[0]);
        tc::load_bT(Si, LDQ, 0, 8 * k, lane, bh[1], bl[1]);
#pragma unroll
        for (int term = 0; term < 3; ++term)
#pragma unroll
          for (int tq = 0; tq < 4; ++tq)
            mma(acc[tq], term == 2 ? al[tq >> 1] : ah[tq >> 1], term == 1 ? bl[tq & 1] : bh[tq & 1]);
      }
      // corners for samples rc .. rc+15: A = [Re bx | Im bx], K = 16
      const int rc = xs ? 0 : 16;
#pragma unroll
      for (int k0 = 0; k0 < 2 * B2; k0 += 8) {
        uint32_t ah[4], al[4], bh[2][2], bl[2][2];
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int s = rc + g + 8 * h, kk = k0 + t + 4 * e;
            const float v = (s < nb) ? st[ST_BX + s * LDS + 2 * (kk & 7) + (kk >> 3)] : 0.0f;
            split(v, ah[h + 2 * e], al[h + 2 * e]);
          }
        tc::load_bT(sm + I_XR, LDX, 0, k0, lane, bh[0], bl[0]);
        tc::load_bT(sm + I_XI, LDX, 0, k0, lane, bh[1], bl[1]);
#pragma unroll
        for (int term = 0; term < 3; ++term)
#pragma unroll
          for (int ri = 0; ri < 2; ++ri) mma(acc[4 + ri], term == 2 ? al : ah, term == 1 ? bl[ri] : bh[ri]);
      }
      // side and corner terms: the lane holds Q[s][k] and RR[s][k] for k = 2t, 2t + 1;
      // sum the boundary factors times them, then over the quad's four lanes
      const float* bq = st + (xs ? ST_BX : ST_BY);  // x-sides pair with bx, y-sides with by
#pragma unroll
      for (int h = 0; h < 6; ++h) {  // rows: side block 0 (g, g+8), block 1 (16+g, 24+g), corners (rc+g, rc+g+8)
        const int s = (h < 4) ? g + 8 * (h & 1) + 16 * (h >> 1) : rc + g + 8 * (h & 1);
        const int tr = (h < 4) ? 2 * (h >> 1) : 4;  // tile pair of this row
        const float* fac = (h < 4) ? bq : st + ST_BY;
        float2 v = make_float2(0.0f, 0.0f);
        if (s < nb) {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int k = 2 * t + e;
            const float2 f = *reinterpret_cast<const float2*>(fac + s * LDS + 2 * k);
            v = cadd(v, cmul(f, make_float2(acc[tr][2 * (h & 1) + e], acc[tr + 1][2 * (h & 1) + e])));
          }
        }
        v.x += __shfl_xor_sync(0xffffffffu, v.x, 1);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, 1);
        v.x += __shfl_xor_sync(0xffffffffu, v.x, 2);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, 2);
        if (t == 0 && s < nb) {
          if (h < 4) {  // x-sides times wy, y-sides times wx
            const float4 ww = *reinterpret_cast<const float4*>(st + ST_W + 4 * s);
            v = xs ? cmul(make_float2(ww.z, ww.w), v) : cmul(make_float2(ww.x, ww.y), v);
          }
          *reinterpret_cast<float2*>(tbuf + 2 * ((h < 4 ? (xs ? 1 : 2) : 3) * SBT + s)) = v;
        }
      }
    }
  }
  __syncthreads();  // the last batch's terms written
  finish(sm + O_T + (buf ^ 1) * T_SIZE, sb_prev, nb_prev);
  if (norm_part) {  // ||y||^2 over this item's samples (all in warp 0): lanes in a fixed order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nacc += __shfl_down_sync(0xffffffffu, nacc, o);
    if (threadIdx.x == 0) norm_part[it] = nacc;
  }
}

template <typename R>
gs_status set_smem_attr(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) GS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return GS_OK;
}

template <typename F>
gs_status dispatch_wb(int W, int B2, F&& f) {
  auto with_w = [&](auto wc) -> gs_status {
    switch (B2) {
      case 0: return f(wc, std::integral_constant<int, 0>());
      case 4: return f(wc, std::integral_constant<int, 4>());
      case 8: return f(wc, std::integral_constant<int, 8>());
      default: return f(wc, std::integral_constant<int, -1>());
    }
  };
  switch (W) {
    case 8: return with_w(std::integral_constant<int, 8>());
    case 12: return with_w(std::integral_constant<int, 12>());
    case 16: return with_w(std::integral_constant<int, 16>());
  }
  set_error("Kaiser-Bessel half-width m = %d has no compiled 2D kernel (4, 6 or 8)", W / 2);
  return GS_EUNSUPPORTED;
}

}  // namespace dev

template <typename R>
gs_status launch_interp2d(Plan* P, PrecData<R>& D, const C<R>* x, C<R>* y, const int32_t* perm, cudaStream_t st,
                         double* norm_part, const C<R>* hrows, bool dfl) {
  using namespace dev;
  const int b = P->b, b2 = 2 * b, tile = P->tile;
  if (P->nwork == 0) return GS_OK;
  if (P->lattice) return lattice_pick<R>(P, D, x, y, perm, st, norm_part, hrows);
  const C<R>* hb = hrows ? hrows : D.hbuf;
  return dispatch_wb(2 * D.m, b2, [&](auto wc, auto bc) -> gs_status {
    constexpr int W = decltype(wc)::value;
    constexpr int B2 = decltype(bc)::value;
    const int PW = tile + W;
    if (sizeof(R) == 4 && W == 8 && B2 == 8 && tile == 16 && !std::getenv("GS_NO_TC")) {
      const size_t shc = (size_t)tci::N_SMEM * sizeof(float);
      gs_status e = set_smem_attr<R>((const void*)k_interp2d_tc, shc);
      if (e != GS_OK) return e;
      GS_LAUNCH("interp2d<f32>", st,
                k_interp2d_tc<<<P->nwork, 128, shc, st>>>(
                    P->work, P->work_order, P->fl, (const float*)D.win, (const float2*)D.w, (const float2*)D.bf,
                    (const float2*)D.grid, (const float2*)hb, (const float2*)D.side, (int)P->n,
                    (const float2*)x, (int)P->N, P->M, P->nbx, perm, (float2*)y, norm_part));
      GS_CUDA(cudaGetLastError());
      return GS_OK;
    }
    const size_t sh = ((size_t)PW * PW + 2 * (size_t)b2 * PW + (size_t)b2 * b2) * sizeof(C<R>);
    if constexpr (std::is_same<R, double>::value && B2 >= 0) {
      // float64 in double-float arithmetic (GS_DF64 set: for every float64 apply)
      if ((dfl || std::getenv("GS_DF64")) && !norm_part && D.win) {
        gs_status e = set_smem_attr<R>((const void*)k_interp2d_df<W, B2>, sh);  // float4 per staged value
        if (e != GS_OK) return e;
        GS_LAUNCH("interp2d<df64>", st,
                  k_interp2d_df<W, B2><<<P->nwork, 128, sh, st>>>(P->work, P->work_order, P->fl, D.win, D.w, D.bf,
                                                                  D.grid, hb, D.side, (int)P->n, x, (int)P->N, P->M,
                                                                  P->nbx, tile, perm, y));
        GS_CUDA(cudaGetLastError());
        return GS_OK;
      }
    }
    gs_status e = set_smem_attr<R>((const void*)k_interp2d<R, W, B2>, sh);
    if (e != GS_OK) return e;
    GS_LAUNCH(pname<R>("interp2d<f32>", "interp2d<f64>"), st,
              k_interp2d<R, W, B2><<<P->nwork, 128, sh, st>>>(P->work, P->work_order, P->fl, D.frac, D.win, D.w, D.bf, b, D.grid,
                                                              hb, D.side, (int)P->n, (R)D.beta, x, (int)P->N,
                                                              P->M, P->nbx, tile, perm, y, norm_part));
    GS_CUDA(cudaGetLastError());
    return GS_OK;
  });
}

template <typename R>
gs_status launch_spread2d(Plan* P, PrecData<R>& D, const C<R>* u, const int32_t* perm, C<R>* part, cudaStream_t st) {
  using namespace dev;
  const int b = P->b, b2 = 2 * b, tile = P->tile;
  if (sizeof(R) == 4 && D.m == 4 && b2 == 8 && tile == 16 && D.part_stride == tc5::PART && !std::getenv("GS_NO_TC")) {
    const size_t sh = (size_t)tc5::N_SMEM * sizeof(float);
    gs_status e = set_smem_attr<R>((const void*)k_spread2d_tc5, sh);
    if (e != GS_OK) return e;
    // a programmatic dependent launch (unless P->pdl is off): the CTAs' set-up (TMEM,
    // barriers, operand buffers, table staging) overlaps the end of the kernel before it
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)P->nwork);
    cfg.blockDim = dim3(tc5::THREADS);
    cfg.dynamicSmemBytes = sh;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = P->pdl ? 1 : 0;
    GS_LAUNCH("spread2d<f32>", st,
              GS_CUDA(cudaLaunchKernelEx(&cfg, k_spread2d_tc5, P->work, P->work_order, P->fl, (const float*)D.win,
                                         (const float2*)D.w, (const float2*)D.bf, (const float2*)u, perm, P->M,
                                         P->nbx, (float2*)part, D.part_stride, P->flag + FL_TIMEOUT)));
    GS_CUDA(cudaGetLastError());
    return GS_OK;
  }
  return dispatch_wb(2 * D.m, b2, [&](auto wc, auto bc) -> gs_status {
    constexpr int W = decltype(wc)::value;
    constexpr int B2 = decltype(bc)::value;
    const int warps = 4;
    const int batch = sizeof(R) == 4 ? 64 : 32;
    const int PW = tile + W;
    const size_t wsz = (size_t)PW * PW + 2 * (size_t)b2 * PW;
    const size_t sh = ((size_t)warps * wsz + (size_t)warps * b2 * b2 + (size_t)batch * (3 + 2 * b2)) * sizeof(C<R>) +
                      (size_t)batch * (2 * W + 1) * sizeof(R) + (size_t)batch * 2 * sizeof(int) + 16;
    gs_status e = set_smem_attr<R>((const void*)k_spread2d<R, W, B2>, sh);
    if (e != GS_OK) return e;
    GS_LAUNCH(pname<R>("spread2d<f32>", "spread2d<f64>"), st,
              k_spread2d<R, W, B2><<<P->nwork, warps * 32, sh, st>>>(P->work, P->work_order, P->fl, D.frac, D.win, D.w, D.bf, b, u,
                                                                     perm, P->M, P->nbx, tile, (R)D.beta, batch, part,
                                                                     D.part_stride));
    GS_CUDA(cudaGetLastError());
    return GS_OK;
  });
}

}  // namespace gs
