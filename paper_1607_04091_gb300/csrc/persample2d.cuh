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

// window values of the W taps of sample s along dimension d: float32 from the
// plan's table, float64 evaluated exactly
template <typename R, int W> struct WinEval;
template <int W> struct WinEval<float, W> {
  static __device__ inline void get(const float* __restrict__ win, int64_t s, int d, float, float, float* out) {
    const float* p = win + ((int64_t)s * 2 + d) * W;
#pragma unroll
    for (int a = 0; a < W; ++a) out[a] = __ldg(p + a);
  }
};
template <int W> struct WinEval<double, W> {
  static __device__ inline void get(const double*, int64_t, int, double t, double beta, double* out) {
#pragma unroll
    for (int a = 0; a < W; ++a) out[a] = kb_window(t + (double)(W / 2 - 1 - a), W / 2, beta);
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
    const int32_t* __restrict__ work, const int32_t* __restrict__ fl, const R* __restrict__ frac,
    const R* __restrict__ win, const C<R>* __restrict__ w, const C<R>* __restrict__ bf, int b_rt,
    const C<R>* __restrict__ grid, const C<R>* __restrict__ hbuf, const C<R>* __restrict__ side, int n, R beta,
    const C<R>* __restrict__ x, int N, int64_t M, int nbx, int tile, const int32_t* __restrict__ perm,
    C<R>* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int m = W / 2;
  const int b2 = (B2 >= 0) ? B2 : 2 * b_rt;
  const int b = b2 / 2;
  const int PW = tile + W;  // staged row i <-> grid point o - m + 1 + i
  const int nm = n - 1;
  C<R>* G = reinterpret_cast<C<R>*>(smraw);
  C<R>* S0 = G + PW * PW;   // x-side k along y
  C<R>* S1 = S0 + b2 * PW;  // y-side k along x
  C<R>* XC = S1 + b2 * PW;  // corner coefficients [ky][kx]
  const int bin = work[3 * blockIdx.x], s0 = work[3 * blockIdx.x + 1], s1 = work[3 * blockIdx.x + 2];
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
    const int kx = t % b2, ky = t / b2;
    XC[t] = x[(int64_t)bcol(ky, b, N) * N + bcol(kx, b, N)];
  }
  __syncthreads();
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
    const int32_t* __restrict__ work, const int32_t* __restrict__ fl, const R* __restrict__ frac,
    const R* __restrict__ win, const C<R>* __restrict__ w, const C<R>* __restrict__ bf, int b_rt,
    const C<R>* __restrict__ u, const int32_t* __restrict__ perm, int64_t M, int nbx, int tile, R beta, int batch,
    C<R>* __restrict__ part, int64_t stride) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int b2 = (B2 >= 0) ? B2 : 2 * b_rt;
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
    cka[q] = (ch < b2 * b2) ? 3 + ch % b2 : 0;       // A[kx]
    ckb[q] = (ch < b2 * b2) ? 3 + b2 + ch / b2 : 0;  // conj(by[ky])
  }
  const int bin = work[3 * blockIdx.x], s0 = work[3 * blockIdx.x + 1], s1 = work[3 * blockIdx.x + 2];
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
  C<R>* out = part + blockIdx.x * stride;
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

// ---------------------------------------------------------------- tensor-core spread
// float32, W = 8 taps, 2b = 8 boundary columns, 16 x 16 tiles.  For one work item
// every output of the spread is a sum over its samples of outer products:
//   P[x][y]   += (v_s wx_s[x - px_s]) wy_s[y - py_s]      interior, v = u conj(wx wy)
//   S0[k][y]  += v0_s[k] wy_s[y - py_s]                    x-sides,  v0 = u conj(bx_k) conj(wy)
//   S1[k][x]  += v1_s[k] wx_s[x - px_s]                    y-sides,  v1 = u conj(wx) conj(by_k)
//   Cc[kx][ky]+= A_s[kx] conj(by_s[ky])                     corners,  A = u conj(bx)
// i.e. GEMMs with K = samples.  Phase 1 (thread per sample) writes a batch of 32
// samples as dense operand rows in shared memory; phase 2 accumulates the output
// tiles in registers with mma.sync m16n8k8 TF32 using the 3xTF32 split
// (a_hi b_hi + a_hi b_lo + a_lo b_hi, float32-level accuracy).  Output: the same
// partial-tile layout as k_spread2d.
namespace tc {
constexpr int SBT = 32;         // samples per batch (the K of one round)
constexpr int LD32 = 40;        // row stride of 32-wide operands (bank-conflict free fragments)
constexpr int LD16 = 24;        // row stride of 16- and 8-wide operands

__device__ inline uint32_t tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ inline void split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32(x);
  lo = tf32(x - __uint_as_float(hi));
}
__device__ inline void mma(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ inline void mma3(float* c, const uint32_t* ah, const uint32_t* al, const uint32_t* bh,
                            const uint32_t* bl) {
  mma(c, ah, bh);
  mma(c, ah, bl);
  mma(c, al, bh);
}
// A fragment (16 x 8, rows m0.., k-columns k0..) from an operand stored [k][m]
__device__ inline void load_a(const float* A, int ld, int m0, int k0, int lane, uint32_t* hi, uint32_t* lo) {
  const int g = lane >> 2, t = lane & 3;
  split(A[(k0 + t) * ld + m0 + g], hi[0], lo[0]);
  split(A[(k0 + t) * ld + m0 + g + 8], hi[1], lo[1]);
  split(A[(k0 + t + 4) * ld + m0 + g], hi[2], lo[2]);
  split(A[(k0 + t + 4) * ld + m0 + g + 8], hi[3], lo[3]);
}
// B fragment (8 x 8, k-rows k0.., columns n0..) from an operand stored [k][n]
__device__ inline void load_b(const float* B, int ld, int n0, int k0, int lane, uint32_t* hi, uint32_t* lo) {
  const int g = lane >> 2, t = lane & 3;
  split(B[(k0 + t) * ld + n0 + g], hi[0], lo[0]);
  split(B[(k0 + t + 4) * ld + n0 + g], hi[1], lo[1]);
}
}  // namespace tc

static __global__ void __launch_bounds__(128) k_spread2d_tc(
    const int32_t* __restrict__ work, const int32_t* __restrict__ fl, const float* __restrict__ win,
    const float2* __restrict__ w, const float2* __restrict__ bf, const float2* __restrict__ u,
    const int32_t* __restrict__ perm, int64_t M, int nbx, float2* __restrict__ part, int64_t stride) {
  using namespace tc;
  constexpr int W = 8, B2 = 8, TILE = 16, PW = TILE + W;
  extern __shared__ __align__(16) float sm[];
  float* Ar = sm;                    // [SBT][LD32]  (v wx) real part, rows x = px + a
  float* Ai = Ar + SBT * LD32;       // imaginary part
  float* By = Ai + SBT * LD32;       // wy at columns y = py + c
  float* Bx = By + SBT * LD32;       // wx at columns x = px + a
  float* V0r = Bx + SBT * LD32;      // [SBT][LD16] x-side coefficients
  float* V0i = V0r + SBT * LD16;
  float* V1r = V0i + SBT * LD16;     // y-side coefficients
  float* V1i = V1r + SBT * LD16;
  float* Kr = V1i + SBT * LD16;      // A = u conj(bx)
  float* Ki = Kr + SBT * LD16;
  float* Cr = Ki + SBT * LD16;       // conj(by)
  float* Ci = Cr + SBT * LD16;
  constexpr int NST = 4 * SBT * LD32 + 8 * SBT * LD16;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bin = work[3 * blockIdx.x], s0 = work[3 * blockIdx.x + 1], s1 = work[3 * blockIdx.x + 2];
  const int ox = (bin % nbx) * TILE, oy = (bin / nbx) * TILE;
  // accumulators: [re/im or second product][n-block 0..3][4]
  float acc[2][4][4];
  float cacc[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
      if (j < 2)
#pragma unroll
        for (int q = 0; q < 4; ++q) cacc[j][q] = 0.0f;
    }
  // operands start at zero; afterwards each thread clears only the windows it wrote
  for (int i = threadIdx.x; i < NST; i += blockDim.x) sm[i] = 0.0f;
  int prev_px = -1, prev_py = -1;
  for (int sb = s0; sb < s1; sb += SBT) {
    const int nb = min(SBT, s1 - sb);
    if (threadIdx.x < SBT && prev_px >= 0) {
      const int j = threadIdx.x;
#pragma unroll
      for (int a = 0; a < W; ++a) {
        Ar[j * LD32 + prev_px + a] = 0.0f;
        Ai[j * LD32 + prev_px + a] = 0.0f;
        Bx[j * LD32 + prev_px + a] = 0.0f;
        By[j * LD32 + prev_py + a] = 0.0f;
      }
      if (j >= nb) {  // no sample in this slot now: clear its boundary rows too
#pragma unroll
        for (int k = 0; k < B2; ++k) {
          V0r[j * LD16 + k] = V0i[j * LD16 + k] = V1r[j * LD16 + k] = V1i[j * LD16 + k] = 0.0f;
          Kr[j * LD16 + k] = Ki[j * LD16 + k] = Cr[j * LD16 + k] = Ci[j * LD16 + k] = 0.0f;
        }
      }
      prev_px = -1;
    }
    __syncthreads();
    if (threadIdx.x < nb) {
      const int j = threadIdx.x, s = sb + j;
      const float2 us = u[perm ? perm[s] : s];
      const int px = fl[s] - ox + 1, py = fl[M + s] - oy + 1;
      const float* wxp = win + ((int64_t)s * 2) * W;
      const float* wyp = wxp + W;
      const float2 wxs = w[s], wys = w[M + s];
      const float2 vi = cmulc(cmulc(us, wxs), wys);
      const float2 uwx = cmulc(us, wxs);
      prev_px = px;
      prev_py = py;
#pragma unroll
      for (int a = 0; a < W; ++a) {
        const float wa = __ldg(wxp + a), wc = __ldg(wyp + a);
        Ar[j * LD32 + px + a] = vi.x * wa;
        Ai[j * LD32 + px + a] = vi.y * wa;
        Bx[j * LD32 + px + a] = wa;
        By[j * LD32 + py + a] = wc;
      }
#pragma unroll
      for (int k = 0; k < B2; ++k) {
        const float2 bxk = bf[(int64_t)s * B2 + k], byk = bf[(M + s) * B2 + k];
        const float2 ak = cmulc(us, bxk);
        const float2 v0 = cmulc(ak, wys);
        const float2 v1 = cmulc(uwx, byk);
        V0r[j * LD16 + k] = v0.x;
        V0i[j * LD16 + k] = v0.y;
        V1r[j * LD16 + k] = v1.x;
        V1i[j * LD16 + k] = v1.y;
        Kr[j * LD16 + k] = ak.x;
        Ki[j * LD16 + k] = ak.y;
        Cr[j * LD16 + k] = byk.x;
        Ci[j * LD16 + k] = -byk.y;
      }
    }
    __syncthreads();
    // phase 2: warp 0/1 interior rows 0-15 / 16-31; warp 2 x-sides (+ corners with A = Kr);
    // warp 3 y-sides (+ corners with A = Ki)
    const float* A0 = (wid < 2) ? Ar : (wid == 2 ? V0r : V1r);
    const float* A1 = (wid < 2) ? Ai : (wid == 2 ? V0i : V1i);
    const int lda = (wid < 2) ? LD32 : LD16;
    const int m0 = (wid == 1) ? 16 : 0;
    const float* Bm = (wid == 3) ? Bx : By;
    const float* Ka = (wid == 2) ? Kr : Ki;
    for (int k0 = 0; k0 < SBT; k0 += 8) {
      uint32_t a0h[4], a0l[4], a1h[4], a1l[4];
      load_a(A0, lda, m0, k0, lane, a0h, a0l);
      load_a(A1, lda, m0, k0, lane, a1h, a1l);
#pragma unroll
      for (int nbk = 0; nbk < 4; ++nbk) {
        uint32_t bh[2], bl[2];
        load_b(Bm, LD32, nbk * 8, k0, lane, bh, bl);
        mma3(acc[0][nbk], a0h, a0l, bh, bl);
        mma3(acc[1][nbk], a1h, a1l, bh, bl);
      }
      if (wid >= 2) {
        uint32_t kh[4], kl[4], ch[2], cl[2];
        load_a(Ka, LD16, 0, k0, lane, kh, kl);
        load_b(Cr, LD16, 0, k0, lane, ch, cl);
        mma3(cacc[0], kh, kl, ch, cl);
        load_b(Ci, LD16, 0, k0, lane, ch, cl);
        mma3(cacc[1], kh, kl, ch, cl);
      }
    }
    __syncthreads();
  }
  // write the partial tile: P | S0 | S1 | corners
  const int g = lane >> 2, t = lane & 3;
  float2* out = part + blockIdx.x * stride;
  float* cs = sm;  // corner products exchanged between warps 2 and 3: [2 warps][2][16][8]
  if (wid < 2) {
#pragma unroll
    for (int nbk = 0; nbk < 4; ++nbk)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int x = (wid == 1 ? 16 : 0) + g + ((q & 2) ? 8 : 0), y = nbk * 8 + 2 * t + (q & 1);
        if (x < PW && y < PW) out[x * PW + y] = make_float2(acc[0][nbk][q], acc[1][nbk][q]);
      }
  } else {
    float2* S = out + PW * PW + (wid == 3 ? B2 * PW : 0);
#pragma unroll
    for (int nbk = 0; nbk < 4; ++nbk)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = g + ((q & 2) ? 8 : 0), c = nbk * 8 + 2 * t + (q & 1);
        if (k < B2 && c < PW) S[k * PW + c] = make_float2(acc[0][nbk][q], acc[1][nbk][q]);
      }
    // warp 2: Kr*Cr, Kr*Ci ; warp 3: Ki*Cr, Ki*Ci  (Ci holds -Im(by))
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int kx = g + ((q & 2) ? 8 : 0), ky = 2 * t + (q & 1);
        cs[(((wid - 2) * 2 + h) * 16 + kx) * 8 + ky] = cacc[h][q];
      }
  }
  __syncthreads();
  if (threadIdx.x < B2 * B2) {
    const int kx = threadIdx.x % B2, ky = threadIdx.x / B2;
    const float rr = cs[((0 * 2 + 0) * 16 + kx) * 8 + ky];  // Re(A) Re(conj by)
    const float ri = cs[((0 * 2 + 1) * 16 + kx) * 8 + ky];  // Re(A) Im(conj by)
    const float ir = cs[((1 * 2 + 0) * 16 + kx) * 8 + ky];  // Im(A) Re(conj by)
    const float ii = cs[((1 * 2 + 1) * 16 + kx) * 8 + ky];  // Im(A) Im(conj by)
    out[PW * PW + 2 * B2 * PW + kx + B2 * ky] = make_float2(rr - ii, ri + ir);
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
gs_status launch_interp2d(Plan* P, PrecData<R>& D, const C<R>* x, C<R>* y, const int32_t* perm, cudaStream_t st) {
  using namespace dev;
  const int b = P->b, b2 = 2 * b, tile = P->tile;
  if (P->nwork == 0) return GS_OK;
  return dispatch_wb(2 * D.m, b2, [&](auto wc, auto bc) -> gs_status {
    constexpr int W = decltype(wc)::value;
    constexpr int B2 = decltype(bc)::value;
    const int PW = tile + W;
    const size_t sh = ((size_t)PW * PW + 2 * (size_t)b2 * PW + (size_t)b2 * b2) * sizeof(C<R>);
    gs_status e = set_smem_attr<R>((const void*)k_interp2d<R, W, B2>, sh);
    if (e != GS_OK) return e;
    GS_LAUNCH(pname<R>("interp2d<f32>", "interp2d<f64>"), st,
              k_interp2d<R, W, B2><<<P->nwork, 128, sh, st>>>(P->work, P->fl, D.frac, D.win, D.w, D.bf, b, D.grid,
                                                              D.hbuf, D.side, (int)P->n, (R)D.beta, x, (int)P->N,
                                                              P->M, P->nbx, tile, perm, y));
    GS_CUDA(cudaGetLastError());
    return GS_OK;
  });
}

template <typename R>
gs_status launch_spread2d(Plan* P, PrecData<R>& D, const C<R>* u, const int32_t* perm, C<R>* part, cudaStream_t st) {
  using namespace dev;
  const int b = P->b, b2 = 2 * b, tile = P->tile;
  if (sizeof(R) == 4 && D.m == 4 && b2 == 8 && tile == 16 && !std::getenv("GS_NO_TC")) {
    const size_t sh = (size_t)(4 * tc::SBT * tc::LD32 + 8 * tc::SBT * tc::LD16) * sizeof(float);
    gs_status e = set_smem_attr<R>((const void*)k_spread2d_tc, sh);
    if (e != GS_OK) return e;
    GS_LAUNCH("spread2d<f32>", st,
              k_spread2d_tc<<<P->nwork, 128, sh, st>>>(P->work, P->fl, (const float*)D.win, (const float2*)D.w,
                                                       (const float2*)D.bf, (const float2*)u, perm, P->M, P->nbx,
                                                       (float2*)part, D.part_stride));
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
              k_spread2d<R, W, B2><<<P->nwork, warps * 32, sh, st>>>(P->work, P->fl, D.frac, D.win, D.w, D.bf, b, u,
                                                                     perm, P->M, P->nbx, tile, (R)D.beta, batch, part,
                                                                     D.part_stride));
    GS_CUDA(cudaGetLastError());
    return GS_OK;
  });
}

}  // namespace gs
