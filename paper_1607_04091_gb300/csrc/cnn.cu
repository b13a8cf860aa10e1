// Learned warm start: a residual CNN x0 = u + f(u) on the 2-channel image of
// the density-compensated adjoint u = T^H y (channel 0 real, 1 imaginary part;
// pixel (j, i) = coefficient i + N j).  f = L 3x3 convolutions (zero padding)
// with ReLU between them.  Training (float32 weights, Adam) and inference
// (bfloat16 weights, float32 accumulation) run in these kernels; the paper has no
// learned component, this is an addition beside the method.
//
// Layout: activations NCHW float32, weights [c_out][c_in][3][3] float32
// (+ a bfloat16 copy), biases [c_out].  H and W must be multiples of 16.  The
// convolutions and the weight gradient run on the tensor cores (bfloat16
// operands, float32 accumulation; see k_conv3_tc).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "gs_internal.h"

struct gs_cnn_s {
  int H = 0, W = 0, C = 0, L = 0, maxB = 0;
  std::vector<int> cin, cout;
  std::vector<int64_t> woff, boff;
  int64_t nw = 0, nb = 0;
  float *w = nullptr, *b = nullptr, *gw = nullptr, *gb = nullptr;
  float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
  float* wflip = nullptr;  // flipped / transposed weights for the input gradient
  __nv_bfloat16* wbf = nullptr;
  std::vector<float*> act;  // L + 1 activations, maxB x C_l x H x W
  float *g0 = nullptr, *g1 = nullptr;  // gradient ping-pong, maxB x Cmax x H x W
  float* part = nullptr;    // weight-gradient partials
  double* red = nullptr;    // loss partials
  int64_t part_cap = 0;
  int step = 0;
  bool bf_valid = false;
};

namespace gs {
namespace {

constexpr int TS = 16;      // pixel tile edge
constexpr int CI_CHUNK = 8; // input channels staged per pass

__device__ inline float wval(float v) { return v; }
__device__ inline float wval(__nv_bfloat16 v) { return __bfloat162float(v); }

// ---------------------------------------------------------------- tensor-core convolutions
// The 3x3 convolutions and the weight gradient are implicit GEMMs on the tensor
// cores (mma.sync m16n8k16, bfloat16 operands, float32 accumulation); operands
// are gathered from a staged input tile through a table of per-k offsets (no
// im2col buffer).  TERMS = 3 splits every operand x = hi + lo into two bfloat16
// (hi = x rounded, lo = the remainder rounded) and sums hi*hi + hi*lo + lo*hi,
// ~16 significant bits per product (training and the gradient check); TERMS = 1
// is the plain bfloat16 product (inference with bfloat16 weights).
namespace tcc {
constexpr int HALO = (TS + 2) * (TS + 2);  // staged input tile with its 1-pixel border
__device__ inline uint32_t pack(float lo_col, float hi_col) {  // two bf16, the lower k in the low half
  __nv_bfloat162 v = __floats2bfloat162_rn(lo_col, hi_col);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ inline void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}
__device__ inline void mma16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// offset in the staged tile of k = c * 9 + tap (tap = 3 dy + dx).  Beyond K (the
// padding of K to a multiple of 16): offset 0, a finite staged value, whose
// product meets a zero weight (convolution) or lands in an output column that is
// never stored (weight gradient).  Every gather adds at most 15 (TS + 2) + 15 to
// an offset, which keeps it inside the Cin x 18 x 18 staged tile.
__device__ inline int koffset(int k, int K) {
  return k < K ? (k / 9) * HALO + ((k % 9) / 3) * (TS + 2) + (k % 3) : 0;
}
__host__ __device__ inline int kpad(int K) { return (K + 15) & ~15; }
}  // namespace tcc

template <typename WT>
inline size_t conv_smem(int Cin, int CO, int terms) {
  const int K = Cin * 9, Kp = tcc::kpad(K), NP = (CO + 7) / 8 * 8;
  return (size_t)(Cin * tcc::HALO + 4) * sizeof(float) + (size_t)Kp * sizeof(int) +
         (size_t)NP * (Kp / 2) * sizeof(uint32_t) * (terms == 3 ? 2 : 1);
}

// out[b][o][y][x] = bias[o] + sum_c sum_t w[o][c][t] in[b][c][y+dy-1][x+dx-1] (ReLU optional).
// CTA = 16 x 16 pixels of one image, 8 warps; warp w takes pixel rows 2w, 2w + 1
// (one m16 tile each: M = the 16 pixels of a row), N = output channels, K = c x tap.
template <int CO, int TERMS, typename WT>
__global__ void __launch_bounds__(256) k_conv3_tc(const float* __restrict__ in, int Cin, const WT* __restrict__ w,
                                                  const float* __restrict__ bias, float* __restrict__ out, int H,
                                                  int W, int relu) {
  using namespace tcc;
  constexpr int NT = (CO + 7) / 8, NP = NT * 8;
  extern __shared__ __align__(16) unsigned char smc[];
  const int K = Cin * 9, Kp = kpad(K), KH = Kp / 2;
  float* sh = reinterpret_cast<float*>(smc);        // [Cin][18][18] (+4 floats of alignment)
  int* koff = reinterpret_cast<int*>(sh + Cin * HALO + 4);
  uint32_t* bh = reinterpret_cast<uint32_t*>(koff + Kp);  // [NP][Kp / 2] weight pairs, hi
  uint32_t* bl = bh + NP * KH;                            // lo (TERMS == 3)
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31, g = lane >> 2, tq = lane & 3;
  const int x0 = blockIdx.x * TS, y0 = blockIdx.y * TS, img = blockIdx.z;
  const float* inb = in + (int64_t)img * Cin * H * W;
  for (int i = tid; i < Cin * HALO; i += blockDim.x) {
    const int c = i / HALO, r = i - c * HALO;
    const int yy = y0 + r / (TS + 2) - 1, xx = x0 + r % (TS + 2) - 1;
    sh[i] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? inb[((int64_t)c * H + yy) * W + xx] : 0.0f;
  }
  for (int k = tid; k < Kp; k += blockDim.x) koff[k] = koffset(k, K);
  for (int i = tid; i < NP * KH; i += blockDim.x) {
    const int n = i / KH, kk = 2 * (i - n * KH);
    const float v0 = (n < CO && kk < K) ? wval(w[(int64_t)n * K + kk]) : 0.0f;
    const float v1 = (n < CO && kk + 1 < K) ? wval(w[(int64_t)n * K + kk + 1]) : 0.0f;
    if (TERMS == 3) split2(v0, v1, bh[i], bl[i]);
    else bh[i] = pack(v0, v1);
  }
  __syncthreads();
  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.0f;
  const int r0 = 2 * wid;
  for (int k0 = 0; k0 < Kp; k0 += 16) {
    const int ka = k0 + 2 * tq, kb = ka + 8;
    const int oa0 = koff[ka], oa1 = koff[ka + 1], ob0 = koff[kb], ob1 = koff[kb + 1];
    uint32_t wh[NT][2], wl[NT][2];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      wh[nt][0] = bh[(nt * 8 + g) * KH + ka / 2];
      wh[nt][1] = bh[(nt * 8 + g) * KH + kb / 2];
      if (TERMS == 3) {
        wl[nt][0] = bl[(nt * 8 + g) * KH + ka / 2];
        wl[nt][1] = bl[(nt * 8 + g) * KH + kb / 2];
      }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int base = (r0 + mt) * (TS + 2) + g;  // pixel (row r0 + mt, column g); + 8 for column g + 8
      const float e0 = sh[oa0 + base], e1 = sh[oa1 + base], e2 = sh[oa0 + base + 8], e3 = sh[oa1 + base + 8];
      const float e4 = sh[ob0 + base], e5 = sh[ob1 + base], e6 = sh[ob0 + base + 8], e7 = sh[ob1 + base + 8];
      uint32_t ah[4], al[4];
      if (TERMS == 3) {
        split2(e0, e1, ah[0], al[0]);
        split2(e2, e3, ah[1], al[1]);
        split2(e4, e5, ah[2], al[2]);
        split2(e6, e7, ah[3], al[3]);
      } else {
        ah[0] = pack(e0, e1);
        ah[1] = pack(e2, e3);
        ah[2] = pack(e4, e5);
        ah[3] = pack(e6, e7);
      }
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        mma16816(acc[mt][nt], ah, wh[nt]);
        if (TERMS == 3) {
          mma16816(acc[mt][nt], ah, wl[nt]);
          mma16816(acc[mt][nt], al, wh[nt]);
        }
      }
    }
  }
  float* ob = out + (int64_t)img * CO * H * W;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int o = nt * 8 + 2 * tq + (q & 1), px = g + ((q & 2) ? 8 : 0);
        if (o >= CO) continue;
        float v = acc[mt][nt][q] + (bias ? bias[o] : 0.0f);
        if (relu) v = fmaxf(v, 0.0f);
        ob[((int64_t)o * H + y0 + r0 + mt) * W + x0 + px] = v;
      }
}

// wflip[c][o][t] = w[o][c][8 - t]: the input gradient is the convolution of the
// output gradient with these weights (c_out and c_in swapped, taps reversed)
__global__ void k_flip(const float* __restrict__ w, int Cout, int Cin, float* __restrict__ wf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Cout * Cin * 9) return;
  const int o = i / (Cin * 9), r = i % (Cin * 9), c = r / 9, t = r % 9;
  wf[((int64_t)c * Cout + o) * 9 + (8 - t)] = w[i];
}

// g *= (act > 0)
__global__ void k_relu_mask(float* __restrict__ g, const float* __restrict__ act, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!(act[i] > 0.0f)) g[i] = 0.0f;
}

// weight-gradient partials of one band of 16 rows of one image:
// part[band][o][c][t] = sum_{pixels} g[o][y][x] in[c][y+dy-1][x+dx-1], a GEMM with
// M = c_out, N = c_in x tap, K = the band's pixels (16 per MMA step: one row of a
// 16 x 16 tile), 3xBF16.  9 warps; warp w takes the n8 tiles w, w + 9, w + 18, w + 27.
constexpr int WG_WARPS = 9;
inline size_t wgrad_smem(int Cin, int Cout) {
  const int MP = Cout <= 16 ? 16 : 32, NP = (Cin * 9 + 7) / 8 * 8;
  return (size_t)(Cin * tcc::HALO + 4) * sizeof(float) + (size_t)NP * sizeof(int) +
         (size_t)MP * (TS * TS / 2) * sizeof(uint32_t) * 2;
}
__global__ void __launch_bounds__(WG_WARPS * 32) k_wgrad_tc(const float* __restrict__ in, int Cin,
                                                            const float* __restrict__ g, int Cout, int H, int W,
                                                            float* __restrict__ part) {
  using namespace tcc;
  extern __shared__ __align__(16) unsigned char smc[];
  const int K = Cin * 9, NT = (K + 7) / 8, NP = NT * 8, MT = Cout <= 16 ? 1 : 2, MP = 16 * MT;
  constexpr int PH = TS * TS / 2;                   // pixel pairs of a tile
  float* sh = reinterpret_cast<float*>(smc);        // [Cin][18][18] (+4 floats of alignment)
  int* noff = reinterpret_cast<int*>(sh + Cin * HALO + 4);
  uint32_t* gh = reinterpret_cast<uint32_t*>(noff + NP);  // [MP][PH] gradient pairs, hi
  uint32_t* gl = gh + MP * PH;                            // lo
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
  const int band = blockIdx.x, img = blockIdx.y, y0 = band * TS;
  const float* inb = in + (int64_t)img * Cin * H * W;
  const float* gb = g + (int64_t)img * Cout * H * W;
  for (int n = tid; n < NP; n += blockDim.x) noff[n] = koffset(n, K);
  float acc[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[mt][j][q] = 0.0f;
  for (int x0 = 0; x0 < W; x0 += TS) {
    __syncthreads();
    for (int i = tid; i < Cin * HALO; i += blockDim.x) {
      const int c = i / HALO, r = i - c * HALO;
      const int yy = y0 + r / (TS + 2) - 1, xx = x0 + r % (TS + 2) - 1;
      sh[i] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? inb[((int64_t)c * H + yy) * W + xx] : 0.0f;
    }
    for (int i = tid; i < MP * PH; i += blockDim.x) {
      const int o = i / PH, pp = i - o * PH, p = 2 * pp;
      float v0 = 0.0f, v1 = 0.0f;
      if (o < Cout) {
        const float* row = gb + ((int64_t)o * H + y0 + p / TS) * W + x0 + p % TS;
        v0 = row[0];
        v1 = row[1];
      }
      split2(v0, v1, gh[i], gl[i]);
    }
    __syncthreads();
    for (int r = 0; r < TS; ++r) {  // K step: the 16 pixels of tile row r
      uint32_t ah[2][4], al[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        if (mt >= MT) break;
        const int o = mt * 16 + gq, pa = (r * TS + 2 * tq) / 2, pb = pa + 4;
        ah[mt][0] = gh[o * PH + pa];
        al[mt][0] = gl[o * PH + pa];
        ah[mt][1] = gh[(o + 8) * PH + pa];
        al[mt][1] = gl[(o + 8) * PH + pa];
        ah[mt][2] = gh[o * PH + pb];
        al[mt][2] = gl[o * PH + pb];
        ah[mt][3] = gh[(o + 8) * PH + pb];
        al[mt][3] = gl[(o + 8) * PH + pb];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int nt = wid + WG_WARPS * j;
        if (nt >= NT) break;
        const int off = noff[nt * 8 + gq] + r * (TS + 2) + 2 * tq;  // pixels 2 tq, 2 tq + 1 (+ 8) of row r
        uint32_t bh[2], bl[2];
        split2(sh[off], sh[off + 1], bh[0], bl[0]);
        split2(sh[off + 8], sh[off + 9], bh[1], bl[1]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          if (mt >= MT) break;
          mma16816(acc[mt][j], ah[mt], bh);
          mma16816(acc[mt][j], ah[mt], bl);
          mma16816(acc[mt][j], al[mt], bh);
        }
      }
    }
  }
  float* pout = part + ((int64_t)img * gridDim.x + band) * (int64_t)Cout * K;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    if (mt >= MT) break;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nt = wid + WG_WARPS * j;
      if (nt >= NT) break;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int o = mt * 16 + gq + ((q & 2) ? 8 : 0), n = nt * 8 + 2 * tq + (q & 1);
        if (o < Cout && n < K) pout[(int64_t)o * K + n] = acc[mt][j][q];
      }
    }
  }
}

// gw[i] = sum over partials (fixed order)
__global__ void k_sum_parts(const float* __restrict__ part, int nparts, int64_t n, float* __restrict__ gw) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.0f;
  for (int k = 0; k < nparts; ++k) s += part[(int64_t)k * n + i];
  gw[i] = s;
}

// gb[o] = sum_b sum_pixels g[b][o][:]
__global__ void k_bgrad(const float* __restrict__ g, int B, int Cout, int64_t HW, float* __restrict__ gb) {
  __shared__ float red[256];
  const int o = blockIdx.x;
  float s = 0.0f;
  for (int b = 0; b < B; ++b)
    for (int64_t i = threadIdx.x; i < HW; i += blockDim.x) s += g[((int64_t)b * Cout + o) * HW + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) gb[o] = red[0];
}

// x0 = u + f; g = 2 (x0 - target) / n; loss partials
__global__ void k_loss(const float* __restrict__ u, const float* __restrict__ f, const float* __restrict__ tgt,
                       int64_t n, float* __restrict__ g, double* __restrict__ red) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = u[i] + f[i] - tgt[i];
    g[i] = 2.0f * d / (float)n;
    s += (double)d * d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) red[blockIdx.x] = sh[0];
}

__global__ void k_residual(const float* __restrict__ u, const float* __restrict__ f, float* __restrict__ x0,
                           int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x0[i] = u[i] + f[i];
}

// Adam (Kingma-Ba) with bias correction
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float c1, float c2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ o, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) o[i] = __float2bfloat16(w[i]);
}

// He-uniform weights U(-sqrt(6/fan_in), +) from a splitmix64 hash of (seed, index);
// the last layer starts at zero so that the untrained network is x0 = u
__global__ void k_init(float* __restrict__ w, int64_t n, int64_t off, int fan_in, uint64_t seed, int zero) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(off + i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const double uni = (double)(z >> 11) * (1.0 / 9007199254740992.0);  // [0, 1)
  const double a = sqrt(6.0 / (double)fan_in);
  w[i] = zero ? 0.0f : (float)((2.0 * uni - 1.0) * a);
}

inline int blocks(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

// bfloat16 weights (inference): one bfloat16 product; float32 weights (training,
// gradients): the three-term split
template <typename WT> constexpr int conv_terms() { return std::is_same<WT, __nv_bfloat16>::value ? 1 : 3; }

template <int CO, typename WT>
gs_status conv_launch(const float* in, int Cin, const WT* w, const float* bias, float* out, int B, int H, int W,
                      int relu, cudaStream_t st) {
  constexpr int TERMS = conv_terms<WT>();
  const size_t sh = conv_smem<WT>(Cin, CO, TERMS);
  if (sh > 48 * 1024)
    GS_CUDA(cudaFuncSetAttribute((const void*)k_conv3_tc<CO, TERMS, WT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sh));
  dim3 grid(W / TS, H / TS, B);
  GS_LAUNCH("cnn_conv3", st, k_conv3_tc<CO, TERMS, WT><<<grid, 256, sh, st>>>(in, Cin, w, bias, out, H, W, relu));
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

template <typename WT>
gs_status conv(const float* in, int Cin, const WT* w, const float* bias, float* out, int Cout, int B, int H, int W,
               int relu, cudaStream_t st) {
  switch (Cout) {
    case 2: return conv_launch<2, WT>(in, Cin, w, bias, out, B, H, W, relu, st);
    case 8: return conv_launch<8, WT>(in, Cin, w, bias, out, B, H, W, relu, st);
    case 16: return conv_launch<16, WT>(in, Cin, w, bias, out, B, H, W, relu, st);
    case 32: return conv_launch<32, WT>(in, Cin, w, bias, out, B, H, W, relu, st);
  }
  set_error("convolution with %d output channels has no compiled kernel (2, 8, 16, 32)", Cout);
  return GS_EUNSUPPORTED;
}

template <typename T>
gs_status dalloc(T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, (count ? count : 1) * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    return GS_ENOMEM;
  }
  return GS_OK;
}

// forward through all layers with float32 weights, keeping activations
gs_status forward_train(gs_cnn_s* N, const float* u, int B, cudaStream_t st) {
  const int64_t img = (int64_t)2 * N->H * N->W * B;
  GS_CUDA(cudaMemcpyAsync(N->act[0], u, img * sizeof(float), cudaMemcpyDeviceToDevice, st));
  for (int l = 0; l < N->L; ++l)
    GS_TRY(conv<float>(N->act[l], N->cin[l], N->w + N->woff[l], N->b + N->boff[l], N->act[l + 1], N->cout[l], B,
                       N->H, N->W, l < N->L - 1, st));
  return GS_OK;
}

// loss and gradients (gw, gb) for a batch; loss into *loss (host)
gs_status backward(gs_cnn_s* N, const float* u, const float* tgt, int B, double* loss, cudaStream_t st) {
  GS_TRY(forward_train(N, u, B, st));
  const int64_t HW = (int64_t)N->H * N->W, n = 2 * HW * B;
  const int nbk = 256;
  GS_LAUNCH("cnn_loss", st, k_loss<<<nbk, 256, 0, st>>>(u, N->act[N->L], tgt, n, N->g0, N->red));
  float* g = N->g0;
  float* gnext = N->g1;
  for (int l = N->L - 1; l >= 0; --l) {
    const int Ci = N->cin[l], Co = N->cout[l];
    if (l < N->L - 1) GS_LAUNCH("cnn_relu_mask", st, k_relu_mask<<<blocks(B * Co * HW), 256, 0, st>>>(g, N->act[l + 1], (int64_t)B * Co * HW));
    const int nbands = N->H / TS;
    const int64_t nwl = (int64_t)Co * Ci * 9;
    const size_t shw = wgrad_smem(Ci, Co);
    if (shw > 48 * 1024)
      GS_CUDA(cudaFuncSetAttribute((const void*)k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shw));
    GS_LAUNCH("cnn_wgrad", st, k_wgrad_tc<<<dim3(nbands, B), WG_WARPS * 32, shw, st>>>(N->act[l], Ci, g, Co, N->H, N->W,
                                                                                      N->part));
    GS_LAUNCH("cnn_wgrad_sum", st, k_sum_parts<<<blocks(nwl), 256, 0, st>>>(N->part, nbands * B, nwl, N->gw + N->woff[l]));
    GS_LAUNCH("cnn_bgrad", st, k_bgrad<<<Co, 256, 0, st>>>(g, B, Co, HW, N->gb + N->boff[l]));
    if (l > 0) {
      GS_LAUNCH("cnn_flip", st, k_flip<<<blocks(nwl), 256, 0, st>>>(N->w + N->woff[l], Co, Ci, N->wflip));
      GS_TRY(conv<float>(g, Co, N->wflip, nullptr, gnext, Ci, B, N->H, N->W, 0, st));
      std::swap(g, gnext);
    }
  }
  std::vector<double> hred(nbk);
  GS_CUDA(cudaMemcpyAsync(hred.data(), N->red, nbk * sizeof(double), cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));
  double s = 0.0;
  for (double v : hred) s += v;
  *loss = s / (double)n;
  return GS_OK;
}

void free_net(gs_cnn_s* N) {
  void* ps[] = {N->w, N->b, N->gw, N->gb, N->mw, N->vw, N->mb, N->vb, N->wflip, N->wbf, N->g0, N->g1, N->part,
                N->red};
  for (void* p : ps)
    if (p) cudaFree(p);
  for (float* a : N->act)
    if (a) cudaFree(a);
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_cnn_create(gs_cnn* out, int H, int W, int channels, int depth, int max_batch, uint64_t seed,
                        void* stream) {
  if (!out || H < 16 || W < 16 || H % 16 || W % 16 || depth < 2 || depth > 16 || max_batch < 1 ||
      (channels != 8 && channels != 16 && channels != 32)) {
    set_error("gs_cnn_create: need H, W multiples of 16, channels in {8, 16, 32}, 2 <= depth <= 16, max_batch >= 1");
    return GS_EINVAL;
  }
  *out = nullptr;
  gs_cnn_s* N = new (std::nothrow) gs_cnn_s();
  if (!N) return GS_ENOMEM;
  N->H = H;
  N->W = W;
  N->C = channels;
  N->L = depth;
  N->maxB = max_batch;
  for (int l = 0; l < depth; ++l) {
    N->cin.push_back(l == 0 ? 2 : channels);
    N->cout.push_back(l == depth - 1 ? 2 : channels);
    N->woff.push_back(N->nw);
    N->boff.push_back(N->nb);
    N->nw += (int64_t)N->cin[l] * N->cout[l] * 9;
    N->nb += N->cout[l];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t HW = (int64_t)H * W;
  gs_status s = GS_OK;
  auto A = [&](gs_status r) {
    if (s == GS_OK) s = r;
  };
  A(dalloc(&N->w, N->nw));
  A(dalloc(&N->b, N->nb));
  A(dalloc(&N->gw, N->nw));
  A(dalloc(&N->gb, N->nb));
  A(dalloc(&N->mw, N->nw));
  A(dalloc(&N->vw, N->nw));
  A(dalloc(&N->mb, N->nb));
  A(dalloc(&N->vb, N->nb));
  A(dalloc(&N->wflip, (size_t)channels * channels * 9));
  A(dalloc(&N->wbf, N->nw));
  N->act.assign(depth + 1, nullptr);
  for (int l = 0; l <= depth; ++l) A(dalloc(&N->act[l], (size_t)max_batch * (l == 0 ? 2 : N->cout[l - 1]) * HW));
  A(dalloc(&N->g0, (size_t)max_batch * channels * HW));
  A(dalloc(&N->g1, (size_t)max_batch * channels * HW));
  N->part_cap = (int64_t)(H / 16) * max_batch * channels * channels * 9;
  A(dalloc(&N->part, (size_t)N->part_cap));
  A(dalloc(&N->red, 256));
  if (s != GS_OK) {
    free_net(N);
    delete N;
    return s;
  }
  cudaMemsetAsync(N->b, 0, N->nb * sizeof(float), st);
  cudaMemsetAsync(N->mw, 0, N->nw * sizeof(float), st);
  cudaMemsetAsync(N->vw, 0, N->nw * sizeof(float), st);
  cudaMemsetAsync(N->mb, 0, N->nb * sizeof(float), st);
  cudaMemsetAsync(N->vb, 0, N->nb * sizeof(float), st);
  for (int l = 0; l < depth; ++l) {
    const int64_t nwl = (int64_t)N->cin[l] * N->cout[l] * 9;
    k_init<<<blocks(nwl), 256, 0, st>>>(N->w + N->woff[l], nwl, N->woff[l], N->cin[l] * 9, seed, l == depth - 1);
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_net(N);
    delete N;
    return cuda_fail(e, "gs_cnn_create");
  }
  *out = N;
  return GS_OK;
}

void gs_cnn_destroy(gs_cnn net) {
  if (!net) return;
  cudaDeviceSynchronize();
  free_net(net);
  delete net;
}

gs_status gs_cnn_forward(gs_cnn N, const float* u, float* x0, int B, int use_bf16, void* stream) {
  if (!N || !u || !x0 || B < 1 || B > N->maxB) {
    set_error("gs_cnn_forward: bad arguments (1 <= B <= max_batch)");
    return GS_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (use_bf16 && !N->bf_valid) {
    k_to_bf16<<<blocks(N->nw), 256, 0, st>>>(N->w, N->wbf, N->nw);
    GS_CUDA(cudaGetLastError());
    N->bf_valid = true;
  }
  const float* h = u;
  for (int l = 0; l < N->L; ++l) {
    gs_status s = use_bf16 ? conv<__nv_bfloat16>(h, N->cin[l], N->wbf + N->woff[l], N->b + N->boff[l],
                                                  N->act[l + 1], N->cout[l], B, N->H, N->W, l < N->L - 1, st)
                           : conv<float>(h, N->cin[l], N->w + N->woff[l], N->b + N->boff[l], N->act[l + 1],
                                         N->cout[l], B, N->H, N->W, l < N->L - 1, st);
    if (s != GS_OK) return s;
    h = N->act[l + 1];
  }
  const int64_t n = (int64_t)2 * N->H * N->W * B;
  GS_LAUNCH("cnn_residual", st, k_residual<<<blocks(n), 256, 0, st>>>(u, N->act[N->L], x0, n));
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

gs_status gs_cnn_gradients(gs_cnn N, const float* u, const float* target, int B, float* grad_host, double* loss) {
  if (!N || !u || !target || B < 1 || B > N->maxB) {
    set_error("gs_cnn_gradients: bad arguments");
    return GS_EINVAL;
  }
  double l = 0.0;
  gs_status s = backward(N, u, target, B, &l, 0);
  if (s != GS_OK) return s;
  if (grad_host) {
    GS_CUDA(cudaMemcpy(grad_host, N->gw, N->nw * sizeof(float), cudaMemcpyDeviceToHost));
    GS_CUDA(cudaMemcpy(grad_host + N->nw, N->gb, N->nb * sizeof(float), cudaMemcpyDeviceToHost));
  }
  if (loss) *loss = l;
  return GS_OK;
}

gs_status gs_cnn_train_step(gs_cnn N, const float* u, const float* target, int B, float lr, double* loss,
                            void* stream) {
  if (!N || !u || !target || B < 1 || B > N->maxB || !(lr > 0.0f)) {
    set_error("gs_cnn_train_step: bad arguments");
    return GS_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double l = 0.0;
  gs_status s = backward(N, u, target, B, &l, st);
  if (s != GS_OK) return s;
  N->step += 1;
  const float c1 = 1.0f - powf(0.9f, (float)N->step), c2 = 1.0f - powf(0.999f, (float)N->step);
  GS_LAUNCH("cnn_adam", st, k_adam<<<blocks(N->nw), 256, 0, st>>>(N->w, N->gw, N->mw, N->vw, N->nw, lr, c1, c2));
  GS_LAUNCH("cnn_adam", st, k_adam<<<blocks(N->nb), 256, 0, st>>>(N->b, N->gb, N->mb, N->vb, N->nb, lr, c1, c2));
  GS_CUDA(cudaGetLastError());
  N->bf_valid = false;
  if (loss) *loss = l;
  return GS_OK;
}

gs_status gs_cnn_weights(gs_cnn N, float* host, int64_t* count) {
  if (!N || !count) {
    set_error("gs_cnn_weights: bad arguments");
    return GS_EINVAL;
  }
  *count = N->nw + N->nb;
  if (host) {
    GS_CUDA(cudaMemcpy(host, N->w, N->nw * sizeof(float), cudaMemcpyDeviceToHost));
    GS_CUDA(cudaMemcpy(host + N->nw, N->b, N->nb * sizeof(float), cudaMemcpyDeviceToHost));
  }
  return GS_OK;
}

gs_status gs_cnn_set_weights(gs_cnn N, const float* host, int64_t count) {
  if (!N || !host || count != N->nw + N->nb) {
    set_error("gs_cnn_set_weights: need %lld values", N ? (long long)(N->nw + N->nb) : 0LL);
    return GS_EINVAL;
  }
  GS_CUDA(cudaMemcpy(N->w, host, N->nw * sizeof(float), cudaMemcpyHostToDevice));
  GS_CUDA(cudaMemcpy(N->b, host + N->nw, N->nb * sizeof(float), cudaMemcpyHostToDevice));
  N->bf_valid = false;
  return GS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- learned solve
namespace gs {
namespace {

// sum |v|^2 of n complex64 values into out[0] (one block, fixed order)
__global__ void k_sq1(const float2* __restrict__ v, int64_t n, double* __restrict__ out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)v[i].x * v[i].x + (double)v[i].y * v[i].y;
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

// coefficients (complex64, i + N j) -> image [2][N][N] / s, s = rms of the image
__global__ void k_coef_to_image(const float2* __restrict__ u, int64_t n, const double* __restrict__ sq,
                                float* __restrict__ img, float* __restrict__ scale) {
  const double s = sqrt(sq[0] / (2.0 * (double)n));
  const float inv = s > 0.0 ? (float)(1.0 / s) : 0.0f;
  if (blockIdx.x == 0 && threadIdx.x == 0) scale[0] = (float)s;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    img[i] = u[i].x * inv;
    img[n + i] = u[i].y * inv;
  }
}

// image [2][N][N] * s -> coefficients (complex128)
__global__ void k_image_to_coef(const float* __restrict__ img, int64_t n, const float* __restrict__ scale,
                                double2* __restrict__ x) {
  const double s = scale[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = make_double2(s * img[i], s * img[n + i]);
}

__global__ void k_c128_to_c64(const double2* __restrict__ a, float2* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}


}  // namespace
}  // namespace gs

namespace gs {
namespace {
// x = rms(u) * net(u / rms(u)), u = T^H y (float32 adjoint): the learned start
gs_status learned_start(gs_plan plan, gs_cnn net, const void* y, void* x, cudaStream_t st) {
  if (!plan || !net || !y || !x) {
    set_error("learned start: plan, net, y and x must be non-NULL");
    return GS_EINVAL;
  }
  Plan* P = &plan->P;
  gs_cnn_s* N = net;
  if (P->dims != 2 || N->H != P->N || N->W != P->N) {
    set_error("learned start: the network's image (%d x %d) must be the plan's 2D coefficient grid (%lld)", N->H,
              N->W, (long long)P->N);
    return GS_EINVAL;
  }
  const int64_t nc = P->ncoef, M = P->M;
  PrecData<float>& F = P->f;
  // u = T^H y (float32), its image scaled to unit rms
  GS_TRY(gather_sorted<double>(P, (const double2*)y, (double2*)P->y64, st));
  k_c128_to_c64<<<blocks(M), 256, 0, st>>>((const double2*)P->y64, F.vr, M);
  GS_TRY(apply_TH<float>(P, F, F.vr, F.vs, nullptr, st));
  double* sq = P->scal + 40;  // scratch slots beyond the solver's
  float* img_in = N->g0;      // network buffers serve as staging (2 N^2 floats each)
  float* img_out = N->g1;
  float* scale = reinterpret_cast<float*>(P->scal + 42);
  k_sq1<<<1, 1024, 0, st>>>(F.vs, nc, sq);
  k_coef_to_image<<<blocks(nc), 256, 0, st>>>(F.vs, nc, sq, img_in, scale);
  GS_CUDA(cudaGetLastError());
  GS_TRY(gs_cnn_forward(N, img_in, img_out, 1, 1, st));
  k_image_to_coef<<<blocks(nc), 256, 0, st>>>(img_out, nc, scale, (double2*)x);
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}
}  // namespace
}  // namespace gs

extern "C" gs_status gs_solve_learned(gs_plan plan, gs_cnn net, const void* y, void* x, const gs_solve_opts* opts,
                                      gs_solve_info* info, int* used_warm_start, void* stream) {
  GS_TRY(learned_start(plan, net, y, x, (cudaStream_t)stream));
  Plan* P = &plan->P;
  // solve from x0; the solve keeps x0 only if ||T^H (y - T x0)|| < ||T^H y|| (else zero start)
  gs_solve_opts o = {1e-6, 1000, GS_SOLVE_MIXED, 0, 8, 0.0};
  if (opts) o = *opts;
  o.x0_given = 1;
  gs_status r = gs_solve(plan, y, x, &o, info, stream);
  if (used_warm_start) {
    double w = 1.0;
    cudaMemcpy(&w, P->scal + 32, sizeof(double), cudaMemcpyDeviceToHost);  // the solver's kept-start flag
    *used_warm_start = (w != 0.0) ? 1 : 0;
  }
  return r;
}

extern "C" gs_status gs_solve_batch_learned(const gs_plan* plans, int B, gs_cnn net, const void* const* y,
                                            void* const* x, const gs_solve_opts* opts, gs_solve_info* infos,
                                            void* stream) {
  if (!plans || !y || !x || B < 1 || !net) {
    set_error("gs_solve_batch_learned: need plans, net, y, x non-NULL and B >= 1");
    return GS_EINVAL;
  }
  for (int i = 0; i < B; ++i) GS_TRY(learned_start(plans[i], net, y[i], x[i], (cudaStream_t)stream));
  gs_solve_opts o = {1e-6, 1000, GS_SOLVE_MIXED, 0, 8, 0.0};
  if (opts) o = *opts;
  o.x0_given = 1;
  return gs_solve_batch(plans, B, y, x, &o, infos, stream);
}

extern "C" gs_status gs_cnn_pair(gs_plan plan, const void* y, const void* x, float* u_img, float* x_img,
                                 void* stream) {
  if (!plan || !y || !u_img) {
    set_error("gs_cnn_pair: plan, y and u_img must be non-NULL");
    return GS_EINVAL;
  }
  Plan* P = &plan->P;
  if (P->dims != 2) {
    set_error("gs_cnn_pair: 2D plans only");
    return GS_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nc = P->ncoef, M = P->M;
  PrecData<float>& F = P->f;
  GS_TRY(gather_sorted<double>(P, (const double2*)y, (double2*)P->y64, st));
  k_c128_to_c64<<<blocks(M), 256, 0, st>>>((const double2*)P->y64, F.vr, M);
  GS_TRY(apply_TH<float>(P, F, F.vr, F.vs, nullptr, st));
  double* sq = P->scal + 40;
  float* scale = reinterpret_cast<float*>(P->scal + 42);
  k_sq1<<<1, 1024, 0, st>>>(F.vs, nc, sq);
  k_coef_to_image<<<blocks(nc), 256, 0, st>>>(F.vs, nc, sq, u_img, scale);
  if (x && x_img) {
    k_c128_to_c64<<<blocks(nc), 256, 0, st>>>((const double2*)x, F.vz, nc);
    k_coef_to_image<<<blocks(nc), 256, 0, st>>>(F.vz, nc, sq, x_img, scale);  // same scale as u
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}
