// 2D Voronoi density weights and the density delta (App. B, eq.
// Voronoi_tesselation): the weight of sample xi_m is the area of its Voronoi cell
// within Y_K = [-K, K]^2, and delta = sup over Y_K of the distance to the nearest
// sample, attained at a vertex of some cell.
//
// One thread per sample builds its cell by clipping the square with the
// bisector half-plane |x - xi_m| <= |x - xi_j| of nearby samples j, found through
// a uniform bucket grid visited in rings of growing Chebyshev distance.  After
// ring r every unvisited sample is at least r h away (h the bucket size), and a
// sample can cut the cell only if it lies within twice the cell's largest vertex
// distance R of xi_m, so the search stops once r h >= 2 R: the cell is exact, not
// a k-nearest-neighbour approximation.  All arithmetic is float64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gs_internal.h"

namespace gs {
namespace {

constexpr int VMAX = 64;  // vertices of a cell at most (a Voronoi cell has ~6 on average)

__global__ void k_voronoi2d(const double2* __restrict__ pts, const int32_t* __restrict__ cell_start,
                            const int32_t* __restrict__ order, int64_t M, int G, double K, double h,
                            double* __restrict__ mu, double* __restrict__ rmax, int* __restrict__ err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  double px[2][VMAX], py[2][VMAX];
  int cur = 0, nv = 4;
  px[0][0] = -K, py[0][0] = -K;
  px[0][1] = K, py[0][1] = -K;
  px[0][2] = K, py[0][2] = K;
  px[0][3] = -K, py[0][3] = K;
  const double2 s = pts[i];
  const int bi = min(G - 1, max(0, (int)floor((s.x + K) / h)));
  const int bj = min(G - 1, max(0, (int)floor((s.y + K) / h)));
  bool overflow = false;
  for (int r = 0; r < G; ++r) {
    // stop once every unvisited sample is at least twice the cell's reach away
    double R2 = 0.0;
    for (int v = 0; v < nv; ++v) {
      const double dx = px[cur][v] - s.x, dy = py[cur][v] - s.y;
      R2 = fmax(R2, dx * dx + dy * dy);
    }
    if (r >= 1 && (double)(r - 1) * h * ((double)(r - 1) * h) >= 4.0 * R2) break;
    for (int cj = bj - r; cj <= bj + r; ++cj) {
      if (cj < 0 || cj >= G) continue;
      const bool edge_row = (cj == bj - r || cj == bj + r);
      for (int ci = bi - r; ci <= bi + r; ci += (edge_row || r == 0) ? 1 : 2 * r) {
        if (ci < 0 || ci >= G) continue;
        const int c = cj * G + ci;
        for (int q = cell_start[c]; q < cell_start[c + 1]; ++q) {
          const int64_t j = order[q];
          if (j == i || nv == 0) continue;
          const double2 t = pts[j];
          // |x - s|^2 <= |x - t|^2  <=>  2 (t - s) . x <= |t|^2 - |s|^2
          const double a = 2.0 * (t.x - s.x), b = 2.0 * (t.y - s.y);
          const double cc = (t.x * t.x + t.y * t.y) - (s.x * s.x + s.y * s.y);
          const int nx = cur ^ 1;
          int m = 0;
          for (int v = 0; v < nv; ++v) {
            const int w = (v + 1 == nv) ? 0 : v + 1;
            const double fp = a * px[cur][v] + b * py[cur][v] - cc;
            const double fq = a * px[cur][w] + b * py[cur][w] - cc;
            if (fp <= 0.0) {
              if (m < VMAX) px[nx][m] = px[cur][v], py[nx][m] = py[cur][v];
              ++m;
            }
            if ((fp < 0.0 && fq > 0.0) || (fq < 0.0 && fp > 0.0)) {
              const double u = fp / (fp - fq);
              if (m < VMAX) {
                px[nx][m] = px[cur][v] + u * (px[cur][w] - px[cur][v]);
                py[nx][m] = py[cur][v] + u * (py[cur][w] - py[cur][v]);
              }
              ++m;
            }
          }
          if (m > VMAX) {
            overflow = true;
            m = VMAX;
          }
          nv = m;
          cur = nx;
        }
      }
    }
  }
  double area = 0.0, R2 = 0.0;
  for (int v = 0; v < nv; ++v) {
    const int w = (v + 1 == nv) ? 0 : v + 1;
    area += px[cur][v] * py[cur][w] - px[cur][w] * py[cur][v];
    const double dx = px[cur][v] - s.x, dy = py[cur][v] - s.y;
    R2 = fmax(R2, dx * dx + dy * dy);
  }
  mu[i] = nv >= 3 ? 0.5 * fabs(area) : 0.0;
  rmax[i] = sqrt(R2);
  if (overflow) atomicExch(err, 1);
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_voronoi_2d(const double* xi, int64_t M, double K, double* mu, double* delta, void* stream) {
  if (!xi || !mu || M < 1 || M > ((int64_t)1 << 31) - 1 || !(K > 0.0) || !std::isfinite(K)) {
    set_error("gs_voronoi_2d: need xi, mu non-NULL, 1 <= M < 2^31 and a finite K > 0");
    return GS_EINVAL;
  }
  for (int64_t i = 0; i < 2 * M; ++i)
    if (!std::isfinite(xi[i]) || std::fabs(xi[i]) > K) {
      set_error("gs_voronoi_2d: xi[%lld] = %g is not finite or outside [-K, K] (K = %g)", (long long)i, xi[i], K);
      return GS_EINVAL;
    }
  cudaStream_t st = (cudaStream_t)stream;
  // bucket grid of ~2 samples per bucket over Y_K, samples ordered by bucket (host counting sort)
  const int G = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (int64_t)std::ceil(std::sqrt((double)M / 2.0))));
  const double h = 2.0 * K / G;
  std::vector<int32_t> start((size_t)G * G + 1, 0), order(M), key(M);
  for (int64_t s = 0; s < M; ++s) {
    const int bi = std::min(G - 1, std::max(0, (int)std::floor((xi[2 * s] + K) / h)));
    const int bj = std::min(G - 1, std::max(0, (int)std::floor((xi[2 * s + 1] + K) / h)));
    key[s] = bj * G + bi;
    ++start[key[s] + 1];
  }
  for (size_t c = 0; c < (size_t)G * G; ++c) start[c + 1] += start[c];
  {
    std::vector<int32_t> fill(start.begin(), start.end() - 1);
    for (int64_t s = 0; s < M; ++s) order[fill[key[s]]++] = (int32_t)s;
  }
  double2* pts = nullptr;
  int32_t *cs = nullptr, *ord = nullptr;
  double *mud = nullptr, *rmd = nullptr;
  int* err = nullptr;
  auto release = [&]() {
    cudaFree(pts);
    cudaFree(cs);
    cudaFree(ord);
    cudaFree(mud);
    cudaFree(rmd);
    cudaFree(err);
  };
  cudaError_t e = cudaMalloc(&pts, M * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&cs, start.size() * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&ord, M * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&mud, M * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&rmd, M * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e != cudaSuccess) {
    release();
    set_error("gs_voronoi_2d: device allocation failed (%s)", cudaGetErrorString(e));
    return GS_ENOMEM;
  }
  e = cudaMemcpyAsync(pts, xi, M * sizeof(double2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cs, start.data(), start.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ord, order.data(), M * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    GS_LAUNCH("voronoi2d", st, k_voronoi2d<<<(M + 127) / 128, 128, 0, st>>>(pts, cs, ord, M, G, K, h, mud, rmd, err));
    e = cudaGetLastError();
  }
  std::vector<double> rm(M);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(mu, mud, M * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rm.data(), rmd, M * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  release();
  if (e != cudaSuccess) return cuda_fail(e, "gs_voronoi_2d");
  if (herr) {
    set_error("gs_voronoi_2d: a cell needed more than %d vertices", VMAX);
    return GS_EUNSUPPORTED;
  }
  if (delta) *delta = *std::max_element(rm.begin(), rm.end());
  return GS_OK;
}
