// Plan-time constants computed on the host in float64: the Daubechies filter,
// moments of phi, and the boundary matrices U, V and v1(0) of the
// Cohen-Daubechies-Vial edge functions.  A few hundred flops per plan; the
// per-sample tables are built on the GPU from these (tables.cu).
//
// Filter (App. A): m0(xi) = sum_k h_k exp(-2 pi i k xi), m0(0) = 1, supp phi =
// [-p+1, p] (Sec. 3.3).  Daubechies extremal phase with p vanishing moments:
// |m0|^2 = cos^2p(pi xi) P(sin^2 pi xi), P(y) = sum_{k<p} C(p-1+k,k) y^k, and the
// spectral factor keeps, for each root y of P, the root |z| > 1 of
// z^2 - (2 - 4y) z + 1 = 0 (z = exp(-2 pi i xi)); largest taps first.
//
// Edge functions (Sec. 3.3; App. A.1, eq. dilation_eq_lphi): the span of
// x^a 1_[0,inf) minus its interior part, a < p, written over the half-line
// restricted translates phi(.-l) 1_[0,inf), l = -p+1..p-1.  Staircase basis:
// f_k has coefficient 1 at l = k and 0 at the other l in 0..p-1, so supp f_k =
// [0, p+k]; Cholesky of their Gram matrix orthonormalises them in order (the
// Gram-Schmidt of the nested supports), and phi^L_k has a positive coefficient
// at l = k, i.e. h^L_{k,p+2k} > 0 when the last filter tap is positive.  The
// two-scale relation of the restricted translates gives H (exact, from the
// l = 0..p-1 block) and h (n >= p).  Right side: the same on the reflected
// filter h_rev[k] = h[1-k], phi^R_k(x) = phi^L_k[rev](-x).
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "gs_internal.h"

namespace gs {

namespace {

using cd = std::complex<double>;

double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// Roots of sum_{k=0}^{deg} c[k] y^k by Durand-Kerner, then Newton polishing.
std::vector<cd> poly_roots(const std::vector<double>& c) {
  const int deg = (int)c.size() - 1;
  std::vector<cd> r;
  if (deg < 1) return r;
  std::vector<cd> a(deg + 1);
  for (int k = 0; k <= deg; ++k) a[k] = c[k] / c[deg];  // monic
  auto eval = [&](cd y) {
    cd v = a[deg];
    for (int k = deg - 1; k >= 0; --k) v = v * y + a[k];
    return v;
  };
  auto deval = [&](cd y) {
    cd v = a[deg] * double(deg);
    for (int k = deg - 1; k >= 1; --k) v = v * y + a[k] * double(k);
    return v;
  };
  double rad = 0.0;
  for (int k = 0; k < deg; ++k) rad = std::max(rad, std::abs(a[k]));
  rad = 1.0 + rad;
  r.resize(deg);
  for (int i = 0; i < deg; ++i) r[i] = std::polar(0.5 * rad, 0.4 + 2.0 * M_PI * i / deg);
  for (int it = 0; it < 2000; ++it) {
    double mv = 0.0;
    for (int i = 0; i < deg; ++i) {
      cd den = 1.0;
      for (int j = 0; j < deg; ++j)
        if (j != i) den *= (r[i] - r[j]);
      cd d = eval(r[i]) / den;
      r[i] -= d;
      mv = std::max(mv, std::abs(d));
    }
    if (mv < 1e-16) break;
  }
  for (int i = 0; i < deg; ++i)
    for (int it = 0; it < 4; ++it) {
      cd d = deval(r[i]);
      if (std::abs(d) == 0.0) break;
      r[i] -= eval(r[i]) / d;
    }
  return r;
}

// Dense solve A X = B in place (A n x n row-major, B n x m), partial pivoting.
bool lu_solve(std::vector<double> A, int n, std::vector<double>& B, int m) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
      for (int k = 0; k < m; ++k) std::swap(B[c * m + k], B[piv * m + k]);
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      if (f == 0.0) continue;
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      for (int k = 0; k < m; ++k) B[r * m + k] -= f * B[c * m + k];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    for (int k = 0; k < m; ++k) {
      double s = B[c * m + k];
      for (int j = c + 1; j < n; ++j) s -= A[c * n + j] * B[j * m + k];
      B[c * m + k] = s / A[c * n + c];
    }
  }
  return true;
}

// Edge constants for filter taps h[j], j = k + p - 1, k = -p+1..p.
bool edge_side(int p, const double* h, EdgeConst* out) {
  const int nt = 2 * p;       // taps
  const int nl = 2 * p - 1;   // restricted translates l = -p+1..p-1
  auto tap = [&](int k) -> double { return (k < -p + 1 || k > p) ? 0.0 : h[k + p - 1]; };
  const double s2 = std::sqrt(2.0);

  // moments mu_a, a < p
  std::vector<double> mu(p, 0.0);
  mu[0] = 1.0;
  for (int a = 1; a < p; ++a) {
    double s = 0.0;
    for (int b = 0; b < a; ++b) {
      double hk = 0.0;
      for (int k = -p + 1; k <= p; ++k) hk += tap(k) * std::pow((double)k, a - b);
      s += binom(a, b) * mu[b] * hk;
    }
    mu[a] = std::ldexp(s, -a) / (1.0 - std::ldexp(1.0, -a));
  }
  // Mt[a][l]: int x^a phi(x - l) dx
  std::vector<double> Mt(p * nl);
  for (int a = 0; a < p; ++a)
    for (int li = 0; li < nl; ++li) {
      double l = li - (p - 1), v = 0.0;
      for (int b = 0; b <= a; ++b) v += binom(a, b) * std::pow(l, a - b) * mu[b];
      Mt[a * nl + li] = v;
    }

  // half-line Gram A[a][b] = int_0^inf phi(x-a) phi(x-b), a, b = -p+1..p-1.
  // Unknown for a, b <= p-2; delta_ab once max(a,b) >= p-1; 0 once min(a,b) <= -p.
  const int nu = nl - 1;  // unknown indices -p+1..p-2
  auto known = [&](int a, int b, double* v) -> bool {
    if (a >= p - 1 || b >= p - 1) { *v = (a == b) ? 1.0 : 0.0; return true; }
    if (a <= -p || b <= -p) { *v = 0.0; return true; }
    return false;
  };
  std::vector<double> Ag(nl * nl, 0.0);
  if (nu > 0) {
    const int ns = nu * nu;
    std::vector<double> S(ns * ns, 0.0), rhs(ns, 0.0);
    for (int ia = 0; ia < nu; ++ia)
      for (int ib = 0; ib < nu; ++ib) {
        int a = ia - (p - 1), b = ib - (p - 1), row = ia * nu + ib;
        S[row * ns + row] += 1.0;
        for (int i = -p + 1; i <= p; ++i)
          for (int j = -p + 1; j <= p; ++j) {
            double w = 2.0 * tap(i) * tap(j), v;
            int aa = 2 * a + i, bb = 2 * b + j;
            if (known(aa, bb, &v)) rhs[row] += w * v;
            else S[row * ns + (aa + p - 1) * nu + (bb + p - 1)] -= w;
          }
      }
    if (!lu_solve(S, ns, rhs, 1)) return false;
    for (int ia = 0; ia < nl; ++ia)
      for (int ib = 0; ib < nl; ++ib) {
        int a = ia - (p - 1), b = ib - (p - 1);
        double v;
        Ag[ia * nl + ib] = known(a, b, &v) ? v : rhs[ia * nu + ib];
      }
  } else {
    Ag[0] = 1.0;
  }

  // staircase basis B = S^-1 Mt, S = Mt restricted to columns l = 0..p-1
  std::vector<double> Sb(p * p), B(p * nl);
  for (int a = 0; a < p; ++a)
    for (int c = 0; c < p; ++c) Sb[a * p + c] = Mt[a * nl + (c + p - 1)];
  // B = Sb^-1 Mt: solve Sb X = Mt
  std::vector<double> X = Mt;
  if (!lu_solve(Sb, p, X, nl)) return false;
  B = X;
  // Gram Gf = B Ag B^T, Cholesky Gf = L L^T
  std::vector<double> Gf(p * p, 0.0), L(p * p, 0.0);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) {
      double s = 0.0;
      for (int a = 0; a < nl; ++a)
        for (int b = 0; b < nl; ++b) s += B[i * nl + a] * Ag[a * nl + b] * B[j * nl + b];
      Gf[i * p + j] = s;
    }
  for (int i = 0; i < p; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = Gf[i * p + j];
      for (int k = 0; k < j; ++k) s -= L[i * p + k] * L[j * p + k];
      if (i == j) {
        if (s <= 0.0) return false;
        L[i * p + i] = std::sqrt(s);
      } else {
        L[i * p + j] = s / L[j * p + j];
      }
    }
  // C = L^-1 B (forward substitution): phi^L_k = sum_l C[k][l] phi(.-l) 1_[0,inf)
  std::vector<double> C(p * nl);
  for (int k = 0; k < p; ++k)
    for (int l = 0; l < nl; ++l) {
      double s = B[k * nl + l];
      for (int j = 0; j < k; ++j) s -= L[k * p + j] * C[j * nl + l];
      C[k * nl + l] = s / L[k * p + k];
    }
  const double hlast = s2 * tap(p);
  if (hlast < 0.0)
    for (double& v : C) v = -v;

  // two-scale: phi^L_k(x)/sqrt2 = sum_n D[k][n] phi(2x - n) 1_[0,inf),
  // D[k][n] = sum_l C[k][l] hon[n - 2l], n = -p+1..3p-2 (n <= -p vanish on [0,inf))
  const int nn = 4 * p - 2;
  std::vector<double> D(p * nn, 0.0);
  for (int k = 0; k < p; ++k)
    for (int li = 0; li < nl; ++li) {
      int l = li - (p - 1);
      for (int t = -p + 1; t <= p; ++t) {
        int n = 2 * l + t;
        if (n >= -p + 1) D[k * nn + (n + p - 1)] += C[k * nl + li] * s2 * tap(t);
      }
    }
  // H from the l = 0..p-1 block, where C is lower triangular: H Cb = Db
  std::vector<double> H(p * p);
  {
    // H^T = Cb^-T Db^T: solve Cb^T H^T = Db^T
    std::vector<double> CbT(p * p), rhs(p * p);
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) {
        CbT[i * p + j] = C[j * nl + (i + p - 1)];
        rhs[i * p + j] = D[j * nn + (i + p - 1)];
      }
    if (!lu_solve(CbT, p, rhs, p)) return false;
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) H[j * p + i] = rhs[i * p + j];
  }
  // nestedness residual over all edge translates n = -p+1..p-1
  double nest = 0.0;
  for (int k = 0; k < p; ++k)
    for (int li = 0; li < nl; ++li) {
      double s = 0.0;
      for (int j = 0; j < p; ++j) s += H[k * p + j] * C[j * nl + li];
      nest = std::max(nest, std::fabs(s - D[k * nn + li]));
    }
  out->p = p;
  out->nest_residual = nest;
  for (int k = 0; k < p; ++k) {
    for (int j = 0; j < p; ++j) out->U[k][j] = H[k * p + j] / s2;
    for (int m = 0; m < 2 * p - 1; ++m) out->V[k][m] = D[k * nn + (m + 2 * p - 1)] / s2;
  }
  // v1(0) = (I - U)^-1 V 1
  std::vector<double> IU(p * p), r(p);
  for (int i = 0; i < p; ++i) {
    double s = 0.0;
    for (int m = 0; m < 2 * p - 1; ++m) s += out->V[i][m];
    r[i] = s;
    for (int j = 0; j < p; ++j) IU[i * p + j] = (i == j ? 1.0 : 0.0) - out->U[i][j];
  }
  if (!lu_solve(IU, p, r, 1)) return false;
  for (int i = 0; i < p; ++i) out->v10[i] = r[i];
  return true;
}

}  // namespace

bool daubechies_taps(int p, double* h) {
  if (p < 1 || p > GS_MAX_P) return false;
  std::vector<double> pc(p);
  for (int k = 0; k < p; ++k) pc[k] = binom(p - 1 + k, k);
  std::vector<cd> ys = poly_roots(pc);
  std::vector<cd> q(1, cd(1.0, 0.0));
  auto mul = [&](cd c0, cd c1) {  // q *= (c0 + c1 z)
    std::vector<cd> r(q.size() + 1, cd(0.0, 0.0));
    for (size_t i = 0; i < q.size(); ++i) {
      r[i] += q[i] * c0;
      r[i + 1] += q[i] * c1;
    }
    q.swap(r);
  };
  for (int i = 0; i < p; ++i) mul(1.0, 1.0);
  for (const cd& y : ys) {
    cd bq = 2.0 - 4.0 * y;
    cd disc = std::sqrt(bq * bq - 4.0);
    cd z1 = (bq + disc) / 2.0, z2 = (bq - disc) / 2.0;
    cd z = std::abs(z1) > std::abs(z2) ? z1 : z2;
    mul(-z, 1.0);
  }
  double sum = 0.0;
  for (const cd& c : q) sum += c.real();
  for (int j = 0; j < 2 * p; ++j) h[j] = q[j].real() / sum;
  return true;
}

bool build_constants(int p, Constants* c) {
  std::memset(c, 0, sizeof(*c));
  c->p = p;
  if (!daubechies_taps(p, c->h)) return false;
  // moments mu_0..mu_2 (any p) for the Taylor tail of phi-hat at tiny arguments
  double mu[3] = {1.0, 0.0, 0.0};
  for (int a = 1; a < 3; ++a) {
    double s = 0.0;
    for (int b = 0; b < a; ++b) {
      double hk = 0.0;
      for (int k = -p + 1; k <= p; ++k) hk += c->h[k + p - 1] * std::pow((double)k, a - b);
      s += binom(a, b) * mu[b] * hk;
    }
    mu[a] = std::ldexp(s, -a) / (1.0 - std::ldexp(1.0, -a));
  }
  c->mu1 = mu[1];
  c->mu2 = mu[2];
  if (p == 1) return true;  // Haar: no edge functions (Sec. 3.3)
  double hrev[2 * GS_MAX_P];
  for (int k = -p + 1; k <= p; ++k) hrev[k + p - 1] = c->h[(1 - k) + p - 1];
  return edge_side(p, c->h, &c->left) && edge_side(p, hrev, &c->right);
}

}  // namespace gs
