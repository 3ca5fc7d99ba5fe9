// Host-side LGL basis in FP64 (Sec. 2.1: nodes of (1 - xi^2) P_N', the (N+1)-point Lobatto
// quadrature of Eq. (lag_coefs), and the nodal differentiation matrix of the Lagrange basis of
// Eq. (lagrange_pol)).  Computed once per degree, then rounded to FP32 for the FP32 path.
//
// Interior nodes: zeros of P_N', i.e. of the Jacobi polynomial P^{(1,1)}_{N-1}, found as the
// eigenvalues of its symmetric tridiagonal Jacobi matrix (off-diagonal
// sqrt(k (k+2) / ((2k+1)(2k+3)))) by Sturm-sequence bisection, then polished by Newton steps in
// long double.  Weights 2 / (N (N+1) P_N(xi)^2).  D = V_r V^{-1} with the orthonormal Legendre
// Vandermonde V and its derivative V_r, inverted by Gauss-Jordan elimination in long double.
#include <cmath>
#include <cstring>

#include "ndg_internal.h"

namespace ndg {

namespace {

// Number of eigenvalues of the symmetric tridiagonal (diag 0, off-diagonal e) below x.
int sturm_count(const long double* e, int m, long double x) {
  int count = 0;
  long double q = -x;  // d_0 - x with d = 0
  if (q < 0) ++count;
  for (int k = 1; k < m; ++k) {
    long double denom = (q == 0.0L) ? 1e-300L : q;
    q = -x - e[k - 1] * e[k - 1] / denom;
    if (q < 0) ++count;
  }
  return count;
}

// Legendre P_N(x) and P_N'(x), long double.
void legendre(int N, long double x, long double* p, long double* dp) {
  long double p0 = 1.0L, p1 = x, d0 = 0.0L, d1 = 1.0L;
  if (N == 0) { *p = 1.0L; *dp = 0.0L; return; }
  for (int k = 1; k < N; ++k) {
    long double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    long double d2 = d0 + (2 * k + 1) * p1;  // P'_{k+1} = P'_{k-1} + (2k+1) P_k
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *p = p1;
  *dp = d1;
}

// Orthonormal Legendre value and derivative: sqrt((2j+1)/2) P_j.
void legendre_on(int j, long double x, long double* v, long double* dv) {
  long double p, dp;
  legendre(j, x, &p, &dp);
  long double s = sqrtl((2.0L * j + 1.0L) / 2.0L);
  *v = s * p;
  *dv = s * dp;
}

bool invert(int n, long double* A /* n*n, replaced by its inverse */) {
  long double M[kMaxN * 2 * kMaxN];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j)
      M[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0L : 0.0L);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(M[r * 2 * n + c]) > fabsl(M[piv * 2 * n + c])) piv = r;
    if (M[piv * 2 * n + c] == 0.0L) return false;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) {
        long double t = M[c * 2 * n + j];
        M[c * 2 * n + j] = M[piv * 2 * n + j];
        M[piv * 2 * n + j] = t;
      }
    long double inv = 1.0L / M[c * 2 * n + c];
    for (int j = 0; j < 2 * n; ++j) M[c * 2 * n + j] *= inv;
    for (int r = 0; r < n; ++r)
      if (r != c) {
        long double f = M[r * 2 * n + c];
        if (f != 0.0L)
          for (int j = 0; j < 2 * n; ++j) M[r * 2 * n + j] -= f * M[c * 2 * n + j];
      }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[i * n + j] = M[i * 2 * n + n + j];
  return true;
}

}  // namespace

bool build_basis(int N, Basis* b) {
  if (N < 1 || N > kMaxDegree) return false;
  const int n = N + 1;
  std::memset(b, 0, sizeof(*b));
  b->degree = N;
  long double x[kMaxN];
  x[0] = -1.0L;
  x[N] = 1.0L;
  const int m = N - 1;  // interior nodes
  if (m > 0) {
    long double e[kMaxN];
    for (int k = 1; k < m; ++k) e[k - 1] = sqrtl((long double)k * (k + 2) / ((2.0L * k + 1) * (2.0L * k + 3)));
    for (int r = 0; r < m; ++r) {  // r-th smallest eigenvalue by bisection on [-1, 1]
      long double lo = -1.0L, hi = 1.0L;
      for (int it = 0; it < 200; ++it) {
        long double mid = 0.5L * (lo + hi);
        if (sturm_count(e, m, mid) > r) hi = mid; else lo = mid;
      }
      long double xr = 0.5L * (lo + hi);
      for (int it = 0; it < 3; ++it) {  // Newton on P_N' with P_N'' from the Legendre equation
        long double p, dp;
        legendre(N, xr, &p, &dp);
        long double d2p = (2.0L * xr * dp - N * (N + 1.0L) * p) / (1.0L - xr * xr);
        if (d2p != 0.0L) xr -= dp / d2p;
      }
      x[r + 1] = xr;
    }
  }
  for (int i = 0; i < n; ++i) {
    long double p, dp;
    legendre(N, x[i], &p, &dp);
    b->xi[i] = (double)x[i];
    b->w[i] = (double)(2.0L / (N * (N + 1.0L) * p * p));
  }
  long double V[kMaxN * kMaxN], Vr[kMaxN * kMaxN];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) legendre_on(j, x[i], &V[i * n + j], &Vr[i * n + j]);
  // M^-1 = V V^T (orthonormal modal basis): the exact-mass lift vectors, scaled by the end weights
  for (int l = 0; l < n; ++l) {
    long double lo = 0.0L, hi = 0.0L;
    for (int j = 0; j < n; ++j) {
      lo += V[l * n + j] * V[0 * n + j];
      hi += V[l * n + j] * V[N * n + j];
    }
    b->lift_exact_lo[l] = (double)(lo * b->w[0]);
    b->lift_exact_hi[l] = (double)(hi * b->w[N]);
  }
  if (!invert(n, V)) return false;
  long double D[kMaxN * kMaxN];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      long double s = 0.0L;
      for (int k = 0; k < n; ++k) s += Vr[i * n + k] * V[k * n + j];
      D[i * n + j] = s;
    }
  for (int i = 0; i < n * n; ++i) b->D[i] = (double)D[i];
  // Even-odd split of the centro-antisymmetric D (D[N-i][N-m] = -D[i][m]): with
  // Fe[m] = F[m] + F[N-m], Fo[m] = F[m] - F[N-m] (m < h = (N+1)/2 pairs),
  //   (DF)_i = E_i + O_i, (DF)_{N-i} = E_i - O_i,
  //   E_i = sum_m Ae[i][m] Fo[m], Ae = (D[i][m] - D[i][N-m]) / 2,
  //   O_i = sum_m Bo[i][m] Fe[m] (+ D[i][mid] F[mid] for even N), Bo = (D[i][m] + D[i][N-m]) / 2.
  const int h = n / 2;
  for (int i = 0; i < h; ++i)
    for (int mm = 0; mm < h; ++mm) {
      b->Ae[i * kMaxN + mm] = (double)(0.5L * (D[i * n + mm] - D[i * n + (N - mm)]));
      b->Bo[i * kMaxN + mm] = (double)(0.5L * (D[i * n + mm] + D[i * n + (N - mm)]));
    }
  if (n % 2 == 1) {
    const int mid = N / 2;
    for (int i = 0; i < h; ++i) b->Cmid[i] = (double)D[i * n + mid];
    for (int mm = 0; mm < h; ++mm) b->Dmid[mm] = (double)D[mid * n + mm];
  }
  return true;
}

}  // namespace ndg
