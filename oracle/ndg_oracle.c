/*
 * ndg_oracle.c -- ORACLE. This is test infrastructure, not part of the product.
 *
 * Plain, slow, single-threaded CPU implementation in IEEE binary64 of the method of
 * arXiv:2510.05254 ("Performance of a high-order MPI-Kokkos accelerated fluid solver"),
 * Section 2 "Methods": the nodal discontinuous Galerkin (NDG) spatial operator on
 * Legendre-Gauss-Lobatto (LGL) nodes, with the Lax-Friedrichs / upwind numerical flux, driven
 * by the explicit Runge-Kutta schemes RK3, RK4 and RK6 of Section 2.3.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the CUDA path shares no code
 * with it and never calls it.
 *
 * It follows the paper's steps in the paper's order and form, one line of nodes at a time:
 *   - LGL nodes: roots of (1 - xi^2) P_N'(xi) (Sec. 2.1, after Eq. (lagrange_pol)), found by
 *     Newton iteration on P_N' started from Chebyshev-Gauss-Lobatto points.
 *   - Quadrature weights w_k = 2 / (N (N+1) P_N(xi_k)^2) (the textbook LGL weights; the paper
 *     uses a (p+1)-point Gauss-Lobatto quadrature, Eq. (lag_coefs), without printing them).
 *   - D[k][l] = h_l'(xi_k): the derivative of the paper's Lagrange polynomial, Eq. (lagrange_pol),
 *     evaluated at the nodes (closed form obtained from the Legendre equation).
 *   - Weak form with integration by parts (Sec. 2.1, the evolution equation after Eq. (LF)), the
 *     mass matrix lumped by the quadrature, Eq. (lag_coefs):
 *        (dx/2) w_l dU_l/dt = sum_k w_k F_k D[k][l] - ( Fhat_R delta_{lN} - Fhat_L delta_{l0} ),
 *     applied along every axis of a tensor-product element (face integrals by LGL quadrature).
 *   - Numerical flux, Eq. (LF): Fhat = 1/2 [F(U-) + F(U+) - alpha (U+ - U-)], alpha the largest
 *     |eigenvalue| of the flux Jacobian at the border (local Lax-Friedrichs); for advection the
 *     upwind choice F(U-) if a >= 0 else F(U+), which is the same value.
 *   - Fluxes: linear advection Eq. (advection1d)/(advection2d); isothermal Euler Eq. (eulerIso2d).
 *   - Periodic boundaries (Sec. 3.1).
 *   - Runge-Kutta: Eq. (RK3), Eq. (RK4), Eq. (RK6) as printed (RK3 read as explained below).
 *   - L2 norm (Sec. 3.1) by LGL quadrature on every element.
 *
 * Readings of passages that are ambiguous or garbled in the paper:
 *   1. Mass matrix: lumped, int h_k h_l ~= w_k delta_kl (Eq. (lag_coefs)), as the paper's equations
 *      state.  Its cited textbook NDG uses the exact mass matrix instead; that variant is kept as
 *      an option (mass = ORC_MASS_EXACT): M[k][l] = int h_k h_l exactly (Gauss-Legendre
 *      quadrature with N+1 points), and the weak form is solved with M in place of diag(w).
 *   2. Element map Eq. (transformation) has no element offset; x = x_{j-1/2} + (dx/2)(xi + 1).
 *   3. "N" is both the element count and the degree; here N is the degree, n = N+1 nodes/axis.
 *   4. Local Lax-Friedrichs: alpha = max over both sides of |lambda_max|; isothermal Euler has
 *      eigenvalues u_n and u_n +- c, so alpha = max(|u_n^-|, |u_n^+|) + c.
 *   5. RK3: the printed k_3 = dt (k_1 + 3 F(U^N + k_2)) / 4 mixes dt into k_1 twice; read as
 *      k_3 = (3 k_1 + 3 dt F(U^N + k_2)) / 4 (Heun's third-order method, b = (1/4, 0, 3/4)).
 *   6. Mach number: the paper's M = a/u_max is read as u_max/a.
 *   7. Time step: not given in the paper; dt = CFL * h_min / lambda with h_min the smallest
 *      physical LGL spacing and lambda = sum_k |a_k| (advection) or
 *      max over nodes of sum_k |u_k| + dim * c (isothermal Euler).
 *
 * Layout (the interface shared with the library, so that one array feeds both):
 *   U[v][e][node], v < nvar, e = ex + Ex*(ey + Ey*ez), node = i + n*(j + n*k).
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -pthread -fPIC -shared ndg_oracle.c -lm
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 16

enum { ORC_ADVECTION = 0, ORC_ISO_EULER = 1 };
enum { ORC_FLUX_UPWIND = 0, ORC_FLUX_LLF = 1 };
enum { ORC_MASS_LUMPED = 0, ORC_MASS_EXACT = 1 };

typedef struct {
  int dim;        /* 1, 2 or 3 */
  int degree;     /* N >= 1 */
  int elems[3];   /* elements per axis (unused axes: 1) */
  int equation;   /* ORC_ADVECTION or ORC_ISO_EULER */
  int flux;       /* ORC_FLUX_UPWIND or ORC_FLUX_LLF */
  double length[3]; /* domain [0, length[a]] per axis */
  double velocity[3]; /* advection velocity a */
  double sound_speed; /* isothermal sound speed (the paper's a in Eq. (eulerIso2d)) */
  int mass;       /* ORC_MASS_LUMPED (the paper's) or ORC_MASS_EXACT */
} orc_problem;

/* ------------------------------------------------------------------------------------------ */
/* Legendre polynomials by the three-term recurrence                                           */
/* ------------------------------------------------------------------------------------------ */

/* P_N(x) and P_{N-1}(x). */
static void legendre(int N, double x, double* pN, double* pNm1) {
  double p0 = 1.0, p1 = x;
  if (N == 0) { *pN = 1.0; *pNm1 = 0.0; return; }
  for (int k = 1; k < N; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *pN = p1;
  *pNm1 = p0;
}

/* LGL nodes (ascending) and weights for degree N: xi_0 = -1, xi_N = +1, interior nodes are the
 * roots of P_N'.  Newton on P_N' uses P_N'' from the Legendre equation
 * (1 - x^2) P'' = 2 x P' - N(N+1) P. */
int orc_lgl(int N, double* xi, double* w) {
  if (N < 1 || N >= ORC_MAXN) return -1;
  const double pi = 3.14159265358979323846;
  for (int k = 0; k <= N; ++k) {
    double x = -cos(pi * k / N);
    if (k > 0 && k < N) {
      for (int it = 0; it < 100; ++it) {
        double pN, pNm1;
        legendre(N, x, &pN, &pNm1);
        double dp = N * (x * pN - pNm1) / (x * x - 1.0);      /* P_N'(x) */
        double d2p = (2.0 * x * dp - N * (N + 1.0) * pN) / (1.0 - x * x); /* P_N''(x) */
        double step = dp / d2p;
        x -= step;
        if (fabs(step) < 1e-16) break;
      }
    }
    xi[k] = x;
  }
  xi[0] = -1.0;
  xi[N] = 1.0;
  for (int k = 0; k <= N; ++k) {
    double pN, pNm1;
    legendre(N, xi[k], &pN, &pNm1);
    w[k] = 2.0 / (N * (N + 1.0) * pN * pN);
  }
  return 0;
}

/* D[k*(N+1) + l] = h_l'(xi_k) for the Lagrange polynomial of Eq. (lagrange_pol).  Off the
 * diagonal the numerator (x^2-1) P_N'(x) of h_l vanishes at every node and has derivative
 * N(N+1) P_N(x), so h_l'(xi_k) = P_N(xi_k) / (P_N(xi_l) (xi_k - xi_l)).  On the diagonal the
 * derivative is -N(N+1)/4 at xi = -1, +N(N+1)/4 at xi = +1 and 0 at the interior nodes. */
int orc_dmat(int N, const double* xi, double* D) {
  if (N < 1 || N >= ORC_MAXN) return -1;
  int n = N + 1;
  double P[ORC_MAXN];
  for (int k = 0; k < n; ++k) {
    double pNm1;
    legendre(N, xi[k], &P[k], &pNm1);
  }
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) {
      double d;
      if (k != l) d = P[k] / (P[l] * (xi[k] - xi[l]));
      else if (k == 0) d = -N * (N + 1.0) / 4.0;
      else if (k == N) d = N * (N + 1.0) / 4.0;
      else d = 0.0;
      D[k * n + l] = d;
    }
  return 0;
}

/* The Lagrange polynomial h_i of Eq. (lagrange_pol) on the nodes xi, evaluated at x. */
static double lagrange(int N, const double* xi, int i, double x) {
  double v = 1.0;
  for (int j = 0; j <= N; ++j)
    if (j != i) v *= (x - xi[j]) / (xi[i] - xi[j]);
  return v;
}

/* Mass matrix of the Lagrange basis on the LGL nodes, M[k*(N+1) + l] ~ int_{-1}^{1} h_k h_l:
 * exact = 0: lumped by the LGL quadrature of Eq. (lag_coefs), diag(w);
 * exact = 1: integrated exactly by Gauss-Legendre quadrature with N+1 points (exact to degree
 *            2N+1; the integrand has degree 2N).  Gauss nodes: Newton on P_{N+1} from the
 *            usual cosine guesses; weights 2 / ((1 - x^2) P_{N+1}'(x)^2). */
int orc_mass(int N, int exact, double* M) {
  if (N < 1 || N >= ORC_MAXN) return -1;
  int n = N + 1;
  double xi[ORC_MAXN], w[ORC_MAXN];
  orc_lgl(N, xi, w);
  for (int q = 0; q < n * n; ++q) M[q] = 0.0;
  if (!exact) {
    for (int k = 0; k < n; ++k) M[k * n + k] = w[k];
    return 0;
  }
  const double pi = 3.14159265358979323846;
  const int m = n; /* Gauss points */
  for (int q = 0; q < m; ++q) {
    double x = cos(pi * (q + 0.75) / (m + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double pm, pm1;
      legendre(m, x, &pm, &pm1);
      dp = m * (x * pm - pm1) / (x * x - 1.0); /* P_m'(x) */
      double step = pm / dp;
      x -= step;
      if (fabs(step) < 1e-16) break;
    }
    double pm, pm1;
    legendre(m, x, &pm, &pm1);
    dp = m * (x * pm - pm1) / (x * x - 1.0);
    double wq = 2.0 / ((1.0 - x * x) * dp * dp);
    double hv[ORC_MAXN];
    for (int k = 0; k < n; ++k) hv[k] = lagrange(N, xi, k, x);
    for (int k = 0; k < n; ++k)
      for (int l = 0; l < n; ++l) M[k * n + l] += wq * hv[k] * hv[l];
  }
  return 0;
}

/* In-place inverse of the n x n matrix A (Gauss-Jordan elimination with partial pivoting). */
static int invert(int n, double* A) {
  double B[ORC_MAXN * ORC_MAXN];
  for (int i = 0; i < n * n; ++i) B[i] = 0.0;
  for (int i = 0; i < n; ++i) B[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return -1;
    for (int j = 0; j < n; ++j) {
      double t = A[c * n + j]; A[c * n + j] = A[piv * n + j]; A[piv * n + j] = t;
      t = B[c * n + j]; B[c * n + j] = B[piv * n + j]; B[piv * n + j] = t;
    }
    double d = A[c * n + c];
    for (int j = 0; j < n; ++j) { A[c * n + j] /= d; B[c * n + j] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[r * n + c];
      for (int j = 0; j < n; ++j) { A[r * n + j] -= f * A[c * n + j]; B[r * n + j] -= f * B[c * n + j]; }
    }
  }
  for (int i = 0; i < n * n; ++i) A[i] = B[i];
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Problem geometry                                                                              */
/* ------------------------------------------------------------------------------------------ */

static int nvar_of(const orc_problem* p) {
  return p->equation == ORC_ADVECTION ? 1 : p->dim + 1;
}

static int ipow(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

int orc_nvar(const orc_problem* p) { return nvar_of(p); }

int64_t orc_ndof(const orc_problem* p) {
  int64_t ne = 1;
  for (int a = 0; a < p->dim; ++a) ne *= p->elems[a];
  return ne * ipow(p->degree + 1, p->dim) * nvar_of(p);
}

static int check_problem(const orc_problem* p) {
  if (p->dim < 1 || p->dim > 3) return -1;
  if (p->degree < 1 || p->degree >= ORC_MAXN) return -1;
  for (int a = 0; a < p->dim; ++a)
    if (p->elems[a] < 1 || !(p->length[a] > 0.0)) return -1;
  if (p->equation != ORC_ADVECTION && p->equation != ORC_ISO_EULER) return -1;
  if (p->equation == ORC_ISO_EULER && p->flux != ORC_FLUX_LLF) return -1;
  if (p->mass != ORC_MASS_LUMPED && p->mass != ORC_MASS_EXACT) return -1;
  return 0;
}

/* Node coordinates X[a][e][node] for a < dim (reading 2 of the element map). */
int orc_node_coords(const orc_problem* p, double* X) {
  if (check_problem(p)) return -1;
  int N = p->degree, n = N + 1, d = p->dim;
  double xi[ORC_MAXN], w[ORC_MAXN];
  orc_lgl(N, xi, w);
  int E[3] = {1, 1, 1};
  for (int a = 0; a < d; ++a) E[a] = p->elems[a];
  int np = ipow(n, d);
  int64_t ne = (int64_t)E[0] * E[1] * E[2];
  for (int a = 0; a < d; ++a) {
    double h = p->length[a] / E[a];
    for (int64_t e = 0; e < ne; ++e) {
      int ei[3] = {(int)(e % E[0]), (int)((e / E[0]) % E[1]), (int)(e / ((int64_t)E[0] * E[1]))};
      for (int node = 0; node < np; ++node) {
        int ii[3] = {node % n, (node / n) % n, node / (n * n)};
        X[((int64_t)a * ne + e) * np + node] = ei[a] * h + 0.5 * h * (xi[ii[a]] + 1.0);
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Fluxes                                                                                        */
/* ------------------------------------------------------------------------------------------ */

/* Physical flux along axis `axis` for one node's state u[nvar]. */
static void physical_flux(const orc_problem* p, int axis, const double* u, double* f) {
  if (p->equation == ORC_ADVECTION) {
    f[0] = p->velocity[axis] * u[0]; /* Eq. (advection2d) */
    return;
  }
  /* Eq. (eulerIso2d): U = (rho, rho u_x, rho u_y, rho u_z); the flux along axis a is
   * (rho u_a, rho u_a u_x, rho u_a u_y, rho u_a u_z) plus rho c^2 on the momentum component a. */
  double rho = u[0];
  double ua = u[1 + axis] / rho;
  double c = p->sound_speed;
  f[0] = u[1 + axis];
  for (int b = 0; b < p->dim; ++b) f[1 + b] = u[1 + b] * ua;
  f[1 + axis] += rho * c * c;
}

/* Numerical flux across a face normal to `axis`, with uL on the low side and uR on the high side
 * of the face (the paper's U- and U+), Eq. (LF). */
static void numerical_flux(const orc_problem* p, int axis, const double* uL, const double* uR,
                           double* fhat) {
  int nv = nvar_of(p);
  double fL[4], fR[4];
  physical_flux(p, axis, uL, fL);
  physical_flux(p, axis, uR, fR);
  if (p->equation == ORC_ADVECTION && p->flux == ORC_FLUX_UPWIND) {
    /* upwind: the state the characteristic comes from */
    for (int v = 0; v < nv; ++v) fhat[v] = p->velocity[axis] >= 0.0 ? fL[v] : fR[v];
    return;
  }
  double alpha;
  if (p->equation == ORC_ADVECTION) {
    alpha = fabs(p->velocity[axis]);
  } else {
    double unL = uL[1 + axis] / uL[0];
    double unR = uR[1 + axis] / uR[0];
    alpha = fmax(fabs(unL), fabs(unR)) + p->sound_speed;
  }
  for (int v = 0; v < nv; ++v) fhat[v] = 0.5 * (fL[v] + fR[v] - alpha * (uR[v] - uL[v]));
}

/* ------------------------------------------------------------------------------------------ */
/* Spatial operator R = L(U)                                                                    */
/* ------------------------------------------------------------------------------------------ */

/* R = L(U) on the elements [e_begin, e_end) only (their nodes of every variable); U is read on
 * those elements and their face neighbours.  orc_rhs is the whole range. */
static int rhs_elements(const orc_problem* p, const double* U, double* R, int64_t e_begin, int64_t e_end) {
  if (check_problem(p)) return -1;
  int N = p->degree, n = N + 1, d = p->dim, nv = nvar_of(p);
  double xi[ORC_MAXN], w[ORC_MAXN], D[ORC_MAXN * ORC_MAXN];
  orc_lgl(N, xi, w);
  orc_dmat(N, xi, D);
  const int exact = p->mass == ORC_MASS_EXACT;
  double Minv[ORC_MAXN * ORC_MAXN];
  if (exact) {
    orc_mass(N, 1, Minv);
    if (invert(n, Minv)) return -1;
  }
  int E[3] = {1, 1, 1};
  for (int a = 0; a < d; ++a) E[a] = p->elems[a];
  int np = ipow(n, d);
  int64_t ne = (int64_t)E[0] * E[1] * E[2];
  int64_t nd = ne * np * nv;
  int stride[3] = {1, n, n * n}; /* node-index stride along each axis */
  (void)nd;
  for (int v = 0; v < nv; ++v)
    for (int64_t q = ((int64_t)v * ne + e_begin) * np; q < ((int64_t)v * ne + e_end) * np; ++q) R[q] = 0.0;

  double u[ORC_MAXN][4], F[ORC_MAXN][4], uLn[4], uRn[4], fhatL[4], fhatR[4], b[ORC_MAXN][4];
  for (int64_t e = e_begin; e < e_end; ++e) {
    int ei[3] = {(int)(e % E[0]), (int)((e / E[0]) % E[1]), (int)(e / ((int64_t)E[0] * E[1]))};
    for (int a = 0; a < d; ++a) {
      double h = p->length[a] / E[a];
      /* periodic neighbours along axis a */
      int lo[3] = {ei[0], ei[1], ei[2]}, hi[3] = {ei[0], ei[1], ei[2]};
      lo[a] = (ei[a] + E[a] - 1) % E[a];
      hi[a] = (ei[a] + 1) % E[a];
      int64_t eL = lo[0] + (int64_t)E[0] * (lo[1] + (int64_t)E[1] * lo[2]);
      int64_t eR = hi[0] + (int64_t)E[0] * (hi[1] + (int64_t)E[1] * hi[2]);
      /* every line of nodes along axis a: the node whose index along a is 0 */
      for (int base = 0; base < np; ++base) {
        int ib[3] = {base % n, (base / n) % n, base / (n * n)};
        if (ib[a] != 0) continue;
        for (int l = 0; l < n; ++l)
          for (int v = 0; v < nv; ++v)
            u[l][v] = U[((int64_t)v * ne + e) * np + base + l * stride[a]];
        for (int v = 0; v < nv; ++v) {
          uLn[v] = U[((int64_t)v * ne + eL) * np + base + N * stride[a]]; /* left neighbour, end N */
          uRn[v] = U[((int64_t)v * ne + eR) * np + base];                 /* right neighbour, end 0 */
        }
        for (int l = 0; l < n; ++l) physical_flux(p, a, u[l], F[l]);
        numerical_flux(p, a, uLn, u[0], fhatL); /* face at xi = -1 */
        numerical_flux(p, a, u[N], uRn, fhatR); /* face at xi = +1 */
        for (int l = 0; l < n; ++l) {
          for (int v = 0; v < nv; ++v) {
            double vol = 0.0;
            for (int k = 0; k < n; ++k) vol += w[k] * F[k][v] * D[k * n + l];
            double surf = 0.0;
            if (l == N) surf -= fhatR[v];
            if (l == 0) surf += fhatL[v];
            b[l][v] = vol + surf;
          }
        }
        /* solve with the mass matrix: lumped diag(w), or the exact M (reading 1) */
        for (int l = 0; l < n; ++l) {
          for (int v = 0; v < nv; ++v) {
            double* out = &R[((int64_t)v * ne + e) * np + base + l * stride[a]];
            if (!exact) {
              *out += (2.0 / h) * b[l][v] / w[l];
            } else {
              double r = 0.0;
              for (int m = 0; m < n; ++m) r += Minv[l * n + m] * b[m][v];
              *out += (2.0 / h) * r;
            }
          }
        }
      }
    }
  }
  return 0;
}

int orc_rhs(const orc_problem* p, const double* U, double* R) {
  if (check_problem(p)) return -1;
  int64_t ne = 1;
  for (int a = 0; a < p->dim; ++a) ne *= p->elems[a];
  return rhs_elements(p, U, R, 0, ne);
}

/* ------------------------------------------------------------------------------------------ */
/* Runge-Kutta schemes of Sec. 2.3, generic over the right-hand side                            */
/* ------------------------------------------------------------------------------------------ */

/* The part of the unknowns one caller updates: index spans [lo, hi), the element range its
 * right-hand side covers, and a barrier that every caller passes before and after each
 * right-hand-side evaluation (NULL for a single caller).  One caller owning everything is the
 * plain sequential scheme; several callers with disjoint parts (orc_step_threads) perform the
 * same operations on every unknown, so their result is bitwise the sequential one. */
typedef struct {
  const int64_t* lo;
  const int64_t* hi;
  int nspans;
  int64_t e_begin, e_end;
  void (*sync)(void* ctx);
  void* sync_ctx;
} orc_part;

typedef int (*rhs_fn)(const void* ctx, const double* U, double* R, const orc_part* part);

#define OWN(i) for (int s_ = 0; s_ < part->nspans; ++s_) for (i = part->lo[s_]; i < part->hi[s_]; ++i)
#define SYNC() do { if (part->sync) part->sync(part->sync_ctx); } while (0)
/* F evaluated once every caller has written its stage argument, and before any overwrites it */
#define EVAL(Y) do { SYNC(); if (F(ctx, (Y), Fy, part)) return -1; SYNC(); } while (0)

/* One step of size dt of the scheme `rk` (3, 4 or 6) for U' = F(U) on this caller's part of
 * the n unknowns.  work must hold 9 * n doubles (shared by all callers). */
static int rk_advance(int rk, int64_t n, double* U, double dt, rhs_fn F, const void* ctx,
                      double* work, const orc_part* part) {
  double* k1 = work;
  double* k2 = work + n;
  double* k3 = work + 2 * n;
  double* k4 = work + 3 * n;
  double* k5 = work + 4 * n;
  double* k6 = work + 5 * n;
  double* k7 = work + 6 * n;
  double* Y = work + 7 * n;  /* stage argument U^N + ... */
  double* Fy = work + 8 * n; /* F(Y) */
  int64_t i;
  if (rk == 3) { /* Eq. (RK3), reading 5 */
    EVAL(U);
    OWN(i) k1[i] = dt * Fy[i] / 3.0;
    OWN(i) Y[i] = U[i] + k1[i];
    EVAL(Y);
    OWN(i) k2[i] = 2.0 * dt * Fy[i] / 3.0;
    OWN(i) Y[i] = U[i] + k2[i];
    EVAL(Y);
    OWN(i) k3[i] = (3.0 * k1[i] + 3.0 * dt * Fy[i]) / 4.0;
    OWN(i) U[i] = U[i] + k3[i];
    return 0;
  }
  if (rk == 4) { /* Eq. (RK4) */
    EVAL(U);
    OWN(i) k1[i] = dt * Fy[i];
    OWN(i) Y[i] = U[i] + k1[i] / 2.0;
    EVAL(Y);
    OWN(i) k2[i] = dt * Fy[i];
    OWN(i) Y[i] = U[i] + k2[i] / 2.0;
    EVAL(Y);
    OWN(i) k3[i] = dt * Fy[i];
    OWN(i) Y[i] = U[i] + k3[i];
    EVAL(Y);
    OWN(i) k4[i] = dt * Fy[i];
    OWN(i) U[i] = U[i] + (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]) / 6.0;
    return 0;
  }
  if (rk == 6) { /* Eq. (RK6), Luther's seven-stage sixth-order scheme, as printed */
    const double s = sqrt(21.0);
    EVAL(U);
    OWN(i) k1[i] = dt * Fy[i];
    OWN(i) Y[i] = U[i] + k1[i];
    EVAL(Y);
    OWN(i) k2[i] = dt * Fy[i];
    OWN(i) Y[i] = U[i] + (3.0 * k1[i] + k2[i]) / 8.0;
    EVAL(Y);
    OWN(i) k3[i] = dt * Fy[i];
    OWN(i) Y[i] = U[i] + (8.0 * k1[i] + 2.0 * k2[i] + 8.0 * k3[i]) / 27.0;
    EVAL(Y);
    OWN(i) k4[i] = dt * Fy[i];
    OWN(i)
      Y[i] = U[i] + (3.0 * (3.0 * s - 7.0) * k1[i] - 8.0 * (7.0 - s) * k2[i] +
                     48.0 * (7.0 - s) * k3[i] - 3.0 * (21.0 - s) * k4[i]) / 392.0;
    EVAL(Y);
    OWN(i) k5[i] = dt * Fy[i];
    OWN(i)
      Y[i] = U[i] + (-5.0 * (231.0 + 51.0 * s) * k1[i] - 40.0 * (7.0 + s) * k2[i] -
                     320.0 * s * k3[i] + 3.0 * (21.0 + 121.0 * s) * k4[i] +
                     392.0 * (6.0 + s) * k5[i]) / 1960.0;
    EVAL(Y);
    OWN(i) k6[i] = dt * Fy[i];
    OWN(i)
      Y[i] = U[i] + (15.0 * (22.0 + 7.0 * s) * k1[i] + 120.0 * k2[i] +
                     40.0 * (7.0 * s - 5.0) * k3[i] - 63.0 * (3.0 * s - 2.0) * k4[i] -
                     14.0 * (49.0 + 9.0 * s) * k5[i] + 70.0 * (7.0 - s) * k6[i]) / 180.0;
    EVAL(Y);
    OWN(i) k7[i] = dt * Fy[i];
    OWN(i)
      U[i] = U[i] + (9.0 * k1[i] + 64.0 * k3[i] + 49.0 * k5[i] + 49.0 * k6[i] + 9.0 * k7[i]) / 180.0;
    return 0;
  }
  return -1;
}

static int pde_rhs(const void* ctx, const double* U, double* R, const orc_part* part) {
  return rhs_elements((const orc_problem*)ctx, U, R, part->e_begin, part->e_end);
}

/* nsteps steps of size dt of scheme rk (3, 4, 6) on the NDG semi-discretisation, in place. */
int orc_step(const orc_problem* p, double* U, double dt, int nsteps, int rk) {
  if (check_problem(p) || nsteps < 0 || !(dt > 0.0) || (rk != 3 && rk != 4 && rk != 6)) return -1;
  int64_t nd = orc_ndof(p);
  double* work = (double*)malloc(sizeof(double) * 9 * (size_t)nd);
  if (!work) return -2;
  const int64_t lo = 0, hi = nd;
  const orc_part whole = {&lo, &hi, 1, 0, nd / nvar_of(p) / ipow(p->degree + 1, p->dim), NULL, NULL};
  int rc = 0;
  for (int s = 0; s < nsteps && rc == 0; ++s) rc = rk_advance(rk, nd, U, dt, pde_rhs, p, work, &whole);
  free(work);
  return rc;
}

/* ---- the same scheme split over threads, for timing on a multi-core host ---------------- */

typedef struct {
  pthread_mutex_t mu;
  pthread_cond_t cv;
  int count, total, generation;
} orc_barrier;

static void barrier_wait(void* ctx) {
  orc_barrier* b = (orc_barrier*)ctx;
  pthread_mutex_lock(&b->mu);
  const int gen = b->generation;
  if (++b->count == b->total) {
    b->count = 0;
    ++b->generation;
    pthread_cond_broadcast(&b->cv);
  } else {
    while (gen == b->generation) pthread_cond_wait(&b->cv, &b->mu);
  }
  pthread_mutex_unlock(&b->mu);
}

typedef struct {
  const orc_problem* p;
  double* U;
  double* work;
  double dt;
  int nsteps, rk, rc;
  int64_t lo[4], hi[4];
  orc_part part;
} orc_worker;

static void* worker_main(void* arg) {
  orc_worker* w = (orc_worker*)arg;
  const int64_t nd = orc_ndof(w->p);
  w->rc = 0;
  for (int s = 0; s < w->nsteps; ++s) {
    /* every thread runs every step (a failing one still passes its barriers: its rc is kept) */
    int rc = rk_advance(w->rk, nd, w->U, w->dt, pde_rhs, w->p, w->work, &w->part);
    if (rc && !w->rc) w->rc = rc;
  }
  return NULL;
}

/* orc_step with the elements split into nthreads contiguous ranges, one thread each: every
 * thread applies the scheme to the unknowns of its elements and evaluates the right-hand side
 * there, with a barrier before and after each evaluation (the stage arguments of neighbouring
 * elements are read across ranges).  Each unknown gets exactly the operations of orc_step, so
 * the result is bitwise that of orc_step.  For timing only; the checker is orc_step. */
int orc_step_threads(const orc_problem* p, double* U, double dt, int nsteps, int rk, int nthreads) {
  if (check_problem(p) || nsteps < 0 || !(dt > 0.0) || (rk != 3 && rk != 4 && rk != 6)) return -1;
  if (nthreads < 1 || nthreads > 4096) return -1;
  const int64_t nd = orc_ndof(p), nv = nvar_of(p), np = ipow(p->degree + 1, p->dim);
  const int64_t ne = nd / nv / np;
  if (nthreads > ne) nthreads = (int)ne;
  double* work = (double*)malloc(sizeof(double) * 9 * (size_t)nd);
  orc_worker* ws = (orc_worker*)calloc((size_t)nthreads, sizeof(orc_worker));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!work || !ws || !th) {
    free(work);
    free(ws);
    free(th);
    return -2;
  }
  orc_barrier bar;
  pthread_mutex_init(&bar.mu, NULL);
  pthread_cond_init(&bar.cv, NULL);
  bar.count = 0;
  bar.total = nthreads;
  bar.generation = 0;
  for (int t = 0; t < nthreads; ++t) {
    orc_worker* w = &ws[t];
    const int64_t e0 = ne * t / nthreads, e1 = ne * (t + 1) / nthreads;
    w->p = p, w->U = U, w->work = work, w->dt = dt, w->nsteps = nsteps, w->rk = rk;
    for (int v = 0; v < nv; ++v) {
      w->lo[v] = (v * ne + e0) * np;
      w->hi[v] = (v * ne + e1) * np;
    }
    w->part.lo = w->lo, w->part.hi = w->hi, w->part.nspans = (int)nv;
    w->part.e_begin = e0, w->part.e_end = e1;
    w->part.sync = nthreads > 1 ? barrier_wait : NULL;
    w->part.sync_ctx = &bar;
  }
  int started = 0, rc = 0;
  for (int t = 1; t < nthreads; ++t) {
    if (pthread_create(&th[t], NULL, worker_main, &ws[t]) != 0) {
      rc = -3;
      break;
    }
    ++started;
  }
  if (rc == 0) {
    worker_main(&ws[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads && rc == 0; ++t) rc = ws[t].rc;
  } else {
    /* a thread could not start: the barrier counts the ones that did (and this one), they all
     * run to the end (on a partial split, so the result is not used), then the call fails */
    pthread_mutex_lock(&bar.mu);
    bar.total = started + 1;
    if (bar.count == bar.total) {
      bar.count = 0;
      ++bar.generation;
      pthread_cond_broadcast(&bar.cv);
    }
    pthread_mutex_unlock(&bar.mu);
    worker_main(&ws[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
  }
  pthread_mutex_destroy(&bar.mu);
  pthread_cond_destroy(&bar.cv);
  free(work);
  free(ws);
  free(th);
  return rc;
}

/* Scalar ODE test problems for the Runge-Kutta code alone:
 * which = 0: y' = lambda y;  which = 1: y' = -y^2. */
typedef struct { int which; double lambda; } ode_ctx;

static int ode_rhs(const void* ctx, const double* y, double* f, const orc_part* part) {
  const ode_ctx* c = (const ode_ctx*)ctx;
  (void)part;
  f[0] = c->which == 0 ? c->lambda * y[0] : -y[0] * y[0];
  return 0;
}

int orc_rk_ode(int rk, int which, double lambda, double y0, double dt, int nsteps, double* y) {
  double work[9];
  ode_ctx c = {which, lambda};
  const int64_t lo = 0, hi = 1;
  const orc_part one = {&lo, &hi, 1, 0, 1, NULL, NULL};
  y[0] = y0;
  for (int s = 0; s < nsteps; ++s)
    if (rk_advance(rk, 1, y, dt, ode_rhs, &c, work, &one)) return -1;
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Norms (Sec. 3.1) by LGL quadrature, and the time-step rule (reading 7)                        */
/* ------------------------------------------------------------------------------------------ */

/* out[0] = L2 = sqrt(int sum_v (U_v - ref_v)^2), out[1] = Linf = max |U - ref| (ref may be NULL,
 * then ref = 0), out[2 + v] = int U_v (mass, momentum), out[6] = number of non-finite values. */
int orc_norms(const orc_problem* p, const double* U, const double* ref, double* out) {
  if (check_problem(p)) return -1;
  int N = p->degree, n = N + 1, d = p->dim, nv = nvar_of(p);
  double xi[ORC_MAXN], w[ORC_MAXN];
  orc_lgl(N, xi, w);
  int E[3] = {1, 1, 1};
  double J = 1.0;
  for (int a = 0; a < d; ++a) {
    E[a] = p->elems[a];
    J *= 0.5 * p->length[a] / E[a];
  }
  int np = ipow(n, d);
  int64_t ne = (int64_t)E[0] * E[1] * E[2];
  double l2 = 0.0, linf = 0.0, integral[4] = {0, 0, 0, 0}, nonfinite = 0.0;
  for (int v = 0; v < nv; ++v)
    for (int64_t e = 0; e < ne; ++e)
      for (int node = 0; node < np; ++node) {
        int ii[3] = {node % n, (node / n) % n, node / (n * n)};
        double wq = J;
        for (int a = 0; a < d; ++a) wq *= w[ii[a]];
        double x = U[((int64_t)v * ne + e) * np + node];
        if (!isfinite(x)) nonfinite += 1.0;
        double diff = ref ? x - ref[((int64_t)v * ne + e) * np + node] : x;
        l2 += wq * diff * diff;
        linf = fmax(linf, fabs(diff));
        integral[v] += wq * x;
      }
  out[0] = sqrt(l2);
  out[1] = linf;
  for (int v = 0; v < 4; ++v) out[2 + v] = integral[v];
  out[6] = nonfinite;
  return 0;
}

double orc_stable_dt(const orc_problem* p, const double* U, double cfl) {
  if (check_problem(p)) return -1.0;
  int N = p->degree, n = N + 1, d = p->dim;
  double xi[ORC_MAXN], w[ORC_MAXN];
  orc_lgl(N, xi, w);
  double gap = 2.0;
  for (int k = 0; k < N; ++k) gap = fmin(gap, xi[k + 1] - xi[k]);
  double hmin = 1e300;
  for (int a = 0; a < d; ++a) hmin = fmin(hmin, 0.5 * p->length[a] / p->elems[a] * gap);
  double lambda = 0.0;
  if (p->equation == ORC_ADVECTION) {
    for (int a = 0; a < d; ++a) lambda += fabs(p->velocity[a]);
  } else {
    int64_t nodes = orc_ndof(p) / (d + 1);
    for (int64_t q = 0; q < nodes; ++q) {
      double s = 0.0;
      for (int a = 0; a < d; ++a) s += fabs(U[(int64_t)(1 + a) * nodes + q] / U[q]);
      lambda = fmax(lambda, s + d * p->sound_speed);
    }
  }
  (void)n;
  if (!(lambda > 0.0)) return -1.0;
  return cfl * hmin / lambda;
}
