// Node-per-thread variant of the fused NDG stage kernel, for the bandwidth-bound FP32 path.
//
// Same method and same work list as stage_kernel (stage_kernel.cuh); what differs is the
// mapping.  Each thread owns one node of one element, for every variable:
//   1. it issues all of its global reads of the stage at once -- the node of the stage input,
//      U^n / ACC for the update, and (on element faces) the neighbour's trace -- so that their
//      latencies overlap, and copies the stage input into the shared tile (unpadded: the
//      line-wise reads below are free of bank conflicts in this mapping);
//   2. isothermal Euler: it evaluates the fluxes of its node along every axis into shared memory;
//   3. per axis it contracts its own row of D (held in registers) with the line through its
//      node, so the right-hand side of its node accumulates in registers across axes;
//   4. face nodes add the lifted numerical-flux term;
//   5. it applies the stage update to its node.
// The element tile is the same as in stage_kernel; a tile never changes any element's
// arithmetic, so results do not depend on the tile size.  The plain (n-term) contraction is
// used: on the FP32 path the arithmetic is not the limit, memory is.
#pragma once

#include "stage_kernel.cuh"

namespace ndg {

template <int DIM, int N, int EQ, typename real>
struct NpGeom {
  static constexpr int n = N + 1;
  static constexpr int NPE = ipow_c(n, DIM);
  static constexpr int NV = EQ == 0 ? 1 : DIM + 1;
  // shared arrays of NPE per element: the tile, plus DIM x DIM momentum fluxes for Euler
  static constexpr int NS = EQ == 0 ? NV : NV + DIM * DIM;
};

template <int DIM, int N, int EQ, typename real>
__global__ void __launch_bounds__(512, 2) stage_kernel_np(const StageArgs<real> args) {
  using G = NpGeom<DIM, N, EQ, real>;
  constexpr int n = G::n, NPE = G::NPE, NV = G::NV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GroupHeader hdr = *args.hdr;
  const int epb = hdr.epb;
  real* sU = reinterpret_cast<real*>(smem_raw);  // [NV][epb][NPE]
  real* sF = sU + NV * epb * NPE;                 // Euler: [a][b][epb][NPE], flux of m_b along a
  const int tid = threadIdx.x;
  const int el = tid / NPE;
  const int node = tid - el * NPE;
  int idx[3] = {node % n, (node / n) % n, node / (n * n)};
  constexpr int stride[3] = {1, n, n * n};
  const StagePlan& plan = args.plan;

  // this thread's row of D along every axis
  real Drow[DIM][n];
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int m = 0; m < n; ++m) Drow[a][m] = args.basis.D[idx[a] * n + m];

  SolveRegs<DIM, real> S;
  for (int tile = blockIdx.x; tile < hdr.ntiles; tile += gridDim.x) {
    const int si = hdr.nsolves > 1 ? find_solve(args.solves, hdr.nsolves, tile) : 0;
    if (si != S.index) S.load(args.solves + si, si, plan);
    const long long nelem = S.nelem;
    const long long e0 = (long long)(tile - S.tile_begin) * epb;
    const int cnt = (int)min((long long)epb, nelem - e0);
    const long long vstride = nelem * NPE;
    const bool active = el < cnt;
    const long long e = e0 + el;
    const long long g = e * NPE + node;  // offset of this node within one variable

    // ---- 1. all global reads of this node up front ----
    real u[NV], base[NV], accv[NV];
    real xt[DIM][NV];  // exterior trace on the face this node lies on (per axis), if any
    bool xt_smem[DIM];
    int xt_el[DIM];
    if (active) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        u[v] = S.uin[v * vstride + g];
        if (plan.in != kUN && plan.acc_mode != 3) base[v] = S.un[v * vstride + g];
        if (plan.acc_mode >= 2) accv[v] = S.acc[v * vstride + g];
        sU[(v * epb + el) * NPE + node] = u[v];
      }
      // element indices fit in 32 bits (checked at creation): 32-bit index arithmetic only
      const unsigned eu = (unsigned)e;
      const unsigned E0 = S.E0, E1 = S.E1;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        xt_smem[a] = true;
        xt_el[a] = 0;
        const bool at_lo = idx[a] == 0, at_hi = idx[a] == N;
        if (!at_lo && !at_hi) continue;
        if (EQ == 0 && (at_lo ? S.qlo[a] : S.qhi[a]) == real(0)) continue;  // downwind face
        unsigned en;
        if (a == 0) {
          const unsigned ex = eu % E0;
          en = at_lo ? eu - ex + (ex == 0 ? E0 - 1 : ex - 1) : eu - ex + (ex == E0 - 1 ? 0 : ex + 1);
        } else if (a == 1) {
          const unsigned ey = (eu / E0) % E1;
          en = at_lo ? (ey == 0 ? eu + (E1 - 1) * E0 : eu - E0) : (ey == E1 - 1 ? eu - (E1 - 1) * E0 : eu + E0);
        } else {
          const unsigned step = E0 * E1, E2 = S.E2;
          const unsigned ez = eu / step;
          en = at_lo ? (ez == 0 ? eu + (E2 - 1) * step : eu - step) : (ez == E2 - 1 ? eu - (E2 - 1) * step : eu + step);
        }
        // the neighbour's node facing this one: index N on the low side, 0 on the high side
        const int nnode = node + (at_lo ? N : -N) * stride[a];
        if ((long long)en >= e0 && (long long)en < e0 + cnt) {
          xt_el[a] = (int)((long long)en - e0) * NPE + nnode;  // read from the shared tile after the barrier
        } else {
          xt_smem[a] = false;
#pragma unroll
          for (int v = 0; v < NV; ++v) xt[a][v] = S.uin[v * vstride + (long long)en * NPE + nnode];
        }
      }
    }
    __syncthreads();

    real rhs[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) rhs[v] = real(0);
    real vel[DIM];
    if constexpr (EQ == 1) {
      // ---- 2. fluxes of the momentum components along every axis (Eq. (eulerIso2d)) ----
      if (active) {
        const real inv = real(1) / u[0];
        const real c2rho = S.c2 * u[0];
#pragma unroll
        for (int a = 0; a < DIM; ++a) vel[a] = u[1 + a] * inv;
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
          for (int b = 0; b < DIM; ++b) {
            real f = u[1 + b] * vel[a];
            if (a == b) f += c2rho;
            sF[((a * DIM + b) * epb + el) * NPE + node] = f;
          }
      }
      __syncthreads();
    }

    if (active) {
      // ---- 3. volume term: own row of D against the line through this node ----
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const int lbase = node - idx[a] * stride[a];
        const real vs = S.vs[a];
        const bool unit = (a == 0) && vs == real(1);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const real* line;
          if (EQ == 0 || v == 0) line = sU + ((EQ == 0 ? 0 : 1 + a) * epb + el) * NPE + lbase;  // F = u or m_a
          else line = sF + ((a * DIM + (v - 1)) * epb + el) * NPE + lbase;
          real c = Drow[a][0] * line[0];
#pragma unroll
          for (int m = 1; m < n; ++m) c = fma(Drow[a][m], line[m * stride[a]], c);
          rhs[v] = unit ? rhs[v] + c : fma(vs, c, rhs[v]);
        }
        // ---- 4. lifted face term on this axis ----
        const bool at_lo = idx[a] == 0, at_hi = idx[a] == N;
        const real q = at_lo ? S.qlo[a] : S.qhi[a];
        if ((at_lo || at_hi) && (EQ == 1 || q != real(0))) {
          real x[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) x[v] = xt_smem[a] ? sU[v * epb * NPE + xt_el[a]] : xt[a][v];
          if constexpr (EQ == 0) {
            // advection: lo face q (x - u), hi face q (u - x); q = 0 on the downwind face
            rhs[0] = fma(q, at_lo ? x[0] - u[0] : u[0] - x[0], rhs[0]);
          } else {
            const real xin = real(1) / x[0];
            const real xun = x[1 + a] * xin;
            const real alpha = fmax(fabs(vel[a]), fabs(xun)) + S.c;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              real fo, fx;  // own and exterior flux component v along a
              if (v == 0) {
                fo = u[1 + a];
                fx = x[1 + a];
              } else {
                fo = u[v] * vel[a] + (v == 1 + a ? S.c2 * u[0] : real(0));
                fx = x[v] * xun + (v == 1 + a ? S.c2 * x[0] : real(0));
              }
              // lo: 1/2 (F(ext) - F(U_0) - alpha (U_0 - ext)); hi: 1/2 (F(U_N) - F(ext) + alpha (ext - U_N))
              const real term = at_lo ? fma(-alpha, u[v] - x[v], fx - fo) : fma(alpha, x[v] - u[v], fo - fx);
              rhs[v] = fma(q, term, rhs[v]);
            }
          }
        }
      }
      // ---- 5. stage update of this node ----
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const long long gv = v * vstride + g;
        const real r = rhs[v];
        if (plan.acc_mode == 3) {
          S.uout[gv] = fma(S.bdt, r, accv[v]);
          continue;
        }
        const real b = plan.in == kUN ? u[v] : base[v];
        real o = fma(S.a_self, r, b);
        for (int j = 0; j < plan.nread; ++j) {  // stored slopes (RK6)
          const real* kj = static_cast<const real*>(args.solves[si].buf[plan.kread[j]]);
          o = fma(S.a_read(plan, j), kj[gv], o);
        }
        S.uout[gv] = o;
        if (plan.acc_mode == 1) S.acc[gv] = fma(S.bdt, r, b);
        else if (plan.acc_mode == 2) S.acc[gv] = fma(S.bdt, r, accv[v]);
        if (S.kw) S.kw[gv] = r;
      }
    }
    __syncthreads();
  }
}

template <int DIM, int N, int EQ, typename real>
void stage_np_shape(int epb, int* threads, size_t* smem) {
  using G = NpGeom<DIM, N, EQ, real>;
  *threads = epb * G::NPE;
  *smem = (size_t)G::NS * epb * G::NPE * sizeof(real);
}

}  // namespace ndg
