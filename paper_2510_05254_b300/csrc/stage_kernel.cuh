// Fused NDG right-hand side + Runge-Kutta stage update (one launch per RK stage).
//
// Method (arXiv:2510.05254, Sec. 2.1-2.3), strong form of the collocated LGL scheme: along every
// axis a of a tensor-product element, for every line of n = N+1 nodes,
//   dU_l/dt += -(2/h_a) (D F_a)_l
//              + (2/h_a)/w_0 (Fhat_lo - F_a(U_0)) delta_{l0}
//              + (2/h_a)/w_N (F_a(U_N) - Fhat_hi) delta_{lN},
// which equals the paper's weak form (volume integral by LGL quadrature, lumped mass of
// Eq. (lag_coefs)) through the summation-by-parts identity W D + D^T W = diag(-1, 0.., 1).
// Fhat is the Lax-Friedrichs flux of Eq. (LF): for advection the upwind flux, for isothermal
// Euler alpha = max(|u_a^-|, |u_a^+|) + c.  The stage update applies the Butcher tableau of
// Eq. (RK3)/(RK4)/(RK6) as described by StagePlan.
//
// With the exact mass matrix (EXACT instantiations) the two lift terms reach every node of the
// line through M^-1 e_0 and M^-1 e_N instead of 1/w_0 and 1/w_N at the ends.
//
// Work decomposition: a CTA owns a tile of `epb` consecutive elements (in the element layout a
// contiguous chunk of every variable).  Phases, separated by __syncthreads:
//   1. copy the tile of the stage input into shared memory: cp.async into the padded layout
//      (x-lines one slot apart), 16-byte cp.async into the aligned FP32 2D layout, one TMA bulk
//      copy per variable into the unpadded FP32 degree-5 layout, or one per 256-byte plane into
//      the plane-padded FP32 3D degree-7 layout (see StageGeom);
//   2. Euler, FP64: velocities u_a = m_a / rho per node into shared memory (FP32 recomputes them
//      per line);
//   3. for each axis a: one thread per line of n nodes evaluates the flux along the line,
//      applies D by its even-odd halves (D is centro-antisymmetric on LGL nodes), adds the
//      lifted face terms at the two ends (neighbour traces from global memory / L2, or from a
//      partition halo; the FP32 degree-7 2D layout and axes with halos read a neighbour inside
//      the tile from shared memory), and accumulates into the shared right-hand side;
//   4. node-parallel stage update with coalesced global reads/writes, four nodes per step in the
//      FP32 16-byte layouts (2D FP64: fused into the y-line pass instead, each thread updating
//      the nodes of its line).
// The grid is persistent: CTAs loop over the tiles of every solve of the launch.
#pragma once

#include <cuda_runtime.h>

#include "ndg_internal.h"
#include "stage_ff.cuh"

namespace ndg {

constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }

// Basis of one degree in the launch's precision, passed by value (lives in the kernel's
// constant bank, so the contraction's coefficients are constant operands).
template <typename real>
struct BasisArgs {
  real Ae[16];   // [i*4 + m], i, m < n/2
  real Bo[16];
  real Cmid[4];  // D[i][mid], odd n
  real Dmid[4];  // D[mid][m], odd n
  real Llo[8];   // exact mass: w_0 (M^-1 e_0)_l, the lift of the low face term onto node l
  real Lhi[8];   // exact mass: w_N (M^-1 e_N)_l
};

// The even-odd halves in FP32 with every coefficient twice, (c, c): operands of the paired FP32
// instructions (FFMA2 / FMUL2) that apply one coefficient to two variables at once.
struct BasisPairs {
  float2 Ae[16];
  float2 Bo[16];
};

template <typename real>
struct StageArgs {
  const SolveDesc* solves;
  const GroupHeader* hdr;
  StagePlan plan;
  BasisArgs<real> basis;
  BasisFF bff;     // float-float halves of the same tables (FP64 path with float-float contraction)
  BasisPairs bp;   // paired FP32 halves (FP32 3D isothermal Euler at degrees 5 and 7)
};

// Per-solve coefficients in the kernel's precision (no conversion in device code).
template <typename real> struct Coef;
template <> struct Coef<double> {
  __device__ static double vol(const SolveDesc* s, int a) { return s->vol_scale[a]; }
  __device__ static double lo(const SolveDesc* s, int a) { return s->lift_lo[a]; }
  __device__ static double hi(const SolveDesc* s, int a) { return s->lift_hi[a]; }
  __device__ static double c(const SolveDesc* s) { return s->c; }
  __device__ static double c2(const SolveDesc* s) { return s->c2; }
};
template <> struct Coef<float> {
  __device__ static float vol(const SolveDesc* s, int a) { return s->f_vol_scale[a]; }
  __device__ static float lo(const SolveDesc* s, int a) { return s->f_lift_lo[a]; }
  __device__ static float hi(const SolveDesc* s, int a) { return s->f_lift_hi[a]; }
  __device__ static float c(const SolveDesc* s) { return s->f_c; }
  __device__ static float c2(const SolveDesc* s) { return s->f_c2; }
};

// The fields of the solve a tile belongs to, kept in registers while consecutive tiles of a CTA
// belong to the same solve (always, for a single-solve launch): re-reading the descriptor per
// tile costs a dozen loads per thread and tile.
template <int DIM, typename real>
struct SolveRegs {
  int index = -1;
  int tile_begin;
  long long nelem;
  unsigned E0, E1, E2;
  const real* uin;
  const real* un;
  real* acc;
  real* uout;
  real* kw;
  real vs[DIM], qlo[DIM], qhi[DIM];
  real c, c2;
  real a_self, bdt, dts;  // a_self * dt', b * dt', dt' = dt * rhs_scale
  const real* halo_lo[DIM];
  const real* halo_hi[DIM];

  __device__ __forceinline__ void load(const SolveDesc* sd, int i, const StagePlan& plan) {
    index = i;
    tile_begin = sd->tile_begin;
    nelem = sd->nelem;
    E0 = (unsigned)sd->E[0];
    E1 = (unsigned)sd->E[1];
    E2 = (unsigned)sd->E[2];
    uin = static_cast<const real*>(sd->buf[plan.in]);
    un = static_cast<const real*>(sd->buf[kUN]);
    acc = static_cast<real*>(sd->buf[kACC]);
    uout = static_cast<real*>(sd->buf[plan.out]);
    kw = plan.kwrite >= 0 ? static_cast<real*>(sd->buf[plan.kwrite]) : nullptr;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      vs[a] = Coef<real>::vol(sd, a);
      qlo[a] = Coef<real>::lo(sd, a);
      qhi[a] = Coef<real>::hi(sd, a);
      halo_lo[a] = static_cast<const real*>(sd->halo_lo[a]);
      halo_hi[a] = static_cast<const real*>(sd->halo_hi[a]);
    }
    c = Coef<real>::c(sd);
    c2 = Coef<real>::c2(sd);
    const double dt = sd->dt * sd->rhs_scale;  // the kernels hold L(U) / rhs_scale
    a_self = (real)(plan.a_self * dt);
    bdt = (real)(plan.b * dt);
    dts = (real)dt;
  }
  // coefficient of stored slope j in the stage combination (RK6)
  __device__ __forceinline__ real a_read(const StagePlan& plan, int j) const {
    if constexpr (sizeof(real) == 4) return plan.a_read_f[j] * dts;
    else return plan.a_read[j] * dts;
  }
};

// Index of the solve owning `tile` (binary search over tile_begin; none for one solve).
__device__ __forceinline__ int find_solve(const SolveDesc* solves, int nsolves, int tile) {
  int lo = 0, hi = nsolves - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (solves[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Asynchronous global -> shared copy of one element (cp.async, no register round trip); many
// can be in flight per thread.  Completed by cp_async_wait_all().
template <typename real>
__device__ __forceinline__ void cp_async_elem(real* smem_dst, const real* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  if constexpr (sizeof(real) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
// Bulk (TMA) copies of contiguous global blocks into shared memory, completed on an mbarrier
// that counts the bytes: one thread arms the barrier with the total and issues the copies, every
// thread waits for the phase.  The wait is bounded: it gives up after a number of polls (each of
// which may suspend the thread for a while; kBulkWaitPolls unless the launch's header sets
// another), and the caller then reports the failure.
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(s) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(s), "r"(bytes) : "memory");
}
// global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_copy(void* smem_dst, const void* gmem_src, unsigned bytes,
                                          unsigned long long* bar) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(d),
               "l"(gmem_src), "r"(bytes), "r"(b)
               : "memory");
}
// true once the barrier's phase of the given parity has completed; false if the polls ran out
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int polls) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(bar);
  for (int i = 0; i < polls; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(s), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// L2 prefetch of `bytes` (a multiple of 16) from a 16-byte aligned global address by the bulk
// copy engine: one instruction for a whole range, nothing to wait for
__device__ __forceinline__ void bulk_prefetch_l2(const void* gmem, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async_16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

template <int N, typename real>
__device__ __forceinline__ void contract_even_odd(const real (&f)[N + 1], real (&out)[N + 1],
                                                  const BasisArgs<real>& B) {
  constexpr int n = N + 1;
  constexpr int H = n / 2;
  real fe[H], fo[H];
#pragma unroll
  for (int m = 0; m < H; ++m) {
    fe[m] = f[m] + f[N - m];
    fo[m] = f[m] - f[N - m];
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    real E = B.Ae[i * 4] * fo[0];
    real O = B.Bo[i * 4] * fe[0];
#pragma unroll
    for (int m = 1; m < H; ++m) {
      E = fma(B.Ae[i * 4 + m], fo[m], E);
      O = fma(B.Bo[i * 4 + m], fe[m], O);
    }
    if (n % 2 == 1) O = fma(B.Cmid[i], f[H], O);
    out[i] = E + O;
    out[N - i] = E - O;
  }
  if (n % 2 == 1) {
    real M = B.Dmid[0] * fo[0];
#pragma unroll
    for (int m = 1; m < H; ++m) M = fma(B.Dmid[m], fo[m], M);
    out[H] = M;
  }
}

// Quotient in the kernel's precision: IEEE division in FP64; in FP32 the reciprocal-based
// __fdividef (2 ulp), well inside the FP32 path's tolerance and a fraction of the instructions.
__device__ __forceinline__ double ratio(double a, double b) { return a / b; }
__device__ __forceinline__ float ratio(float a, float b) { return __fdividef(a, b); }

// A product rounded on its own: the compiler may not contract it into a following add.  Where a
// flux is a plain product, letting the compiler choose would make the rounding depend on the
// surrounding code, and the two thread mappings would no longer agree bit for bit.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// Runge-Kutta stage update of one node (the Butcher tableau of Eq. (RK3)/(RK4)/(RK6) as the
// StagePlan states it): r = L(U) / rhs_scale at the node, bb = U^n there (read unless the last
// stage), aa = ACC there (read when it accumulates), g = its global index.
template <int DIM, typename real>
__device__ __forceinline__ void stage_update_node(const StageArgs<real>& args, const SolveRegs<DIM, real>& S, int si,
                                                  const StagePlan& plan, long long g, real r, real bb, real aa) {
  if (plan.acc_mode == 3) {
    S.uout[g] = fma(S.bdt, r, aa);
    return;
  }
  real o = fma(S.a_self, r, bb);
  for (int j = 0; j < plan.nread; ++j) {
    const real* kj = static_cast<const real*>(args.solves[si].buf[plan.kread[j]]);
    o = fma(S.a_read(plan, j), kj[g], o);
  }
  S.uout[g] = o;
  if (plan.acc_mode == 1) S.acc[g] = fma(S.bdt, r, bb);
  else if (plan.acc_mode == 2) S.acc[g] = fma(S.bdt, r, aa);
  if (S.kw) S.kw[g] = r;
}

// s x + y lane by lane (four FMAs, each rounded as the scalar one)
__device__ __forceinline__ float4 fma4(float s, float4 x, float4 y) {
  return make_float4(fmaf(s, x.x, y.x), fmaf(s, x.y, y.y), fmaf(s, x.z, y.z), fmaf(s, x.w, y.w));
}

// The update of four consecutive nodes g .. g + 3 (16-byte aligned in every array), FP32: r and
// the stage input (U^n at the first stage) read as float4 from shared memory, U^n / ACC as float4
// from global memory; the same arithmetic as stage_update_node, node by node.
template <int DIM>
__device__ __forceinline__ void stage_update_quad(const StageArgs<float>& args, const SolveRegs<DIM, float>& S, int si,
                                                  const StagePlan& plan, long long g, const float* sr, const float* su) {
  const float4 r = *reinterpret_cast<const float4*>(sr);
  float4 b = make_float4(0.f, 0.f, 0.f, 0.f), a = b;
  if (plan.acc_mode >= 2) a = __ldg(reinterpret_cast<const float4*>(S.acc + g));
  if (plan.acc_mode != 3)
    b = plan.in == kUN ? *reinterpret_cast<const float4*>(su) : __ldg(reinterpret_cast<const float4*>(S.un + g));
  if (plan.acc_mode == 3) {
    *reinterpret_cast<float4*>(S.uout + g) =
        make_float4(fmaf(S.bdt, r.x, a.x), fmaf(S.bdt, r.y, a.y), fmaf(S.bdt, r.z, a.z), fmaf(S.bdt, r.w, a.w));
    return;
  }
  if (plan.nread > 0) {
    // stored slopes (RK6): the four nodes at once, one float4 load per slope; per node the
    // operations and their order are stage_update_node's
    float4 o = fma4(S.a_self, r, b);
    for (int j = 0; j < plan.nread; ++j) {
      const float* kj = static_cast<const float*>(args.solves[si].buf[plan.kread[j]]);
      o = fma4(S.a_read(plan, j), __ldg(reinterpret_cast<const float4*>(kj + g)), o);
    }
    *reinterpret_cast<float4*>(S.uout + g) = o;
    if (plan.acc_mode == 1) *reinterpret_cast<float4*>(S.acc + g) = fma4(S.bdt, r, b);
    else if (plan.acc_mode == 2) *reinterpret_cast<float4*>(S.acc + g) = fma4(S.bdt, r, a);
    if (S.kw) *reinterpret_cast<float4*>(S.kw + g) = r;
    return;
  }
  *reinterpret_cast<float4*>(S.uout + g) =
      make_float4(fmaf(S.a_self, r.x, b.x), fmaf(S.a_self, r.y, b.y), fmaf(S.a_self, r.z, b.z), fmaf(S.a_self, r.w, b.w));
  if (plan.acc_mode == 1)
    *reinterpret_cast<float4*>(S.acc + g) =
        make_float4(fmaf(S.bdt, r.x, b.x), fmaf(S.bdt, r.y, b.y), fmaf(S.bdt, r.z, b.z), fmaf(S.bdt, r.w, b.w));
  else if (plan.acc_mode == 2)
    *reinterpret_cast<float4*>(S.acc + g) =
        make_float4(fmaf(S.bdt, r.x, a.x), fmaf(S.bdt, r.y, a.y), fmaf(S.bdt, r.z, a.z), fmaf(S.bdt, r.w, a.w));
  if (S.kw) *reinterpret_cast<float4*>(S.kw + g) = r;
}
template <int DIM>
__device__ __forceinline__ void stage_update_quad(const StageArgs<double>&, const SolveRegs<DIM, double>&, int,
                                                  const StagePlan&, long long, const double*, const double*) {}

// Where a line's two neighbour traces come from (element indices fit in 32 bits, checked at
// creation): the periodic neighbours along axis a, or a partition halo on a partition boundary.
struct LineTrace {
  long long elo, ehi;   // neighbour elements
  bool lo_halo, hi_halo;
  long long hoff, hvs;  // halo offset of this line's face node (variable 0), stride per variable
};

// Element coordinates of element index eu: two divisions, once per thread and tile, instead of
// several per axis and line.
struct ElemXYZ {
  unsigned x, y, z;
};
__device__ __forceinline__ ElemXYZ elem_xyz(unsigned eu, unsigned E0, unsigned E1) {
  const unsigned r = eu / E0;
  return ElemXYZ{eu - r * E0, r % E1, r / E1};
}

template <int L>
__device__ __forceinline__ LineTrace line_trace(int a, unsigned eu, ElemXYZ c, int line, unsigned E0, unsigned E1,
                                                unsigned E2, bool halo_lo, bool halo_hi) {
  LineTrace t;
  unsigned lo_, hi_, te, ca, Ea, ntrans;
  if (a == 0) {
    ca = c.x; Ea = E0; te = c.y + E1 * c.z; ntrans = E1 * E2;
    lo_ = c.x == 0 ? eu + (E0 - 1) : eu - 1;
    hi_ = c.x == E0 - 1 ? eu - (E0 - 1) : eu + 1;
  } else if (a == 1) {
    ca = c.y; Ea = E1; te = c.x + E0 * c.z; ntrans = E0 * E2;
    lo_ = c.y == 0 ? eu + (E1 - 1) * E0 : eu - E0;
    hi_ = c.y == E1 - 1 ? eu - (E1 - 1) * E0 : eu + E0;
  } else {
    const unsigned step = E0 * E1;
    ca = c.z; Ea = E2; te = c.x + E0 * c.y; ntrans = step;
    lo_ = c.z == 0 ? eu + (E2 - 1) * step : eu - step;
    hi_ = c.z == E2 - 1 ? eu - (E2 - 1) * step : eu + step;
  }
  t.elo = lo_;
  t.ehi = hi_;
  t.lo_halo = ca == 0 && halo_lo;
  t.hi_halo = ca == Ea - 1 && halo_hi;
  t.hoff = (long long)te * L + line;
  t.hvs = (long long)ntrans * L;  // transverse elements x lines: one variable's halo
  return t;
}

// (x-lines in shared memory start RS slots apart: RS = n + 1, or a multiple of 4 for 16-byte access;
// 3D planes of n x-lines start PS slots apart, RS n unless the planes are padded)
template <int n, int RS, int PS = RS * n>
__device__ __forceinline__ void line_geometry(int a, int line, int& pbase, int& pstride, int& ubase, int& ustride) {
  if (a == 0) {
    if constexpr (PS == RS * n) pbase = RS * line;
    else pbase = RS * (line % n) + PS * (line / n);
    pstride = 1; ubase = n * line; ustride = 1;
  } else if (a == 1) {
    const int i = line % n, k = line / n;
    pbase = i + PS * k; pstride = RS; ubase = i + n * n * k; ustride = n;
  } else {
    pbase = line % n + RS * (line / n); pstride = PS; ubase = line; ustride = n * n;
  }
}

// One line of n values from shared memory into registers and back.  W > 1 (FP32 only): the line
// is contiguous and 4W-byte aligned and moves as float2 / float4; V switches it on per call.
template <int n, int W, typename real>
__device__ __forceinline__ void load_line(const real* p, int stride, bool V, real (&f)[n]) {
  if constexpr (sizeof(real) == 4 && W == 4 && n % 4 == 0) {
    if (V) {
#pragma unroll
      for (int c = 0; c < n / 4; ++c) {
        const float4 q = reinterpret_cast<const float4*>(p)[c];
        f[4 * c] = q.x; f[4 * c + 1] = q.y; f[4 * c + 2] = q.z; f[4 * c + 3] = q.w;
      }
      return;
    }
  } else if constexpr (sizeof(real) == 4 && W == 2 && n % 2 == 0) {
    if (V) {
#pragma unroll
      for (int c = 0; c < n / 2; ++c) {
        const float2 q = reinterpret_cast<const float2*>(p)[c];
        f[2 * c] = q.x; f[2 * c + 1] = q.y;
      }
      return;
    }
  }
#pragma unroll
  for (int l = 0; l < n; ++l) f[l] = p[l * stride];
}
template <int n, int W, typename real>
__device__ __forceinline__ void store_line(real* p, int stride, bool V, const real (&f)[n]) {
  if constexpr (sizeof(real) == 4 && W == 4 && n % 4 == 0) {
    if (V) {
#pragma unroll
      for (int c = 0; c < n / 4; ++c)
        reinterpret_cast<float4*>(p)[c] = make_float4(f[4 * c], f[4 * c + 1], f[4 * c + 2], f[4 * c + 3]);
      return;
    }
  } else if constexpr (sizeof(real) == 4 && W == 2 && n % 2 == 0) {
    if (V) {
#pragma unroll
      for (int c = 0; c < n / 2; ++c) reinterpret_cast<float2*>(p)[c] = make_float2(f[2 * c], f[2 * c + 1]);
      return;
    }
  }
#pragma unroll
  for (int l = 0; l < n; ++l) p[l * stride] = f[l];
}

// D along one line: FP64 / FP32 even-odd products, or (FF) the float-float version of the same,
// with the FP64 one for a line holding a value that cannot be split into normal floats.
template <int N, typename real, bool FF>
__device__ __forceinline__ void contract_line(const real (&f)[N + 1], real (&out)[N + 1], const StageArgs<real>& args) {
  if constexpr (FF) {
    ff fd[N + 1];
    bool ok = true;
#pragma unroll
    for (int l = 0; l <= N; ++l) ok = ff_split(f[l], fd[l].h, fd[l].l) && ok;
    if (ok) {
      ff od[N + 1];
      contract_even_odd_ff<N>(fd, od, args.bff);
#pragma unroll
      for (int l = 0; l <= N; ++l) out[l] = ff_to_double(od[l]);
      return;
    }
  }
  contract_even_odd<N>(f, out, args.basis);
}

// A bulk-copy wait ran out: flag the launch and every solve in it (the CTA that gives up leaves
// tiles of any of them unprocessed), for the host to report.  Called by one thread.
template <typename real>
__device__ __noinline__ void flag_failure(const StageArgs<real>& args) {
  GroupHeader* h = const_cast<GroupHeader*>(args.hdr);
  atomicExch(&h->err, kStageErrBulkWait);
  const int ns = h->nsolves;
  for (int i = 0; i < ns; ++i)
    if (args.solves[i].status) atomicExch(args.solves[i].status, kStageErrBulkWait);
}

template <int DIM, int N, int EQ, typename real, bool VS = false, bool FF = false>
struct StageGeom {
  static constexpr int n = N + 1;
  static constexpr int L = ipow_c(n, DIM - 1);      // lines per element along one axis
  static constexpr int NPE = ipow_c(n, DIM);        // nodes per element
  static constexpr int NV = EQ == 0 ? 1 : DIM + 1;  // variables
  // VEC (FP32 2D, n = 8 or 4): x-lines 16-byte aligned in shared memory, so the tile copy, the
  // x-line passes and the stage update move four values per instruction.  Row stride RS: an odd
  // number of 16-byte chunks, so eight threads reading eight rows' chunks hit distinct banks;
  // element stride SPE = 8 (mod 32) banks for n = 8 (20 for n = 4), so a warp's y-lines in four
  // (eight) elements do too.  (n = 4: a quarter-warp's float4 rows span two elements and are
  // 2-way; no element stride serves both them and the y-lines.)  Otherwise x-lines are padded by
  // one slot (RS = n + 1).
  // DENSE (FP32 2D / 3D, n = 6): no padding at all -- x-lines read as float2 are conflict-free and
  // y/z lines conflict no more than with padding -- so the tile copy and the update are plain
  // 16-byte streams over contiguous memory.
  // PLANE (FP32 3D, n = 8): x-lines unpadded (32 bytes, read as float4), planes of 8 x-lines 72
  // slots apart (= 8 mod 32 banks), so a warp's y-lines (8 x by 4 z) and z-lines (8 x by 4 y)
  // hit 32 distinct banks; every plane is one contiguous 256-byte block in global and shared
  // memory.
  static constexpr bool VEC = sizeof(real) == 4 && DIM == 2 && (n == 8 || n == 4);
  static constexpr bool DENSE = sizeof(real) == 4 && DIM >= 2 && n == 6;
  static constexpr bool PLANE = sizeof(real) == 4 && DIM == 3 && n == 8;
  static constexpr bool QUAD = VEC || DENSE || PLANE;  // copy and update in 16-byte units
  // BULK (with DENSE and PLANE): the tile is copied by bulk (TMA) copies: DENSE, one per variable
  // (the tile of a variable is one contiguous block in global and shared memory: elements of 6^3
  // FP32 values, 864 bytes, a multiple of 16); PLANE, one per 256-byte plane
  static constexpr bool BULK = DENSE || PLANE;
  static constexpr int XW = (VEC || PLANE) ? 4 : (DENSE ? 2 : 1);  // x-line access width (floats)
  static constexpr int RS = VEC ? (n == 8 ? 12 : 4) : ((DENSE || PLANE) ? n : n + 1);
  static constexpr int PS = PLANE ? n * n + 8 : RS * n;  // plane stride (3D)
  static constexpr int SPE = VEC ? (n == 8 ? 104 : 20) : (PLANE ? n * PS : RS * L);  // shared slots per element
  // FP64 (arithmetic-bound) stages U^n and ACC in shared memory and keeps the Euler velocities
  // there; FP32 (memory-bound) keeps shared memory small for occupancy: U^n / ACC are
  // prefetched into L2 and read directly, velocities are recomputed per line.
  static constexpr bool SLIM = sizeof(real) == 4;
  // EARLY (stage_body): neighbour-trace loads issued with the tile copy and a batched stage
  // update (more loads in flight); it costs registers, and pays only for 1D/2D (measured: 3D and
  // float-float lose occupancy), so 3D and float-float load each axis's traces in its pass (and
  // the FP64 / float-float update there goes one node at a time; FP32 3D moves quads).
  static constexpr int NS = (EQ == 0 || SLIM) ? 2 * NV : 2 * NV + DIM;  // shared arrays of SPE per element
  // GOPS: the update reads U^n / ACC from global memory (after an L2 prefetch issued with the
  // tile) instead of copies staged in shared memory.  FP32 always; FP64 in 3D at degree 7 with one
  // thread per line, where the staged copies take 32 of an Euler element's 84 KB of shared memory
  // and with them half the CTAs an SM holds (measured: 32^3 FP64 5.16 -> 4.36 ms per stage; at
  // degree 5, where registers bind first, 16.07 -> 16.19, so it keeps them; also with the entry's
  // registers capped at 168 (152 used, no spills) and tiles of 2, 3, 4, 6 or 8 elements, up to
  // three CTAs per SM: 18.44, 16.55, 16.17, 16.57, 15.91 ms against 16.07 staged -- 1 % at best).  The
  // line-and-variable mapping keeps them too: the global loads cost registers its large CTAs do
  // not have.  Float-float 3D Euler at degrees 3-6 with one thread per line: with its registers
  // capped at 168 (FF3D_REGS) shared memory binds, and without the staged copies more CTAs fit an
  // SM (degree 5 at 64^3: three CTAs of three elements instead of one of six, 17.07 -> 14.91 ms
  // per stage unrolled; with the rolled variable loop, degree 3 at 96^3 11.91 -> 11.22 ms, degree
  // 4 at 72^3 12.37 -> 10.29 ms, degree 6 at 40^3 5.87 -> 4.87 ms).  At degrees 2 (14.19 ->
  // 14.80 ms at 128^3) and 7 (3.76 -> 3.96 ms) and in 2D the same changes measured slower.
  static constexpr bool FF3D = FF && DIM == 3 && EQ == 1 && N >= 3 && N <= 6 && !VS;
  static constexpr bool GOPS = SLIM || (DIM == 3 && !VS && N == 7) || FF3D;
  static constexpr int NB = GOPS ? 0 : 2 * NV;  // unpadded shared arrays of NPE per element: U^n and ACC
  // threads per element: one per line, or (VS) one per line and variable
  static constexpr int TPE = VS ? L * NV : L;
  __device__ static __forceinline__ int pad(int node) {
    if constexpr (PLANE) return node + (PS - n * n) * (node / (n * n));
    return (node / n) * RS + node % n;
  }
  // shared slot of the first of four consecutive nodes (QUAD: quad q of the tile)
  __device__ static __forceinline__ int quad_slot(int q) {
    if constexpr (DENSE) return 4 * q;
    if constexpr (PLANE) {
      const int el = q / (NPE / 4);
      return el * SPE + pad(4 * (q - el * (NPE / 4)));
    }
    const int el = q / (NPE / 4), node = 4 * (q - el * (NPE / 4));
    return el * SPE + (node / n) * RS + node % n;
  }
};

// VS = false: a thread owns a line for every variable (fewest FP64 operations: the wave speeds
// of the face flux are computed once per line).  VS = true: a thread owns one (line, variable)
// pair, so an Euler CTA has nvar times more threads for the same shared memory; the operations
// per variable are the same, in the same order, so the results are bitwise identical.
// EXACT: the exact-mass variant (face terms lifted by M^-1 e_0 / M^-1 e_N onto every node).
template <int DIM, int N, int EQ, typename real, bool VS, bool FF = false, bool EXACT = false>
__device__ __forceinline__ void stage_body(const StageArgs<real>& args) {
  using G = StageGeom<DIM, N, EQ, real, VS, FF>;
  constexpr int n = G::n, L = G::L, NPE = G::NPE, NV = G::NV, SPE = G::SPE, TPE = G::TPE;
  // float-float 2D Euler at degrees 6-7 (its variable loop rolled, see ROLLV): EARLY and FUSED
  // below pay there too (512^2 degree 7 2.13 -> 1.89 ms per stage, 420^2 degree 6 1.11 -> 1.05;
  // EARLY alone 2.07 / 1.15, FUSED alone 2.13 / 1.11)
  constexpr bool FF2E = FF && DIM == 2 && EQ == 1 && N >= 6 && !VS;
  constexpr bool EARLY = DIM <= 2 && (!FF || FF2E);
  // BPF (FP32, elements a multiple of 16 bytes; Euler or the bulk-copy layouts): the update's
  // U^n / ACC reach L2 by bulk prefetches (16-byte aligned ranges: the arrays are 256-byte
  // aligned).  Measured on the 16-byte 2D layouts: Euler degree 7 170 -> 167 us, advection
  // degree 3 19.6 -> 20.8 us, so advection there keeps the per-line prefetches.
  constexpr bool BPF = G::GOPS && (NPE * sizeof(real)) % 16 == 0 && (G::BULK || EQ == 1 || !G::SLIM);
  // 2D FP64: the y-line threads own whole lines of finished right-hand side and apply the stage
  // update to them directly (no shared round trip, one barrier less: 2D Euler 2.40 -> 2.28 ms per
  // stage).  Elsewhere the extra registers cost more occupancy than the round trip does (measured:
  // FP32 2D Euler 243 -> 260 us, float-float 93 -> 95 us, FP64 3D Euler no gain), so those keep the
  // node-parallel update.
  constexpr bool FUSED = DIM == 2 && !G::SLIM && (!FF || FF2E);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GroupHeader hdr = *args.hdr;
  const int epb = hdr.epb;
  real* const sU = reinterpret_cast<real*>(smem_raw);  // [NV][epb][SPE]: the stage-input tile
  real* sR = sU + NV * epb * SPE;                       // [NV][epb][SPE]
  real* sV = sR + NV * epb * SPE;                       // [DIM][epb][SPE] (Euler)
  real* sB = sU + G::NS * epb * SPE;                    // [NV][epb][NPE]: U^n of the tile (stage update)
  real* sA = sB + NV * epb * NPE;                       // [NV][epb][NPE]: ACC of the tile
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const StagePlan& plan = args.plan;
  // BULK: the mbarrier of the tile copies, after the arrays (16-byte aligned)
  unsigned long long* const mbar = reinterpret_cast<unsigned long long*>(
      smem_raw + (((size_t)G::NS * SPE + (size_t)G::NB * NPE) * epb * sizeof(real) + 15) / 16 * 16);
  const int polls = hdr.wait_polls > 0 ? hdr.wait_polls : kBulkWaitPolls;
  if constexpr (G::BULK) {
    if (tid == 0) mbar_init(mbar);
    __syncthreads();
  }
  unsigned bulk_phase = 0;

  SolveRegs<DIM, real> S;
  for (int tile = blockIdx.x; tile < hdr.ntiles; tile += gridDim.x) {
    // ---- which solve owns this tile; its fields stay in registers while it does not change ----
    const int si = hdr.nsolves > 1 ? find_solve(args.solves, hdr.nsolves, tile) : 0;
    if (si != S.index) S.load(args.solves + si, si, plan);
    const long long nelem = S.nelem;
    const long long e0 = (long long)(tile - S.tile_begin) * epb;
    const int cnt = (int)min((long long)epb, nelem - e0);
    const long long vstride = nelem * NPE;  // elements of one variable
    const real* __restrict__ uin = S.uin;

    // ---- 1. the tile of the stage input, and U^n / ACC when the update reads them, copied into
    //         shared memory asynchronously: every copy of the tile is in flight before the wait ----
    const bool need_un = plan.in != kUN && plan.acc_mode != 3;
    const bool need_acc = plan.acc_mode >= 2;
    {
      const int total = cnt * NPE;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const real* src = uin + v * vstride + e0 * NPE;
        real* dst = sU + v * epb * SPE;
        if constexpr (G::VEC) {
          // 16-byte copies: chunk q = 4 consecutive nodes of one x-line
          constexpr int C = n / 4;
          for (int q = tid; q < total / 4; q += nthr) {
            const int row = q / C, c = q - row * C;
            const int el = row / L, r = row - el * L;
            cp_async_16(dst + el * SPE + r * G::RS + 4 * c, src + 4 * q);
          }
        } else if constexpr (G::BULK) {
          // one bulk copy per variable, issued by thread 0 below
        } else if constexpr (G::DENSE) {
          for (int q = tid; q < total / 4; q += nthr) cp_async_16(dst + 4 * q, src + 4 * q);
        } else {
          for (int idx = tid; idx < total; idx += nthr) {
            const int el = idx / NPE, node = idx - el * NPE;
            cp_async_elem(dst + el * SPE + G::pad(node), src + idx);
          }
        }
        if constexpr (G::GOPS) {
          // start the update's reads now: one L2 prefetch per 128-byte line of U^n / ACC (BPF:
          // one bulk prefetch per array, below)
          if constexpr (!BPF) {
            constexpr int per_line = 128 / (int)sizeof(real);
            for (int idx = tid * per_line; idx < total; idx += nthr * per_line) {
              if (need_un) asm volatile("prefetch.global.L2 [%0];" ::"l"(S.un + v * vstride + e0 * NPE + idx));
              if (need_acc) asm volatile("prefetch.global.L2 [%0];" ::"l"(S.acc + v * vstride + e0 * NPE + idx));
            }
          }
          continue;
        }
        if (need_un) {
          const real* s2 = S.un + v * vstride + e0 * NPE;
          real* d2 = sB + v * epb * NPE;
          for (int idx = tid; idx < total; idx += nthr) cp_async_elem(d2 + idx, s2 + idx);
        }
        if (need_acc) {
          const real* s3 = S.acc + v * vstride + e0 * NPE;
          real* d3 = sA + v * epb * NPE;
          for (int idx = tid; idx < total; idx += nthr) cp_async_elem(d3 + idx, s3 + idx);
        }
      }
    }
    // this tile's U^n / ACC (read by the update) into L2 by the copy engine: one instruction per
    // array instead of one prefetch per 128-byte line and thread (measured: FP32 2D Euler degree
    // 5 244 -> 213 us, 3D Euler degree 7 / 5 270 -> 262 / 1037 -> 999 us; prefetching the stage
    // input of the CTA's next tile as well made 3D slower).  Issued after the tile's own copies.
    auto prefetch_update_operands = [&]() {
      const unsigned bytes = (unsigned)(cnt * NPE * sizeof(real));
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if (need_un) bulk_prefetch_l2(S.un + v * vstride + e0 * NPE, bytes);
        if (need_acc) bulk_prefetch_l2(S.acc + v * vstride + e0 * NPE, bytes);
      }
    };
    if constexpr (BPF && !G::BULK) {
      if (tid == 0) prefetch_update_operands();
    }
    // ---- 1b. neighbour traces outside the tile: their global / halo loads are issued now, so
    //         they are in flight together with the tile's copies ----
    const int el_t = tid / TPE;
    const int line_t = (tid - el_t * TPE) % L;
    real xr_lo[DIM][NV], xr_hi[DIM][NV];  // loaded traces (variables of this line's faces)
    int xs_lo[DIM], xs_hi[DIM];           // shared-memory offset of an in-tile trace, else -1
    if constexpr (EARLY) {
     if (el_t < cnt) {
      const unsigned eu = (unsigned)(e0 + el_t);
      const ElemXYZ exyz = elem_xyz(eu, S.E0, S.E1);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        xs_lo[a] = xs_hi[a] = -1;
        int pbase, pstride, ubase, ustride;
        line_geometry<n, G::RS, G::PS>(a, line_t, pbase, pstride, ubase, ustride);
        const LineTrace t = line_trace<L>(a, eu, exyz, line_t, S.E0, S.E1, S.E2, S.halo_lo[a] != nullptr,
                                          S.halo_hi[a] != nullptr);
        // advection: no flux along a zero-velocity axis, and upwinding zeroes one face
        const bool need_lo = EQ == 1 || (S.vs[a] != real(0) && S.qlo[a] != real(0));
        const bool need_hi = EQ == 1 || (S.vs[a] != real(0) && S.qhi[a] != real(0));
        if (!(G::VEC && n == 8) && S.halo_lo[a] == nullptr && S.halo_hi[a] == nullptr) {
          // no partition halo on this axis: the traces from global memory, in the tile or not
          // (fewer instructions than choosing per line; measured: FP32 2D Euler degree 3 / 5
          // 217 -> 198 / 274 -> 244 us, FP64 2D advection 151 -> 149 us; the 16-byte FP32
          // layout at degree 7 keeps the in-tile reads, which hold fewer registers there)
          const real* plo = uin + t.elo * NPE + ubase + N * ustride;
          const real* phi = uin + t.ehi * NPE + ubase;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            if (need_lo) xr_lo[a][v] = plo[v * vstride];
            if (need_hi) xr_hi[a][v] = phi[v * vstride];
          }
          continue;
        }
        if (need_lo) {
          if (t.lo_halo) {
#pragma unroll
            for (int v = 0; v < NV; ++v) xr_lo[a][v] = S.halo_lo[a][v * t.hvs + t.hoff];
          } else if (t.elo >= e0 && t.elo < e0 + cnt) {
            xs_lo[a] = (int)(t.elo - e0) * SPE + pbase + N * pstride;
          } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) xr_lo[a][v] = uin[v * vstride + t.elo * NPE + ubase + N * ustride];
          }
        }
        if (need_hi) {
          if (t.hi_halo) {
#pragma unroll
            for (int v = 0; v < NV; ++v) xr_hi[a][v] = S.halo_hi[a][v * t.hvs + t.hoff];
          } else if (t.ehi >= e0 && t.ehi < e0 + cnt) {
            xs_hi[a] = (int)(t.ehi - e0) * SPE + pbase;
          } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) xr_hi[a][v] = uin[v * vstride + t.ehi * NPE + ubase];
          }
        }
      }
     }
    }
    if constexpr (G::BULK) {
      if (tid < 32) {
        // order this CTA's earlier generic accesses to sU before the asynchronous writes
        fence_proxy_async_smem();
        const unsigned bytes = (unsigned)(cnt * NPE * sizeof(real));  // 864 / 2048-byte elements
        if (tid == 0) mbar_expect_tx(mbar, bytes * NV);
        if (!hdr.stall_copies) {
          if constexpr (G::PLANE) {
            // one copy per plane, spread over the first warp (after the expected byte count is set)
            __syncwarp();
            constexpr unsigned kPlane = n * n * sizeof(real);
            const int planes = cnt * n;
            for (int k = tid; k < NV * planes; k += 32) {
              const int v = k / planes, pl = k - v * planes;
              const int el = pl / n, z = pl - el * n;
              bulk_copy(sU + (v * epb + el) * SPE + z * G::PS, uin + v * vstride + e0 * NPE + pl * (n * n), kPlane,
                        mbar);
            }
          } else if (tid == 0) {
#pragma unroll
            for (int v = 0; v < NV; ++v) bulk_copy(sU + v * epb * SPE, uin + v * vstride + e0 * NPE, bytes, mbar);
          }
        }
        if constexpr (BPF) {
          if (tid == 0) prefetch_update_operands();
        }
      }
      const bool ok = mbar_wait(mbar, bulk_phase, polls);
      if (!__syncthreads_and(ok)) {
        // the copies did not land in time: flag the launch for the host, give the copies in
        // flight one more bounded wait, and leave
        if (tid == 0) flag_failure(args);
        mbar_wait(mbar, bulk_phase, polls);
        return;
      }
      bulk_phase ^= 1u;
    }
    if constexpr (!G::BULK) {  // (BULK: the vote on the wait above was the barrier)
      cp_async_wait_all();
      __syncthreads();
    }
    // ---- 2. velocities (Euler; the FP32 kernel recomputes them per line instead) ----
    if constexpr (EQ == 1 && !G::SLIM) {
      const int total = cnt * NPE;
      for (int idx = tid; idx < total; idx += nthr) {
        const int el = idx / NPE, node = idx - el * NPE;
        const int s = el * SPE + G::pad(node);
        const real inv = real(1) / sU[s];
#pragma unroll
        for (int a = 0; a < DIM; ++a) sV[a * epb * SPE + s] = sU[(1 + a) * epb * SPE + s] * inv;
      }
      __syncthreads();
    }
    // ---- 3. volume + surface terms, axis by axis (FUSED: the last axis applies the stage update
    //         to the finished right-hand side of its line directly) ----
    const ElemXYZ exyz_t = elem_xyz((unsigned)(e0 + el_t), S.E0, S.E1);  // this thread's element
    // Float-float Euler with one thread per line: the variable loop stays a loop (unrolled, its
    // four float-float contractions made a body that missed the instruction cache).  Measured per
    // RK4 stage, unrolled -> rolled (plain FP64 beside): 3D degree 3 at 96^3 12.95 -> 11.94 ms
    // (14.02), degree 4 at 72^3 14.90 -> 12.38 (13.61), degree 5 at 64^3 14.91 -> 12.59 (16.10),
    // degree 6 at 40^3 7.27 -> 5.88 (6.90), degree 7 at 32^3 4.53 -> 3.74 (4.33); 2D degree 6 at
    // 420^2 1.20 -> 1.11 (1.24), degree 7 at 512^2 2.42 -> 2.10 (2.28); 2D degrees 4 and 5 alike
    // or slower rolled, so they stay unrolled, as does the plain FP64 kernel (3D degree 5: 16.10 ->
    // 16.77 rolled).  The operations and their order are the same.
    constexpr bool ROLLV = FF && EQ == 1 && !VS && ((DIM == 3 && N >= 3) || (DIM == 2 && N >= 6));
    // the variable loop's trip count, hidden from the compiler where the loop stays rolled (a
    // bare unroll pragma unrolls only loops of known trip count; a count on the pragma changed
    // the code, and the registers, of the other kernels too)
    int nv_loop = NV;
    if constexpr (ROLLV) asm volatile("" : "+r"(nv_loop));
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const bool last = FUSED && a == DIM - 1;
      const bool VX = G::XW > 1 && a == 0;  // x-lines contiguous and aligned: float2 / float4 access
      const int el = tid / TPE;
      const int rem = tid - el * TPE;
      const int line = rem % L;
      const int vsel = rem / L;  // the variable this thread owns (VS), else 0
      if (el < cnt) {
        int pbase, pstride, ubase, ustride;
        line_geometry<n, G::RS, G::PS>(a, line, pbase, pstride, ubase, ustride);
        const real* sUe = sU + el * SPE + pbase;
        real* sRe = sR + el * SPE + pbase;
        const real vs = S.vs[a];
        const real qlo = S.qlo[a];
        const real qhi = S.qhi[a];
        // operands of the fused update of variable v's nodes on this line: U^n and ACC where the
        // plan reads them (loaded once the line's right-hand side is done: loaded earlier, they
        // would hold registers through the contraction)
        const long long gline = (e0 + el) * NPE + ubase;  // global node index of l = 0 (variable 0)
        const int bline = el * NPE + ubase;               // the same in the staged U^n / ACC tiles
        auto operands = [&](int v, real (&bb)[n], real (&aa)[n]) {
          const long long g0 = v * vstride + gline;
#pragma unroll
          for (int l = 0; l < n; ++l) {
            if (plan.acc_mode != 3)
              bb[l] = plan.in == kUN ? sUe[v * epb * SPE + l * pstride]
                                     : (G::GOPS ? S.un[g0 + l * ustride] : sB[v * epb * NPE + bline + l * ustride]);
            if (plan.acc_mode >= 2) aa[l] = G::GOPS ? S.acc[g0 + l * ustride] : sA[v * epb * NPE + bline + l * ustride];
          }
        };
        // The right-hand side is kept divided by axis 0's scale (rhs_scale), so axis 0 needs no
        // multiply; a zero scale means advection with no velocity along this axis: no flux.
        if constexpr (EQ == 0) {
          real bb[n], aa[n];
          if (vs == real(0)) {
            // no flux along this axis: the right-hand side is what the other axes left
            if (last) {
              operands(0, bb, aa);
#pragma unroll
              for (int l = 0; l < n; ++l)
                stage_update_node(args, S, si, plan, gline + l * ustride, a == 0 ? real(0) : sRe[l * pstride], bb[l], aa[l]);
            } else if (a == 0) {
#pragma unroll
              for (int l = 0; l < n; ++l) sRe[l * pstride] = real(0);
            }
          } else {
            // upwinding makes one of the two face terms vanish: its trace was not even loaded
            const bool has_lo = qlo != real(0), has_hi = qhi != real(0);
            real xlo = 0, xhi = 0;
            if constexpr (EARLY) {
              if (has_lo) xlo = xs_lo[a] >= 0 ? sU[xs_lo[a]] : xr_lo[a][0];
              if (has_hi) xhi = xs_hi[a] >= 0 ? sU[xs_hi[a]] : xr_hi[a][0];
            } else if (S.halo_lo[a] == nullptr && S.halo_hi[a] == nullptr) {
              // no partition halo on this axis: both traces from global memory (the stage input
              // is read-only during the stage), whether or not the neighbour is in the tile
              const LineTrace t = line_trace<L>(a, (unsigned)(e0 + el), exyz_t, line, S.E0, S.E1, S.E2, false, false);
              if (has_lo) xlo = uin[t.elo * NPE + ubase + N * ustride];
              if (has_hi) xhi = uin[t.ehi * NPE + ubase];
            } else {
              const LineTrace t = line_trace<L>(a, (unsigned)(e0 + el), exyz_t, line, S.E0, S.E1, S.E2,
                                                S.halo_lo[a] != nullptr, S.halo_hi[a] != nullptr);
              if (has_lo)
                xlo = t.lo_halo ? S.halo_lo[a][t.hoff]
                                : (t.elo >= e0 && t.elo < e0 + cnt ? sU[(int)(t.elo - e0) * SPE + pbase + N * pstride]
                                                                   : uin[t.elo * NPE + ubase + N * ustride]);
              if (has_hi)
                xhi = t.hi_halo ? S.halo_hi[a][t.hoff]
                                : (t.ehi >= e0 && t.ehi < e0 + cnt ? sU[(int)(t.ehi - e0) * SPE + pbase]
                                                                   : uin[t.ehi * NPE + ubase]);
            }
            real f[n], out[n], rr[n];
            load_line<n, G::XW>(sUe, pstride, VX, f);
            contract_line<N, real, FF>(f, out, args);
            if (last) operands(0, bb, aa);
            const real flo = xlo - f[0], fhi = f[N] - xhi;
#pragma unroll
            for (int l = 0; l < n; ++l) {
              real r = (a == 0) ? out[l] : fma(vs, out[l], sRe[l * pstride]);
              if constexpr (!EXACT) {
                if (l == 0 && has_lo) r = fma(qlo, flo, r);
                if (l == N && has_hi) r = fma(qhi, fhi, r);
              } else {
                if (has_lo) r = fma(qlo * args.basis.Llo[l], flo, r);
                if (has_hi) r = fma(qhi * args.basis.Lhi[l], fhi, r);
              }
              if (last) stage_update_node(args, S, si, plan, gline + l * ustride, r, bb[l], aa[l]);
              else rr[l] = r;
            }
            if (!last) store_line<n, G::XW>(sRe, pstride, VX, rr);
          }
        } else {
          // exterior traces: node N of the low neighbour, node 0 of the high neighbour
          real xlo[NV], xhi[NV];
          if constexpr (EARLY) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              xlo[v] = xs_lo[a] >= 0 ? sU[v * epb * SPE + xs_lo[a]] : xr_lo[a][v];
              xhi[v] = xs_hi[a] >= 0 ? sU[v * epb * SPE + xs_hi[a]] : xr_hi[a][v];
            }
          } else if (S.halo_lo[a] == nullptr && S.halo_hi[a] == nullptr) {
            // no partition halo on this axis: every trace from global memory (the stage input is
            // read-only during the stage), whether or not the neighbour is in the tile
            const LineTrace t = line_trace<L>(a, (unsigned)(e0 + el), exyz_t, line, S.E0, S.E1, S.E2, false, false);
            const real* plo = uin + t.elo * NPE + ubase + N * ustride;
            const real* phi = uin + t.ehi * NPE + ubase;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              xlo[v] = plo[v * vstride];
              xhi[v] = phi[v * vstride];
            }
          } else {
            const LineTrace t = line_trace<L>(a, (unsigned)(e0 + el), exyz_t, line, S.E0, S.E1, S.E2,
                                              S.halo_lo[a] != nullptr, S.halo_hi[a] != nullptr);
            const bool lo_in = !t.lo_halo && t.elo >= e0 && t.elo < e0 + cnt;
            const bool hi_in = !t.hi_halo && t.ehi >= e0 && t.ehi < e0 + cnt;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              xlo[v] = t.lo_halo ? S.halo_lo[a][v * t.hvs + t.hoff]
                                 : (lo_in ? sU[(v * epb + (int)(t.elo - e0)) * SPE + pbase + N * pstride]
                                          : uin[v * vstride + t.elo * NPE + ubase + N * ustride]);
              xhi[v] = t.hi_halo ? S.halo_hi[a][v * t.hvs + t.hoff]
                                 : (hi_in ? sU[(v * epb + (int)(t.ehi - e0)) * SPE + pbase]
                                          : uin[v * vstride + t.ehi * NPE + ubase]);
            }
          }
          const real c2 = S.c2;
          const real cs = S.c;
          // velocity u_a along the line: from shared memory (FP64) or recomputed (FP32)
          real ua[n];
          real rho[n], ma[n];  // FP32: the density and m_a lines, kept for the fluxes below
          if constexpr (G::SLIM) {
            load_line<n, G::XW>(sUe, pstride, VX, rho);
            load_line<n, G::XW>(sUe + (1 + a) * epb * SPE, pstride, VX, ma);
#pragma unroll
            for (int l = 0; l < n; ++l) ua[l] = ratio(ma[l], rho[l]);
          } else {
            const real* sVa = sV + a * epb * SPE + el * SPE + pbase;
#pragma unroll
            for (int l = 0; l < n; ++l) ua[l] = sVa[l * pstride];
          }
          // normal velocities and LLF alpha at both faces of the line
          const real un0 = ua[0], unN = ua[N];
          const real unlo = ratio(xlo[1 + a], xlo[0]);
          const real unhi = ratio(xhi[1 + a], xhi[0]);
          const real alo = fmax(fabs(unlo), fabs(un0)) + cs;
          const real ahi = fmax(fabs(unN), fabs(unhi)) + cs;
#pragma unroll
          for (int v = 0; v < nv_loop; ++v) {
            if (VS && v != vsel) continue;
            const real* sUv = sUe + v * epb * SPE;
            real bb[n], aa[n];
            real f[n], out[n], rr[n];
            real u0, uN;
            // flux component v along a (Eq. (eulerIso2d)): v = 0: m_a; v = 1 + b: m_b u_a
            // plus c^2 rho when b = a
            if constexpr (G::SLIM) {
              if (v == 0) {
#pragma unroll
                for (int l = 0; l < n; ++l) f[l] = ma[l];
                u0 = rho[0], uN = rho[N];
              } else if (v == 1 + a) {
#pragma unroll
                for (int l = 0; l < n; ++l) f[l] = fma(ma[l], ua[l], c2 * rho[l]);
                u0 = ma[0], uN = ma[N];
              } else {
                real mb[n];
                load_line<n, G::XW>(sUv, pstride, VX, mb);
#pragma unroll
                for (int l = 0; l < n; ++l) f[l] = mul_rn(mb[l], ua[l]);
                u0 = mb[0], uN = mb[N];
              }
            } else if (v == 0) {
              const real* sm = sUe + (1 + a) * epb * SPE;
#pragma unroll
              for (int l = 0; l < n; ++l) f[l] = sm[l * pstride];
            } else if (v == 1 + a) {
#pragma unroll
              for (int l = 0; l < n; ++l) f[l] = fma(sUv[l * pstride], ua[l], c2 * sUe[l * pstride]);
            } else {
#pragma unroll
              for (int l = 0; l < n; ++l) f[l] = mul_rn(sUv[l * pstride], ua[l]);
            }
            contract_line<N, real, FF>(f, out, args);
            real fxlo, fxhi;
            if (v == 0) {
              fxlo = xlo[1 + a];
              fxhi = xhi[1 + a];
            } else if (v == 1 + a) {
              fxlo = fma(xlo[v], unlo, c2 * xlo[0]);
              fxhi = fma(xhi[v], unhi, c2 * xhi[0]);
            } else {
              fxlo = mul_rn(xlo[v], unlo);
              fxhi = mul_rn(xhi[v], unhi);
            }
            if constexpr (!G::SLIM) u0 = sUv[0], uN = sUv[N * pstride];
            real* sRv = sRe + v * epb * SPE;
            if (last) operands(v, bb, aa);
            const long long gv = v * vstride + gline;
            // (Fhat_lo - F(U_0)) = 1/2 (F(ext) - F(U_0) - alpha (U_0 - ext)); qlo carries the 1/2
            const real flo = fma(-alo, u0 - xlo[v], fxlo - f[0]);
            // (F(U_N) - Fhat_hi) = 1/2 (F(U_N) - F(ext) + alpha (ext - U_N))
            const real fhi = fma(ahi, xhi[v] - uN, f[N] - fxhi);
#pragma unroll
            for (int l = 0; l < n; ++l) {
              real r = (a == 0) ? out[l] : fma(vs, out[l], sRv[l * pstride]);
              if constexpr (!EXACT) {
                if (l == 0) r = fma(qlo, flo, r);
                if (l == N) r = fma(qhi, fhi, r);
              } else {
                r = fma(qlo * args.basis.Llo[l], flo, r);
                r = fma(qhi * args.basis.Lhi[l], fhi, r);
              }
              if (last) stage_update_node(args, S, si, plan, gv + l * ustride, r, bb[l], aa[l]);
              else rr[l] = r;
            }
            if (!last) store_line<n, G::XW>(sRv, pstride, VX, rr);
          }
        }
      }
      if (!last) __syncthreads();
    }
    // ---- 4. Runge-Kutta stage update, node-parallel (unless fused into the last axis) ----
    if constexpr (G::QUAD) {
      // four consecutive nodes of one x-line per step: float4 shared reads and global accesses
      // (every state array is 256-byte aligned: the allocation paths check)
      const int quads = cnt * NPE / 4;
      if constexpr (DIM == 3) {
        // quads outside, variables inside: a quad's slot and offset serve every variable
        for (int q = tid; q < quads; q += nthr) {
          const int sl = G::quad_slot(q);
          const long long g = e0 * NPE + 4 * q;
#pragma unroll
          for (int v = 0; v < NV; ++v)
            stage_update_quad(args, S, si, plan, v * vstride + g, sR + v * epb * SPE + sl, sU + v * epb * SPE + sl);
        }
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const real* sRv = sR + v * epb * SPE;
          const real* sUv = sU + v * epb * SPE;
          const long long goff = v * vstride + e0 * NPE;
          for (int q = tid; q < quads; q += nthr) {
            const int sl = G::quad_slot(q);
            stage_update_quad(args, S, si, plan, goff + 4 * q, sRv + sl, sUv + sl);
          }
        }
      }
    } else if constexpr (!FUSED) {
      const int total = cnt * NPE;
      // each thread owns up to B nodes per variable: all of their operands are loaded first, so
      // the loads are in flight together, then the results are computed and stored
      constexpr int B = EARLY ? 8 : (G::GOPS ? 2 : 1);  // (GOPS FP64: 4 cost registers, no time)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const real* sRv = sR + v * epb * SPE;
        const real* sUv = sU + v * epb * SPE;
        const real* sBv = sB + v * epb * NPE;
        const real* sAv = sA + v * epb * NPE;
        const long long goff = v * vstride + e0 * NPE;
        for (int i0 = tid; i0 < total; i0 += nthr * B) {
          real rr[B], bb[B], aa[B];
#pragma unroll
          for (int k = 0; k < B; ++k) {
            const int idx = i0 + k * nthr;
            if (idx >= total) break;
            const int el = idx / NPE, node = idx - el * NPE;
            const int s = el * SPE + G::pad(node);
            const long long g = goff + idx;
            rr[k] = sRv[s];
            if (plan.acc_mode >= 2) aa[k] = G::GOPS ? S.acc[g] : sAv[idx];
            if (plan.acc_mode != 3) bb[k] = plan.in == kUN ? sUv[s] : (G::GOPS ? S.un[g] : sBv[idx]);
          }
#pragma unroll
          for (int k = 0; k < B; ++k) {
            const int idx = i0 + k * nthr;
            if (idx >= total) break;
            stage_update_node(args, S, si, plan, goff + idx, rr[k], bb[k], aa[k]);
          }
        }
      }
    }
    __syncthreads();
  }
}

template <int DIM, int N, int EQ, typename real, bool VS, bool FF = false, bool EXACT = false>
__global__ void stage_kernel(const StageArgs<real> args) {
  stage_body<DIM, N, EQ, real, VS, FF, EXACT>(args);
}
// The same with the register budget capped at 96 per thread (no spills), used for FP32 3D: one CTA
// per SM more than the compiler's own choice of 106 allows (FP32 3D Euler 1.34 -> 1.24 ms per
// stage).  A cap on the other classes would not be neutral: it changes the compiler's allocation.
}  // namespace ndg

#include "stage_euler3d_f32.cuh"

namespace ndg {

// The classes served by euler3d_f32_body: FP32 isothermal Euler in 3D at degrees 5 and 7, one
// thread per line, lumped mass (the line-and-variable mapping and the exact-mass variant stay on
// stage_body).
template <int DIM, int N, int EQ, typename real, bool VS, bool FF, bool EXACT>
constexpr bool use_euler3d_f32() {
  return DIM == 3 && sizeof(real) == 4 && EQ == 1 && (N == 5 || N == 7) && !VS && !FF && !EXACT;
}

template <int DIM, int N, int EQ, typename real, bool VS, bool FF = false, bool EXACT = false>
__global__ void __maxnreg__(96) stage_kernel_r96(const StageArgs<real> args) {
  if constexpr (use_euler3d_f32<DIM, N, EQ, real, VS, FF, EXACT>()) euler3d_f32_body<N>(args);
  else stage_body<DIM, N, EQ, real, VS, FF, EXACT>(args);
}
// Float-float 3D Euler, degrees 3-6, one thread per line (StageGeom::FF3D): registers capped at
// 168 (uncapped the compiler takes 208-240; at degree 5 caps of 136-168 measured alike, below 152
// with spills).
constexpr int FF3D_REGS = 168;
template <int DIM, int N, int EQ, typename real, bool VS, bool FF = false, bool EXACT = false>
__global__ void __maxnreg__(FF3D_REGS) stage_kernel_ff3d(const StageArgs<real> args) {
  stage_body<DIM, N, EQ, real, VS, FF, EXACT>(args);
}
// The entry point of a kernel class.
template <int DIM, int N, int EQ, typename real, bool VS, bool FF = false, bool EXACT = false>
constexpr auto stage_entry() {
  if constexpr (StageGeom<DIM, N, EQ, real, VS, FF>::FF3D && !EXACT)
    return &stage_kernel_ff3d<DIM, N, EQ, real, VS, FF, EXACT>;
  else if constexpr (DIM == 3 && sizeof(real) == 4) return &stage_kernel_r96<DIM, N, EQ, real, VS, FF, EXACT>;
  else return &stage_kernel<DIM, N, EQ, real, VS, FF, EXACT>;
}

template <int DIM, int N, int EQ, typename real, bool VS, bool FF = false, bool EXACT = false>
void stage_shape(int epb, int* threads, size_t* smem) {
  using G = StageGeom<DIM, N, EQ, real, VS, FF>;
  *threads = epb * G::TPE;
  if constexpr (use_euler3d_f32<DIM, N, EQ, real, VS, FF, EXACT>()) {
    *smem = euler3d_f32_smem<N>(epb);
    return;
  }
  *smem = ((size_t)G::NS * G::SPE + (size_t)G::NB * G::NPE) * epb * sizeof(real);
  if constexpr (G::BULK) *smem = (*smem + 15) / 16 * 16 + 16;  // + the bulk copies' mbarrier
}

}  // namespace ndg
