// The RK stage in split form, for verification: per axis a volume-term kernel (K1) and a
// surface-term kernel (K2), then the stage-update kernel (K3), each over global arrays with one
// thread per line (or node).  They apply the operations of the fused stage kernel in the same
// order -- the right-hand side of a node accumulated axis by axis, each axis's face terms added
// right after its volume term, velocities and quotients formed as the fused kernel forms them in
// each precision -- so ndg_step_split reproduces ndg_step bit for bit (lumped mass, FP64 and
// FP32).  The right-hand side lives in a state-sized global array between the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "ndg_internal.h"
#include "stage_kernel.cuh"

namespace ndg {

namespace {

template <typename real>
struct SplitArgs {
  SolveDesc sd;  // the solve (buffers, geometry, dt)
  StagePlan plan;
  BasisArgs<real> basis;
  real* R;       // right-hand side / rhs_scale, element layout
  int axis;
};

template <typename real>
__device__ __forceinline__ real coef_vol(const SolveDesc& s, int a) {
  if constexpr (sizeof(real) == 4) return s.f_vol_scale[a];
  else return s.vol_scale[a];
}
template <typename real>
__device__ __forceinline__ real coef_lo(const SolveDesc& s, int a) {
  if constexpr (sizeof(real) == 4) return s.f_lift_lo[a];
  else return s.lift_lo[a];
}
template <typename real>
__device__ __forceinline__ real coef_hi(const SolveDesc& s, int a) {
  if constexpr (sizeof(real) == 4) return s.f_lift_hi[a];
  else return s.lift_hi[a];
}

// The normal velocity of one node, as the fused kernel forms it: FP32 divides (ratio), FP64
// multiplies the momentum by the reciprocal of the density (its velocity phase).
template <typename real>
__device__ __forceinline__ real node_velocity(real m, real rho) {
  if constexpr (sizeof(real) == 4) return ratio(m, rho);
  else {
    const real inv = real(1) / rho;
    return m * inv;
  }
}

// Global offsets of one line: element e, node index ubase + l * ustride; neighbour elements
// along axis a with periodic wrap.
struct SplitLine {
  long long e, elo, ehi;
  int ubase, ustride;
};
template <int DIM, int n>
__device__ __forceinline__ SplitLine split_line(const SolveDesc& sd, int a, long long e, int line) {
  int pbase, pstride, ubase, ustride;
  line_geometry<n, n, n * n>(a, line, pbase, pstride, ubase, ustride);
  const long long E0 = sd.E[0], E1 = sd.E[1], E2 = sd.E[2];
  const long long x = e % E0, y = (e / E0) % E1, z = e / (E0 * E1);
  SplitLine s;
  s.e = e;
  s.ubase = ubase;
  s.ustride = ustride;
  if (a == 0) {
    s.elo = e - x + (x + E0 - 1) % E0;
    s.ehi = e - x + (x + 1) % E0;
  } else if (a == 1) {
    s.elo = e + (((y + E1 - 1) % E1) - y) * E0;
    s.ehi = e + (((y + 1) % E1) - y) * E0;
  } else {
    s.elo = e + (((z + E2 - 1) % E2) - z) * E0 * E1;
    s.ehi = e + (((z + 1) % E2) - z) * E0 * E1;
  }
  return s;
}

// K1: the volume term of axis a for every line and variable: R = D F (axis 0) or
// R += vs D F (later axes, one FMA), F the flux of Eq. (advection2d) / (eulerIso2d).
template <int DIM, int N, int EQ, typename real>
__global__ void split_volume(const SplitArgs<real> A) {
  constexpr int n = N + 1, L = ipow_c(n, DIM - 1), NPE = ipow_c(n, DIM), NV = EQ == 0 ? 1 : DIM + 1;
  const SolveDesc& sd = A.sd;
  const int a = A.axis;
  const long long nelem = sd.nelem, vstride = nelem * NPE;
  const real* U = static_cast<const real*>(sd.buf[A.plan.in]);
  const real vs = coef_vol<real>(sd, a);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nelem * L;
       t += (long long)gridDim.x * blockDim.x) {
    const SplitLine s = split_line<DIM, n>(sd, a, t / L, (int)(t % L));
    const long long g0 = s.e * NPE + s.ubase;
    if constexpr (EQ == 0) {
      if (vs == real(0)) {  // no flux along this axis
        if (a == 0)
          for (int l = 0; l < n; ++l) A.R[g0 + l * s.ustride] = real(0);
        continue;
      }
      real f[n], out[n];
#pragma unroll
      for (int l = 0; l < n; ++l) f[l] = U[g0 + l * s.ustride];
      contract_even_odd<N>(f, out, A.basis);
#pragma unroll
      for (int l = 0; l < n; ++l) {
        real* r = A.R + g0 + l * s.ustride;
        *r = a == 0 ? out[l] : fma(vs, out[l], *r);
      }
    } else {
      const real c2 = sizeof(real) == 4 ? (real)sd.f_c2 : (real)sd.c2;
      real rho[n], ma[n], ua[n];
#pragma unroll
      for (int l = 0; l < n; ++l) {
        rho[l] = U[g0 + l * s.ustride];
        ma[l] = U[(1 + a) * vstride + g0 + l * s.ustride];
        ua[l] = node_velocity(ma[l], rho[l]);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        real f[n], out[n];
#pragma unroll
        for (int l = 0; l < n; ++l) {
          if (v == 0) f[l] = ma[l];
          else if (v == 1 + a) f[l] = fma(ma[l], ua[l], c2 * rho[l]);
          else f[l] = mul_rn(U[v * vstride + g0 + l * s.ustride], ua[l]);
        }
        contract_even_odd<N>(f, out, A.basis);
#pragma unroll
        for (int l = 0; l < n; ++l) {
          real* r = A.R + v * vstride + g0 + l * s.ustride;
          *r = a == 0 ? out[l] : fma(vs, out[l], *r);
        }
      }
    }
  }
}

// K2: the surface term of axis a for every line and variable (Eq. (LF): upwind for advection,
// local Lax-Friedrichs for isothermal Euler), lifted onto the line's end nodes by the lumped mass.
template <int DIM, int N, int EQ, typename real>
__global__ void split_face(const SplitArgs<real> A) {
  constexpr int n = N + 1, L = ipow_c(n, DIM - 1), NPE = ipow_c(n, DIM), NV = EQ == 0 ? 1 : DIM + 1;
  const SolveDesc& sd = A.sd;
  const int a = A.axis;
  const long long nelem = sd.nelem, vstride = nelem * NPE;
  const real* U = static_cast<const real*>(sd.buf[A.plan.in]);
  const real vs = coef_vol<real>(sd, a), qlo = coef_lo<real>(sd, a), qhi = coef_hi<real>(sd, a);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nelem * L;
       t += (long long)gridDim.x * blockDim.x) {
    const SplitLine s = split_line<DIM, n>(sd, a, t / L, (int)(t % L));
    const long long g0 = s.e * NPE + s.ubase, gN = g0 + N * s.ustride;
    const long long glo = s.elo * NPE + s.ubase + N * s.ustride, ghi = s.ehi * NPE + s.ubase;
    if constexpr (EQ == 0) {
      if (vs == real(0)) continue;
      if (qlo != real(0)) A.R[g0] = fma(qlo, U[glo] - U[g0], A.R[g0]);
      if (qhi != real(0)) A.R[gN] = fma(qhi, U[gN] - U[ghi], A.R[gN]);
    } else {
      const real c2 = sizeof(real) == 4 ? (real)sd.f_c2 : (real)sd.c2;
      const real cs = sizeof(real) == 4 ? (real)sd.f_c : (real)sd.c;
      real xlo[NV], xhi[NV], u0[NV], uN[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        xlo[v] = U[v * vstride + glo];
        xhi[v] = U[v * vstride + ghi];
        u0[v] = U[v * vstride + g0];
        uN[v] = U[v * vstride + gN];
      }
      const real un0 = node_velocity(u0[1 + a], u0[0]), unN = node_velocity(uN[1 + a], uN[0]);
      const real unlo = ratio(xlo[1 + a], xlo[0]);
      const real unhi = ratio(xhi[1 + a], xhi[0]);
      const real alo = fmax(fabs(unlo), fabs(un0)) + cs;
      const real ahi = fmax(fabs(unN), fabs(unhi)) + cs;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        real f0, fN, fxlo, fxhi;  // the line's flux at its end nodes, and at the exterior traces
        if (v == 0) {
          f0 = u0[1 + a], fN = uN[1 + a];
          fxlo = xlo[1 + a], fxhi = xhi[1 + a];
        } else if (v == 1 + a) {
          f0 = fma(u0[1 + a], un0, c2 * u0[0]), fN = fma(uN[1 + a], unN, c2 * uN[0]);
          fxlo = fma(xlo[v], unlo, c2 * xlo[0]), fxhi = fma(xhi[v], unhi, c2 * xhi[0]);
        } else {
          f0 = mul_rn(u0[v], un0), fN = mul_rn(uN[v], unN);
          fxlo = mul_rn(xlo[v], unlo), fxhi = mul_rn(xhi[v], unhi);
        }
        const real flo = fma(-alo, u0[v] - xlo[v], fxlo - f0);
        const real fhi = fma(ahi, xhi[v] - uN[v], fN - fxhi);
        real* R = A.R + v * vstride;
        R[g0] = fma(qlo, flo, R[g0]);
        R[gN] = fma(qhi, fhi, R[gN]);
      }
    }
  }
}

// K3: the Runge-Kutta stage update of every node (the StagePlan of Eq. (RK3)/(RK4)/(RK6)).
template <int DIM, int N, int EQ, typename real>
__global__ void split_update(const SplitArgs<real> A) {
  constexpr int NPE = ipow_c(N + 1, DIM), NV = EQ == 0 ? 1 : DIM + 1;
  const SolveDesc& sd = A.sd;
  const StagePlan& plan = A.plan;
  const long long total = sd.nelem * NPE * NV;
  const real* uin = static_cast<const real*>(sd.buf[plan.in]);
  const real* un = static_cast<const real*>(sd.buf[kUN]);
  real* acc = static_cast<real*>(sd.buf[kACC]);
  real* uout = static_cast<real*>(sd.buf[plan.out]);
  real* kw = plan.kwrite >= 0 ? static_cast<real*>(sd.buf[plan.kwrite]) : nullptr;
  const double dt = sd.dt * sd.rhs_scale;  // the right-hand side is held divided by rhs_scale
  const real a_self = (real)(plan.a_self * dt), bdt = (real)(plan.b * dt), dts = (real)dt;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const real r = A.R[g];
    if (plan.acc_mode == 3) {
      uout[g] = fma(bdt, r, acc[g]);
      continue;
    }
    const real bb = plan.in == kUN ? uin[g] : un[g];
    real o = fma(a_self, r, bb);
    for (int j = 0; j < plan.nread; ++j) {
      const real* kj = static_cast<const real*>(sd.buf[plan.kread[j]]);
      const real aj = sizeof(real) == 4 ? (real)(plan.a_read_f[j] * (float)dts) : (real)(plan.a_read[j] * dts);
      o = fma(aj, kj[g], o);
    }
    uout[g] = o;
    if (plan.acc_mode == 1) acc[g] = fma(bdt, r, bb);
    else if (plan.acc_mode == 2) acc[g] = fma(bdt, r, acc[g]);
    if (kw) kw[g] = r;
  }
}

template <typename real>
BasisArgs<real> split_basis(int N) {
  Basis b;
  build_basis(N, &b);
  BasisArgs<real> t;
  std::memset(&t, 0, sizeof(t));
  const int n = N + 1, h = n / 2;
  for (int i = 0; i < h; ++i)
    for (int m = 0; m < h; ++m) {
      t.Ae[i * 4 + m] = (real)b.Ae[i * kMaxN + m];
      t.Bo[i * 4 + m] = (real)b.Bo[i * kMaxN + m];
    }
  for (int i = 0; i < h; ++i) {
    t.Cmid[i] = (real)b.Cmid[i];
    t.Dmid[i] = (real)b.Dmid[i];
  }
  return t;
}

template <int DIM, int N, int EQ, typename real>
int split_stage(const SolveDesc& sd, const StagePlan& plan, void* R, cudaStream_t s) {
  SplitArgs<real> A;
  A.sd = sd;
  A.plan = plan;
  A.basis = split_basis<real>(N);
  A.R = static_cast<real*>(R);
  constexpr int L = ipow_c(N + 1, DIM - 1), NPE = ipow_c(N + 1, DIM), NV = EQ == 0 ? 1 : DIM + 1;
  const int threads = 128;
  auto blocks = [&](long long work) { return (int)std::max<long long>(1, std::min<long long>((work + threads - 1) / threads, 148 * 32)); };
  for (int a = 0; a < DIM; ++a) {
    A.axis = a;
    split_volume<DIM, N, EQ, real><<<blocks(sd.nelem * L), threads, 0, s>>>(A);
    split_face<DIM, N, EQ, real><<<blocks(sd.nelem * L), threads, 0, s>>>(A);
  }
  split_update<DIM, N, EQ, real><<<blocks(sd.nelem * NPE * NV), threads, 0, s>>>(A);
  return (int)cudaGetLastError();
}

template <int DIM, typename real>
int split_dispatch(int degree, int equation, const SolveDesc& sd, const StagePlan& plan, void* R, cudaStream_t s) {
  switch (degree * 2 + equation) {
    case 2: return split_stage<DIM, 1, 0, real>(sd, plan, R, s);
    case 3: return split_stage<DIM, 1, 1, real>(sd, plan, R, s);
    case 4: return split_stage<DIM, 2, 0, real>(sd, plan, R, s);
    case 5: return split_stage<DIM, 2, 1, real>(sd, plan, R, s);
    case 6: return split_stage<DIM, 3, 0, real>(sd, plan, R, s);
    case 7: return split_stage<DIM, 3, 1, real>(sd, plan, R, s);
    case 8: return split_stage<DIM, 4, 0, real>(sd, plan, R, s);
    case 9: return split_stage<DIM, 4, 1, real>(sd, plan, R, s);
    case 10: return split_stage<DIM, 5, 0, real>(sd, plan, R, s);
    case 11: return split_stage<DIM, 5, 1, real>(sd, plan, R, s);
    case 12: return split_stage<DIM, 6, 0, real>(sd, plan, R, s);
    case 13: return split_stage<DIM, 6, 1, real>(sd, plan, R, s);
    case 14: return split_stage<DIM, 7, 0, real>(sd, plan, R, s);
    case 15: return split_stage<DIM, 7, 1, real>(sd, plan, R, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace

int launch_split_stage(const KernelClass& kc, const SolveDesc& sd, const StagePlan& plan, void* R, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (kc.dtype == 1) {
    if (kc.dim == 1) return split_dispatch<1, float>(kc.degree, kc.equation, sd, plan, R, s);
    if (kc.dim == 2) return split_dispatch<2, float>(kc.degree, kc.equation, sd, plan, R, s);
    return split_dispatch<3, float>(kc.degree, kc.equation, sd, plan, R, s);
  }
  if (kc.dim == 1) return split_dispatch<1, double>(kc.degree, kc.equation, sd, plan, R, s);
  if (kc.dim == 2) return split_dispatch<2, double>(kc.degree, kc.equation, sd, plan, R, s);
  return split_dispatch<3, double>(kc.degree, kc.equation, sd, plan, R, s);
}

}  // namespace ndg
