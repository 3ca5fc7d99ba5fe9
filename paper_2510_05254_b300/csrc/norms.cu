// Norms and conserved integrals by LGL quadrature (Sec. 3.1: L2 = sqrt(int (U - U_ref)^2 dx)),
// accumulated in FP64 for both precisions: warp-shuffle reduction, then a block reduction into
// one partial per block, then a single-block pass over the partials in a fixed order
// (deterministic, no atomics).  Also the layout conversion between the element layout and the
// global node-grid layout.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/ndg.h"
#include "ndg_host.h"
#include "ndg_internal.h"

namespace ndg {

namespace {

struct NormArgs {
  const void* U;
  const void* ref;
  long long nelem;
  int n, npe, dim, nvar, equation;
  double jac;        // prod_a h_a / 2
  double w[kMaxN];   // LGL weights
  double c;          // sound speed (Euler)
  double adv_speed;  // sum_a |a_a| (advection)
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
  return x;
}

// Fields: 0 l2sq, 1 linf, 2..5 integral[v], 6 max_speed, 7 nonfinite.
template <typename real>
__global__ void __launch_bounds__(256) norms_partial(const NormArgs a, double* partials) {
  const real* U = static_cast<const real*>(a.U);
  const real* R = static_cast<const real*>(a.ref);
  const long long nodes = a.nelem * a.npe;
  double f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nodes;
       q += (long long)gridDim.x * blockDim.x) {
    const int node = (int)(q % a.npe);
    double wq = a.jac;
    int rest = node;
    for (int d = 0; d < a.dim; ++d) {
      wq *= a.w[rest % a.n];
      rest /= a.n;
    }
    double speed = 0.0;
    double rho = 1.0;
    for (int v = 0; v < a.nvar; ++v) {
      const double x = (double)U[v * nodes + q];
      const double diff = R ? x - (double)R[v * nodes + q] : x;
      if (!isfinite(x)) f[7] += 1.0;
      f[0] += wq * diff * diff;
      f[1] = fmax(f[1], fabs(diff));
      f[2 + v] += wq * x;
      if (a.equation == 1) {
        if (v == 0) rho = x;
        else speed += fabs(x / rho);
      }
    }
    if (a.equation == 1) f[6] = fmax(f[6], speed + a.dim * a.c);
  }
  __shared__ double red[8][8];  // [field][warp]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double r = (k == 1 || k == 6) ? warp_max(f[k]) : warp_sum(f[k]);
    if (lane == 0) red[k][warp] = r;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int k = threadIdx.x;
    double r = red[k][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      r = (k == 1 || k == 6) ? fmax(r, red[k][w]) : r + red[k][w];
    partials[blockIdx.x * kNormFields + k] = r;
  }
}

__global__ void __launch_bounds__(32) norms_final(const double* partials, int nblocks,
                                                  double adv_speed, int equation, double* out) {
  // one warp; lane k < 8 reduces field k over the blocks in order
  const int k = threadIdx.x;
  if (k < 8) {
    double r = partials[k];
    for (int b = 1; b < nblocks; ++b) {
      const double x = partials[b * kNormFields + k];
      r = (k == 1 || k == 6) ? fmax(r, x) : r + x;
    }
    if (k == 0) r = sqrt(r);
    if (k == 6 && equation == 0) r = adv_speed;
    out[k] = r;
  }
}

template <typename real>
__global__ void relayout_kernel(const real* __restrict__ src, real* __restrict__ dst, long long total,
                                int n, int npe, int dim, int E0, int E1, int E2, bool to_element) {
  const long long per_var = (long long)E0 * E1 * E2 * npe;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long v = q / per_var;
    const long long r = q - v * per_var;
    const long long e = r / npe;
    const int node = (int)(r - e * npe);
    const int i = node % n, j = (node / n) % n, k = node / (n * n);
    const long long ex = e % E0, ey = (e / E0) % E1, ez = e / ((long long)E0 * E1);
    const long long gx = ex * n + i;
    const long long gy = dim > 1 ? ey * n + j : 0;
    const long long gz = dim > 2 ? ez * n + k : 0;
    const long long nx = (long long)E0 * n;
    const long long ny = dim > 1 ? (long long)E1 * n : 1;
    const long long g = v * per_var + (gz * ny + gy) * nx + gx;
    if (to_element) dst[q] = src[g];
    else dst[g] = src[q];
  }
}

}  // namespace

int launch_norms(int dtype, int dim, int degree, int equation, const void* U, const void* ref,
                 long long nelem, double jac, double c, const double* velocity, int nblocks,
                 double* partials, double* result, void* stream) {
  Basis b;
  if (!build_basis(degree, &b)) return (int)cudaErrorInvalidValue;
  NormArgs a;
  a.U = U;
  a.ref = ref;
  a.nelem = nelem;
  a.n = degree + 1;
  a.dim = dim;
  a.npe = 1;
  for (int d = 0; d < dim; ++d) a.npe *= a.n;
  a.nvar = equation == 0 ? 1 : dim + 1;
  a.equation = equation;
  a.jac = jac;
  for (int i = 0; i < kMaxN; ++i) a.w[i] = i < a.n ? b.w[i] : 0.0;
  a.c = c;
  a.adv_speed = 0.0;
  for (int d = 0; d < dim; ++d) a.adv_speed += std::fabs(velocity[d]);
  cudaStream_t s = (cudaStream_t)stream;
  // an error left pending by earlier work (possibly the caller's) is reported, not cleared
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess) return (int)pending;
  if (dtype_bytes(dtype) == 8) norms_partial<double><<<nblocks, 256, 0, s>>>(a, partials);
  else norms_partial<float><<<nblocks, 256, 0, s>>>(a, partials);
  norms_final<<<1, 32, 0, s>>>(partials, nblocks, a.adv_speed, equation, result);
  return (int)cudaGetLastError();  // this call's launch error
}

int launch_relayout(int dtype, int dim, int degree, int nvar, const int* E, const void* src,
                    void* dst, bool to_element, void* stream) {
  const int n = degree + 1;
  int npe = 1;
  for (int d = 0; d < dim; ++d) npe *= n;
  const int E0 = E[0], E1 = dim > 1 ? E[1] : 1, E2 = dim > 2 ? E[2] : 1;
  const long long total = (long long)nvar * E0 * E1 * E2 * npe;
  const int threads = 256;
  long long blocks = (total + threads - 1) / threads;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype_bytes(dtype) == 8)
    relayout_kernel<double><<<(int)blocks, threads, 0, s>>>((const double*)src, (double*)dst, total,
                                                            n, npe, dim, E0, E1, E2, to_element);
  else
    relayout_kernel<float><<<(int)blocks, threads, 0, s>>>((const float*)src, (float*)dst, total, n,
                                                           npe, dim, E0, E1, E2, to_element);
  return (int)cudaGetLastError();
}

}  // namespace ndg

// ------------------------------------------------------------------------------------------
// ndg_norms_noalloc: the norms reduction with its per-block partial sums in a fixed,
// file-scope device array instead of memory allocated by a context.
// ------------------------------------------------------------------------------------------
// Largest number of reduction blocks a call may use: kNoAllocMaxBlocks * kNormFields doubles
// (80 KiB) that every GPU which loads this library keeps until the process exits.
static constexpr int kNoAllocMaxBlocks = 1024;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * ndg::kNormFields];

namespace ndg {
namespace {

// Device address of g_noalloc_partials on the current device.  In host code the symbol names a
// host-side stand-in, never the device memory itself, so the address is looked up (with the
// device current) on every call: cheap once the module is loaded, and never stale -- a cached
// address would dangle after a cudaDeviceReset reloads the module.
int noalloc_scratch(double** out) {
  double* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_partials);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static norms scratch");
  *out = p;
  return NDG_OK;
}

}  // namespace
}  // namespace ndg

extern "C" int ndg_norms_noalloc(const ndg_config* cfg, const void* U, const void* ref, int nblocks,
                                 double* out, void* stream) {
  using namespace ndg;
  if (!cfg || !U || !out) return fail(NDG_EINVAL, "cfg, U and out must not be NULL");
  int rc = check_config(*cfg);
  if (rc) return rc;
  if (nblocks == 0) nblocks = kNormBlocks;
  if (nblocks < 0 || nblocks > kNoAllocMaxBlocks)
    return fail(NDG_EINVAL, "nblocks %d is outside 1..%d, the capacity of the static scratch", nblocks,
                kNoAllocMaxBlocks);
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != cfg->device) {
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  }
  double* scratch = nullptr;
  const cudaError_t pending = cudaPeekAtLastError();
  rc = pending == cudaSuccess ? noalloc_scratch(&scratch)
                              : cuda_fail(pending, "an error of earlier work is pending (reported, not cleared)");
  if (rc == NDG_OK) {
    long long nelem = 1;
    double jac = 1.0;
    for (int a = 0; a < cfg->dim; ++a) {
      nelem *= cfg->elems[a];
      jac *= 0.5 * cfg->length[a] / cfg->elems[a];
    }
    cudaError_t e = (cudaError_t)launch_norms(cfg->dtype, cfg->dim, cfg->degree, cfg->equation, U, ref, nelem,
                                              jac, cfg->sound_speed, cfg->velocity, nblocks, scratch, out,
                                              stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "norms launch");
  }
  if (prev >= 0 && prev != cfg->device) cudaSetDevice(prev);
  return rc;
}
