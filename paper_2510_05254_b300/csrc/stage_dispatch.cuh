// Instantiation of the fused stage kernel for one (precision, dimension) pair, degrees 1..7 and
// both equations.  Each stage_<dtype>_d<dim>.cu includes this with NDG_REAL / NDG_DIM defined
// (and NDG_FF / NDG_EXACT for the float-float and exact-mass variants).
#include <cstring>
#include <mutex>
#include <type_traits>

#include "stage_kernel.cuh"

namespace ndg {

namespace {

#ifndef NDG_FF
#define NDG_FF false
#endif
#ifndef NDG_EXACT
#define NDG_EXACT false  // exact-mass variant (NDG_MASS_EXACT)
#endif

const BasisFF& basis_ff(int N) {
  static BasisFF table[kMaxDegree + 1];
  static std::once_flag once;
  std::call_once(once, [] {
    auto sp = [](double d, float& h, float& l) {
      h = (float)d;
      l = (float)(d - (double)h);
    };
    for (int d = 1; d <= kMaxDegree; ++d) {
      Basis b;
      build_basis(d, &b);
      BasisFF& t = table[d];
      std::memset(&t, 0, sizeof(t));
      const int n = d + 1, h = n / 2;
      for (int i = 0; i < h; ++i)
        for (int m = 0; m < h; ++m) {
          sp(b.Ae[i * kMaxN + m], t.Aeh[i * 4 + m], t.Ael[i * 4 + m]);
          sp(b.Bo[i * kMaxN + m], t.Boh[i * 4 + m], t.Bol[i * 4 + m]);
        }
      for (int i = 0; i < h; ++i) {
        sp(b.Cmid[i], t.Cmidh[i], t.Cmidl[i]);
        sp(b.Dmid[i], t.Dmidh[i], t.Dmidl[i]);
      }
    }
  });
  return table[N];
}

const BasisPairs& basis_pairs(int N) {
  static BasisPairs table[kMaxDegree + 1];
  static std::once_flag once;
  std::call_once(once, [] {
    for (int d = 1; d <= kMaxDegree; ++d) {
      Basis b;
      build_basis(d, &b);
      BasisPairs& t = table[d];
      std::memset(&t, 0, sizeof(t));
      const int n = d + 1, h = n / 2;
      for (int i = 0; i < h; ++i)
        for (int m = 0; m < h; ++m) {
          const float ae = (float)b.Ae[i * kMaxN + m], bo = (float)b.Bo[i * kMaxN + m];
          t.Ae[i * 4 + m] = make_float2(ae, ae);
          t.Bo[i * 4 + m] = make_float2(bo, bo);
        }
    }
  });
  return table[N];
}

template <typename real>
const BasisArgs<real>& basis_args(int N) {
  static BasisArgs<real> table[kMaxDegree + 1];
  static std::once_flag once;
  std::call_once(once, [] {
    for (int d = 1; d <= kMaxDegree; ++d) {
      Basis b;
      build_basis(d, &b);
      BasisArgs<real>& t = table[d];
      std::memset(&t, 0, sizeof(t));
      const int n = d + 1, h = n / 2;
      for (int i = 0; i < h; ++i)
        for (int m = 0; m < h; ++m) {
          t.Ae[i * 4 + m] = (real)b.Ae[i * kMaxN + m];
          t.Bo[i * 4 + m] = (real)b.Bo[i * kMaxN + m];
        }
      for (int i = 0; i < h; ++i) {
        t.Cmid[i] = (real)b.Cmid[i];
        t.Dmid[i] = (real)b.Dmid[i];
      }
      for (int l = 0; l < n; ++l) {
        t.Llo[l] = (real)b.lift_exact_lo[l];
        t.Lhi[l] = (real)b.lift_exact_hi[l];
      }
    }
  });
  return table[N];
}

// Two thread mappings of the same stage (see kLineKernel / kLineVarKernel); the tile autotuner
// picks one per kernel class.
template <int N, int EQ>
void shape_of(int variant, int epb, int* threads, size_t* smem) {
  if (variant == kLineVarKernel) stage_shape<NDG_DIM, N, EQ, NDG_REAL, true, NDG_FF, NDG_EXACT>(epb, threads, smem);
  else stage_shape<NDG_DIM, N, EQ, NDG_REAL, false, NDG_FF, NDG_EXACT>(epb, threads, smem);
}

template <int N, int EQ, bool VS>
void launch_kernel(int grid, int threads, size_t smem, void* stream, const StageArgs<NDG_REAL>& args) {
  stage_entry<NDG_DIM, N, EQ, NDG_REAL, VS, NDG_FF, NDG_EXACT>()<<<grid, threads, smem, (cudaStream_t)stream>>>(args);
}

template <int N, int EQ>
int launch_one(int variant, int grid, int epb, const SolveDesc* solves, const GroupHeader* header,
               const StagePlan& plan, void* stream) {
  StageArgs<NDG_REAL> args;
  args.solves = solves;
  args.hdr = header;
  args.plan = plan;
  args.basis = basis_args<NDG_REAL>(N);
  args.bff = basis_ff(N);
  args.bp = basis_pairs(N);
  int threads;
  size_t smem;
  shape_of<N, EQ>(variant, epb, &threads, &smem);
  // an error left by an earlier call is not this launch's: report it as such
  const cudaError_t stale = cudaGetLastError();
  if (stale != cudaSuccess) return (int)stale;
  if (variant == kLineVarKernel) launch_kernel<N, EQ, true>(grid, threads, smem, stream, args);
  else launch_kernel<N, EQ, false>(grid, threads, smem, stream, args);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFuncAttributes fa{};
    if (variant == kLineVarKernel) cudaFuncGetAttributes(&fa, stage_entry<NDG_DIM, N, EQ, NDG_REAL, true, NDG_FF, NDG_EXACT>());
    else cudaFuncGetAttributes(&fa, stage_entry<NDG_DIM, N, EQ, NDG_REAL, false, NDG_FF, NDG_EXACT>());
    launch_error_detail(grid, threads, smem, fa.maxThreadsPerBlock, fa.numRegs, fa.localSizeBytes,
                        fa.maxDynamicSharedSizeBytes);
  }
  return (int)e;
}

template <typename F>
int occupancy(F fn, int threads, size_t smem, int* max_blocks) {
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return (int)e;
  if (threads > fa.maxThreadsPerBlock) return (int)cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem);
  if (max_blocks) *max_blocks = nb;
  return (int)e;
}

template <int N, int EQ>
int prepare_one(int variant, int epb, int* max_blocks) {
  int threads;
  size_t smem;
  shape_of<N, EQ>(variant, epb, &threads, &smem);
  if (threads > 1024 || threads < 1) return (int)cudaErrorInvalidConfiguration;
  if (variant == kLineVarKernel)
    return occupancy(stage_entry<NDG_DIM, N, EQ, NDG_REAL, true, NDG_FF, NDG_EXACT>(), threads, smem, max_blocks);
  return occupancy(stage_entry<NDG_DIM, N, EQ, NDG_REAL, false, NDG_FF, NDG_EXACT>(), threads, smem, max_blocks);
}

template <int N, int EQ>
void shape_one(int variant, int epb, int* threads, size_t* smem) {
  shape_of<N, EQ>(variant, epb, threads, smem);
}

}  // namespace

#define NDG_CAT2(a, b) a##b
#define NDG_CAT(a, b) NDG_CAT2(a, b)
#define NDG_SWITCH(CALL)                                         \
  switch (degree * 2 + equation) {                               \
    case 2: return CALL<1, 0>; case 3: return CALL<1, 1>;        \
    case 4: return CALL<2, 0>; case 5: return CALL<2, 1>;        \
    case 6: return CALL<3, 0>; case 7: return CALL<3, 1>;        \
    case 8: return CALL<4, 0>; case 9: return CALL<4, 1>;        \
    case 10: return CALL<5, 0>; case 11: return CALL<5, 1>;      \
    case 12: return CALL<6, 0>; case 13: return CALL<6, 1>;      \
    case 14: return CALL<7, 0>; case 15: return CALL<7, 1>;      \
    default: break;                                              \
  }

using LaunchFn = int (*)(int, int, int, const SolveDesc*, const GroupHeader*, const StagePlan&, void*);
using PrepareFn = int (*)(int, int, int*);
using ShapeFn = void (*)(int, int, int*, size_t*);

LaunchFn NDG_CAT(NDG_TAG, _launch)(int degree, int equation) { NDG_SWITCH(&launch_one) return nullptr; }
PrepareFn NDG_CAT(NDG_TAG, _prepare)(int degree, int equation) { NDG_SWITCH(&prepare_one) return nullptr; }
ShapeFn NDG_CAT(NDG_TAG, _shape)(int degree, int equation) { NDG_SWITCH(&shape_one) return nullptr; }

}  // namespace ndg
