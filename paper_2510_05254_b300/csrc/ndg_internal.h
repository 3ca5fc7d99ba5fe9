// Internal declarations shared by the host code and the CUDA kernels of libndg.
#pragma once

#include <cstddef>
#include <cstdint>

namespace ndg {

constexpr int kMaxDegree = 7;
constexpr int kMaxN = kMaxDegree + 1;
constexpr int kMaxStages = 7;

// FP64 LGL basis of one degree (host-built, then uploaded).
struct Basis {
  int degree;
  double xi[kMaxN];
  double w[kMaxN];
  double D[kMaxN * kMaxN];   // D[i*n + m] = h_m'(xi_i), row-major with stride n = degree + 1
  double Ae[kMaxN * kMaxN];  // even-odd halves, stride kMaxN (see build_basis)
  double Bo[kMaxN * kMaxN];
  double Cmid[kMaxN];        // D[i][mid] for odd n
  double Dmid[kMaxN];        // D[mid][m] for odd n
  // exact mass matrix M (= (V V^T)^-1 for the orthonormal Legendre Vandermonde V): the lift
  // vectors w_0 M^-1 e_0 and w_N M^-1 e_N (the lumped mass gives the unit vectors e_0, e_N)
  double lift_exact_lo[kMaxN];
  double lift_exact_hi[kMaxN];
};

bool build_basis(int N, Basis* b);

// Buffer roles of one solve.  UN: the state U^n; ACC: the running sum U^n + dt sum_j b_j k_j;
// S0/S1: ping-pong stage inputs; K0..K6: stored stage slopes (RK6 only).
enum BufRole { kUN = 0, kACC = 1, kS0 = 2, kS1 = 3, kK0 = 4, kNumRoles = 11 };

// What one RK stage reads and writes, common to every solve of a launch (from the tableau).
// With L = L(U_in) the stage's right-hand side:
//   u_out = base + sum_j a_read[j] * dt * K[kread[j]] + a_self * dt * L   (base = UN)
//   acc_mode 1: ACC = base + b*dt*L; 2: ACC += b*dt*L; 3 (last stage): u_out = ACC + b*dt*L;
//   0: ACC untouched.  kwrite >= 0 stores L into that role (the slopes K hold L, not dt*L).
struct StagePlan {
  int in;         // role of the stage input (the tile is read from it, with neighbour traces)
  int out;        // role written with the next stage input (or U^{n+1} at the last stage)
  int kwrite;     // role to store L in, or -1
  int nread;      // number of stored slopes in the stage combination
  int kread[kMaxStages];
  double a_read[kMaxStages];
  float a_read_f[kMaxStages];  // FP32 copies of a_read (for the FP32 kernels)
  double a_self;
  int acc_mode;
  double b;
};

// One solve inside a launch (device memory; read by every CTA working on it).
struct SolveDesc {
  void* buf[kNumRoles];   // device pointers by role (dtype of the launch class)
  int E[3];               // elements per axis (1 beyond dim)
  int tile_begin;         // first global tile index of this solve in the launch
  long long nelem;
  // The kernel computes R' = L(U) / rhs_scale so that the first axis needs no multiply; the
  // stage update multiplies its coefficients by rhs_scale.  rhs_scale = vol of axis 0 unless zero.
  double rhs_scale;
  double vol_scale[3];    // (-2/h_a (Euler) or -2 a_a / h_a (advection)) / rhs_scale, times D F
  double lift_lo[3];      // advection: (2/h_a)(1/w_0) (a_a + |a_a|)/2; Euler: (1/h_a)/w_0; / rhs_scale
  double lift_hi[3];      // advection: (2/h_a)(1/w_N) (a_a - |a_a|)/2; Euler: (1/h_a)/w_N; / rhs_scale
  double c2;              // c^2 (Euler)
  double c;               // c (Euler, LLF alpha)
  double dt;
  // FP32 copies of the geometric coefficients above (an FP32 kernel must not spend FP64
  // operations -- 1/64 of the FP32 rate on B300 -- converting them per node)
  float f_vol_scale[3], f_lift_lo[3], f_lift_hi[3], f_c2, f_c;
  // Partitioned solves: traces of the neighbouring partition across the low / high boundary
  // along each axis, layout [v][transverse element][face node] (face node = the index of the
  // line through it); NULL = periodic wrap inside this solve.
  const void* halo_lo[3];
  const void* halo_hi[3];
  // Device int of the solve's owner (a context's or a serving slot's status word), or NULL: a
  // stage kernel whose bulk-copy wait runs out sets it for every solve of the launch (the CTA
  // that gives up leaves tiles of any of them unprocessed).  Sticky until the owner resets it.
  int* status;
};

// Header of a launch's work list (device memory): tiles are numbered across all solves.  The
// host uploads the fields before `err` (kGroupHeaderUpload bytes) whenever the work list
// changes; `err` is zeroed once when the header is allocated and then written only by the
// kernels, so a flag raised by one launch survives later uploads until the host reads it.
struct GroupHeader {
  int nsolves;
  int ntiles;
  int epb;                // elements per CTA tile
  int variant;            // kernel mapping: kLineKernel or kLineVarKernel
  int wait_polls;         // polls of a bulk-copy wait before it gives up (0: kBulkWaitPolls)
  int stall_copies;       // test switch: arm the bulk-copy barrier but issue no copy, so the
                          // wait runs out (nothing is in flight when the kernel leaves); 0 normally
  int err;                // set by a stage kernel whose bulk-copy wait ran out (0 otherwise)
  int pad;
};
constexpr size_t kGroupHeaderUpload = offsetof(GroupHeader, err);
constexpr int kStageErrBulkWait = 1;
constexpr int kBulkWaitPolls = 1 << 22;

// Thread mappings of one stage (identical arithmetic, bitwise-identical results):
// kLineKernel: one thread per line of n nodes for all variables (fewest FP64 operations);
// kLineVarKernel: one thread per (line, variable): more threads per element for the same
// shared memory (higher occupancy for the multi-variable Euler classes).
enum { kLineKernel = 0, kLineVarKernel = 1 };

// Bytes per state value of a precision code (NDG_F64, NDG_F32, NDG_F64_FF): FP32 is the only
// 4-byte one.
inline int dtype_bytes(int dtype) { return dtype == 1 ? 4 : 8; }

// Kernel class: everything that is a template parameter of the stage kernel.
struct KernelClass {
  int dim, degree, equation, dtype;
  int mass = 0;  // NDG_MASS_LUMPED / NDG_MASS_EXACT (separate kernel instantiations)
  bool operator==(const KernelClass& o) const {
    return dim == o.dim && degree == o.degree && equation == o.equation && dtype == o.dtype && mass == o.mass;
  }
};

// Launch one RK stage of the fused kernel for a group: `grid` CTAs loop over the group's tiles.
// Returns a cudaError_t value.
int launch_stage(const KernelClass& kc, int variant, int grid, int epb, const SolveDesc* solves,
                 const GroupHeader* header, const StagePlan& plan, void* stream);
// One RK stage in split form (per axis a volume-term and a surface-term kernel, then the update
// kernel) over the right-hand-side array R (state-sized, the class's precision); the fused
// kernel's operations in the same order.  FP64 / FP32, lumped mass.  Returns a cudaError_t value.
int launch_split_stage(const KernelClass& kc, const SolveDesc& sd, const StagePlan& plan, void* R, void* stream);
// Records the shape of a failed stage launch; appended to the next error message.
void launch_error_detail(int grid, int threads, size_t smem, int max_threads, int regs, size_t local,
                         int max_dyn_smem);
// Threads and dynamic shared memory of one CTA for a class, mapping and tile size.
void stage_launch_shape(const KernelClass& kc, int variant, int epb, int* threads, size_t* smem_bytes);
// Ensure the kernel's attributes (max dynamic smem) are set; returns cudaError_t.
int prepare_stage_kernel(const KernelClass& kc, int variant, int epb, int* max_blocks_per_sm);

// Upload the basis of every degree to constant memory on the current device (idempotent).
int upload_bases();

// Norm reduction: partial sums per block into `partials` (nblocks * kNormFields doubles), then
// the final single-block pass into `result` (kNormFields doubles).
constexpr int kNormFields = 10;  // l2sq, linf, integral[4], max_speed, nonfinite, spare x2
int launch_norms(int dtype, int dim, int degree, int equation, const void* U, const void* ref,
                 long long nelem, double jac, double c, const double* velocity, int nblocks,
                 double* partials, double* result, void* stream);
constexpr int kNormBlocks = 296;

// Layout conversion between element layout and grid layout (device to device).
int launch_relayout(int dtype, int dim, int degree, int nvar, const int* E, const void* src,
                    void* dst, bool to_element, void* stream);

}  // namespace ndg
