/*
 * ndg.h -- C ABI of libndg, a B300 (sm_103a) implementation of the hot path of the nodal
 * discontinuous Galerkin (NDG) + explicit Runge-Kutta method of arXiv:2510.05254
 * ("Performance of a high-order MPI-Kokkos accelerated fluid solver"), Sec. 2:
 * the DG right-hand side fused with the RK stage update, for linear advection and isothermal
 * Euler in 1D/2D/3D on tensor-product Legendre-Gauss-Lobatto (LGL) elements of degree 1..7.
 *
 * Conventions for every entry point:
 *   - Return value: NDG_OK (0) or a positive NDG_E* code; nothing aborts, exits or traps.  The
 *     message of the last failure on the calling thread is returned by ndg_last_error().
 *   - Pointers are plain host or device addresses, as each argument states.  Inputs are copied;
 *     the caller keeps ownership of its buffers.  Device state is owned by the library and is
 *     released by the matching destroy call.
 *   - Work is enqueued on the context's CUDA stream (ndg_config.stream, a cudaStream_t; NULL lets
 *     the library create its own non-blocking stream).  Only ndg_norms, ndg_get_state (to host),
 *     ndg_stable_dt, ndg_synchronize and the pool calls wait for the GPU.
 *
 * State layouts (argument `layout`):
 *   NDG_LAYOUT_ELEMENT (0): U[v][e][node], v < nvar, e = ex + Ex*(ey + Ey*ez),
 *       node = i + n*(j + n*k), n = degree + 1 (each element's nodes contiguous).
 *   NDG_LAYOUT_GRID (1): U[v][z][y][x] over the global node grid, x = ex*n + i (nodes shared by
 *       two elements appear twice, as in the element layout).
 * Element ex spans [ex*h, (ex+1)*h], h = length/E, node i at ex*h + (h/2)(xi_i + 1) (the paper's
 * Eq. (transformation) with the element offset added).
 */
#ifndef NDG_H
#define NDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
enum {
  NDG_OK = 0,
  NDG_EINVAL = 1,     /* bad argument: dim, degree, element count, flux/equation mismatch, dt, size */
  NDG_ENOMEM = 2,     /* device/host allocation failed, or a memory budget would be exceeded */
  NDG_ECUDA = 3,      /* a CUDA runtime call failed (message carries the CUDA error string) */
  NDG_ENONFINITE = 4, /* ndg_norms found NaN or Inf in the state (the norms are still written) */
  NDG_EAGAIN = 5,     /* pool: result not ready yet */
  NDG_ETIMEOUT = 6,   /* pool: wait ran past its deadline */
  NDG_ESTATE = 7      /* call not valid in the object's current state (e.g. step before set_state) */
};

/* ---- enumerations ---------------------------------------------------------------------- */
enum { NDG_ADVECTION = 0, NDG_ISO_EULER = 1 };   /* Eq. (advection2d), Eq. (eulerIso2d) */
enum { NDG_FLUX_UPWIND = 0, NDG_FLUX_LLF = 1 };  /* Eq. (LF); upwind is valid for advection only */
enum { NDG_RK3 = 3, NDG_RK4 = 4, NDG_RK6 = 6 };  /* Eq. (RK3), Eq. (RK4), Eq. (RK6) */
/* Precision of the GPU path.  NDG_F64: FP64 state and arithmetic.  NDG_F32: FP32 state and
 * arithmetic (norms accumulate in FP64).  NDG_F64_FF: FP64 state, fluxes, face terms and stage
 * update, with the D contraction in float-float (unevaluated sums of two floats) on the FP32
 * pipe -- on B300 an FP64 operation costs 64 FP32 ones -- accurate to ~2^-44 of sum |D||F|
 * (within 1e-12 relative per step of the FP64 path); a line holding a value outside
 * [2^-74, 2^127] in magnitude is contracted in FP64.  The paper computes in FP64 throughout. */
enum { NDG_F64 = 0, NDG_F32 = 1, NDG_F64_FF = 2 };
enum { NDG_LAYOUT_ELEMENT = 0, NDG_LAYOUT_GRID = 1 };
/* Thread mapping of the stage kernel (identical arithmetic, bitwise-identical results):
 * LINE = one thread per line of nodes for all variables (fewest FP64 operations),
 * LINE_VAR = one thread per (line, variable): nvar times more threads per element for the same
 * shared memory (higher occupancy for isothermal Euler).
 * AUTO = the autotuned choice for the kernel class, else LINE. */
enum { NDG_KERNEL_AUTO = 0, NDG_KERNEL_LINE = 1, NDG_KERNEL_LINE_VAR = 2 };
/* Mass matrix of the element basis.  LUMPED (default): the paper's, int h_k h_l ~= w_k delta_kl by
 * the LGL quadrature (Sec. 2.1, Eq. (lag_coefs)), so a face term lifts onto the end node only.
 * EXACT: the exactly integrated mass matrix of the textbook nodal DG method the paper cites; the
 * volume term is unchanged (the LGL quadrature of h_l times a degree N-1 polynomial is exact) and a
 * face term lifts onto every node of the line by M^-1 e_0 / M^-1 e_N.  A correctness variant,
 * not a faster one (two more multiply-adds per node and axis). */
enum { NDG_MASS_LUMPED = 0, NDG_MASS_EXACT = 1 };

typedef struct ndg_ctx ndg_ctx;     /* one solve: state, buffers, stream, launch plan */
typedef struct ndg_batch ndg_batch; /* several solves stepped by one graph per RK step */
typedef struct ndg_pool ndg_pool;   /* serving pool: admission + continuous batching */

/* Problem description.  Start from ndg_config_init() and set what differs. */
typedef struct {
  int dim;            /* 1, 2 or 3 */
  int degree;         /* polynomial degree N, 1..7 (n = N+1 LGL nodes per axis) */
  int elems[3];       /* elements per axis, >= 1 (axes >= dim ignored) */
  int equation;       /* NDG_ADVECTION or NDG_ISO_EULER */
  int flux;           /* NDG_FLUX_UPWIND (advection) or NDG_FLUX_LLF (both equations) */
  int dtype;          /* NDG_F64, NDG_F32 or NDG_F64_FF */
  double length[3];   /* periodic domain [0, length[a]] per axis; default 1 */
  double velocity[3]; /* advection velocity a (advection only); default (1, 0, 0) */
  double sound_speed; /* isothermal sound speed c (Euler only); default 1 */
  void* stream;       /* cudaStream_t to run on; NULL: the context creates its own */
  int elems_per_block;/* elements per CTA of the stage kernel; 0: library default */
  int device;         /* CUDA device ordinal; default 0 */
  int kernel;         /* NDG_KERNEL_AUTO (default), NDG_KERNEL_LINE or NDG_KERNEL_LINE_VAR */
  int mass;           /* NDG_MASS_LUMPED (default) or NDG_MASS_EXACT */
} ndg_config;

/* Norms by LGL quadrature on every element (Sec. 3.1's L2 norm). */
typedef struct {
  double l2;          /* sqrt(sum_v int (U_v - ref_v)^2 dx), ref = 0 when none is given */
  double linf;        /* max |U - ref| over all nodes and variables */
  double integral[4]; /* int U_v dx: mass (v = 0) and momentum (v >= 1) for Euler */
  double max_speed;   /* advection: sum_a |a_a|; Euler: max over nodes of sum_a |u_a| + dim*c */
  double t;           /* simulated time accumulated in FP64 on the host */
  int64_t steps;      /* RK steps taken since the last ndg_set_state */
  int64_t nonfinite;  /* number of NaN/Inf values in U */
} ndg_norms_t;

typedef struct {
  int nvar;            /* 1 (advection) or dim+1 (Euler) */
  int nodes_per_elem;  /* n^dim */
  int64_t nelem;       /* product of elems[a] over a < dim */
  int64_t ndof;        /* nvar * nelem * nodes_per_elem */
  size_t state_bytes;  /* ndof * 8 (FP64, FP64_FF) or ndof * 4 (FP32) */
  size_t device_bytes; /* device memory the context holds now */
  int elems_per_block; /* stage-kernel tile in use */
  int kernel;          /* stage-kernel mapping in use: NDG_KERNEL_LINE or NDG_KERNEL_LINE_VAR */
} ndg_info_t;

/* Fill cfg with defaults: 2D, degree 7, 16x16 elements, advection, upwind, FP64, unit square,
 * velocity (1,0,0), c = 1, stream NULL, elems_per_block 0, device 0, lumped mass.  Returns
 * NDG_EINVAL on NULL. */
int ndg_config_init(ndg_config* cfg);

/* Create a context (Sec. 2: NDG discretisation of a periodic box).  Builds the LGL basis on the
 * host in FP64 (nodes, weights, differentiation matrix), uploads it, allocates the state and
 * RK buffers on the device.  elems[3] is read for a < dim.  Errors: NDG_EINVAL (dim not in 1..3,
 * degree not in 1..7, elems < 1, upwind with Euler, non-positive length or c), NDG_ENOMEM,
 * NDG_ECUDA.  *out is set only on success. */
int ndg_create(int dim, int degree, const int elems[3], int equation, int flux, ndg_ctx** out);
int ndg_create_ex(const ndg_config* cfg, ndg_ctx** out);

/* Release everything the context owns (waits for its stream first).  NULL is accepted. */
int ndg_destroy(ndg_ctx* ctx);

/* Copy a state into the context: nbytes must equal info.state_bytes; src is a host pointer
 * (src_on_device = 0; pageable or pinned) or a device pointer (1) of the context's dtype, in
 * `layout`.  Resets t and the step counter, and clears the failure flag of earlier steps (see
 * ndg_synchronize).  Async on the context stream for device sources; a host source is fully
 * read before the call returns. */
int ndg_set_state(ndg_ctx* ctx, const void* src, size_t nbytes, int src_on_device, int layout);

/* Copy the current state out (same size/layout rules).  To host: waits for the copy, and
 * returns NDG_ECUDA when the context's failure flag is set (see ndg_synchronize). */
int ndg_get_state(ndg_ctx* ctx, void* dst, size_t nbytes, int dst_on_device, int layout);

/* Advance nsteps steps of size dt with Runge-Kutta scheme rk (NDG_RK3/4/6; Eq. (RK3), (RK4),
 * (RK6)).  Each RK stage is one launch of the fused kernel: volume term (sum-factorised D along
 * every axis), numerical flux + lift at the element faces, and the stage update.  Steps are
 * replayed from a CUDA graph.  No host synchronisation.  Errors: NDG_EINVAL (dt <= 0 or not
 * finite, nsteps < 0, unknown rk), NDG_ESTATE (no state set), NDG_ECUDA. */
int ndg_step(ndg_ctx* ctx, double dt, int nsteps, int rk_scheme);

/* The same steps as ndg_step, for verification: every RK stage runs in split form -- per axis a
 * volume-term kernel (sum-factorised D, Sec. 2.1) and a surface-term kernel (numerical flux of
 * Eq. (LF) lifted by the lumped mass), then the stage-update kernel (Eq. (RK3)/(RK4)/(RK6)) --
 * over a state-sized right-hand-side array the context allocates on first use.  The operations
 * are the fused kernel's in the same order, so the result equals ndg_step's bit for bit.  No
 * graph, no tiles; slower.  NDG_F64 and NDG_F32 with the lumped mass (NDG_EINVAL otherwise);
 * other errors as ndg_step. */
int ndg_step_split(ndg_ctx* ctx, double dt, int nsteps, int rk_scheme);

/* Norms of the state, or of state - ref when ref is not NULL (ref has the context's dtype and
 * element layout, on the host if ref_on_device = 0, else on the device).  FP64 accumulation,
 * deterministic (fixed reduction order, no atomics).  Waits for the result.  Returns
 * NDG_ENONFINITE when the state holds NaN/Inf (out is still filled), NDG_ECUDA when the
 * context's failure flag is set (see ndg_synchronize). */
int ndg_norms(ndg_ctx* ctx, const void* ref, int ref_on_device, ndg_norms_t* out);

/* Stable time step dt = cfl * h_min / lambda (h_min the smallest physical LGL node spacing,
 * lambda the max_speed of ndg_norms).  Waits for the result. */
int ndg_stable_dt(ndg_ctx* ctx, double cfl, double* dt);

/* Node coordinates in the element layout, X[a][e][node] for a < dim, into a host buffer of
 * dim * nelem * nodes_per_elem doubles. */
int ndg_node_coords(ndg_ctx* ctx, double* host_out, size_t count);

int ndg_info(const ndg_ctx* ctx, ndg_info_t* out);

/* LGL nodes xi[0..degree] (ascending, xi_0 = -1, xi_N = 1) and quadrature weights w[0..degree]
 * of the library's FP64 host basis (Sec. 2.1): host arrays of degree+1 doubles.  No device
 * access.  NDG_EINVAL for degree outside 1..7 or NULL pointers. */
int ndg_lgl(int degree, double* xi, double* w);

/* The stream the context runs on (a cudaStream_t). */
void* ndg_stream(const ndg_ctx* ctx);

/* Wait for all work queued on the context's stream.  Returns NDG_ECUDA when a stage kernel that
 * stepped this context (alone, in a batch or as a partition block) gave up waiting for its
 * bulk copies into shared memory: every wait is bounded, and a CTA that gives up leaves tiles
 * unprocessed, so the state is not valid.  The flag stays set (ndg_get_state and ndg_norms
 * report it too) until the next ndg_set_state. */
int ndg_synchronize(ndg_ctx* ctx);

/* Test hook for the failure path above.  With polls > 0, every launch work list uploaded after
 * the call (contexts created or given a new dt, batch steps, partitions, pool membership
 * changes) makes the stage kernels that copy their tiles by bulk copies (FP32 degree 5 in
 * 2D/3D, FP32 degree 7 in 3D) arm their copy barrier without issuing the copies and give up
 * after `polls` polls, so the bounded wait runs out and the failure flag is raised; nothing is
 * left in flight.  polls = 0 restores normal operation (the default limit of 2^22 polls).
 * Process-wide; for tests only.  NDG_EINVAL for polls < 0. */
int ndg_debug_stall_copies(int polls);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* ndg_last_error(void);

/* Route the library's device allocations through caller-supplied functions (e.g. a framework's
 * caching allocator).  alloc(bytes, user, stream) returns a device pointer or NULL;
 * free(ptr, user, stream) releases it.  Pass NULLs to return to cudaMalloc/cudaFree.  Affects
 * allocations made after the call.  Pointers must be aligned to 256 bytes, as cudaMalloc's are
 * (the kernels access state arrays in 16-byte units); a less aligned one is handed back to free
 * and the allocating call fails with NDG_ECUDA. */
typedef void* (*ndg_alloc_fn)(size_t bytes, void* user, void* stream);
typedef void (*ndg_free_fn)(void* ptr, void* user, void* stream);
int ndg_set_allocator(ndg_alloc_fn alloc, ndg_free_fn free_fn, void* user);

/* Choose the stage kernel's elements per block and thread mapping for this context by timing
 * the candidates on its own state (which is restored bitwise afterwards).  Results are cached
 * per (dim, degree, equation, dtype) for the process, and in the text file named by the
 * environment variable NDG_AUTOTUNE_CACHE when set.  best_epb / best_ms may be NULL; the mapping
 * chosen is reported by ndg_info. */
int ndg_autotune(ndg_ctx* ctx, int rk_scheme, int* best_epb, double* best_ms);

/* Norms without any allocation.  The paper has no counterpart: this entry point exists for
 * callers that may not allocate device memory -- for example an application that hands all of
 * the GPU's memory to its own pool allocator at start-up, so that a cudaMalloc by a library
 * either fails or breaks its accounting, or a latency-critical loop that cannot afford the
 * device-wide synchronisation cudaMalloc/cudaFree may imply.
 *   cfg describes the problem (dim, degree, elems, equation, dtype, length, velocity,
 *       sound_speed, device; stream and elems_per_block are ignored);
 *   U:   device pointer to the state in element layout, cfg->dtype;
 *   ref: device pointer of the same shape or NULL (then the norms are of U itself);
 *   nblocks: reduction blocks, 0 for the default 296, at most 1024;
 *   out: device pointer to 8 doubles the caller owns, written with l2, linf, integral[0..3],
 *        max_speed, nonfinite count (the ndg_norms_t fields in that order);
 *   stream: cudaStream_t to enqueue on (NULL: the legacy default stream).
 * Asynchronous: nothing waits for the GPU.  The per-block partial sums live in one file-scope
 * device array of 1024 x 10 doubles (80 KiB) that every GPU which loads the library keeps until
 * the process exits; no call allocates or frees anything.  Every call looks the array's device
 * address up (cudaGetSymbolAddress, with cfg->device current); on a device's first call that
 * lookup may load the library's module there -- make that first call before any stream
 * capture.  All calls share the array: each call writes the partials it later reads, so nothing
 * has to start at zero, but calls whose kernels overlap on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller.  Errors: NDG_EINVAL (bad cfg, NULL
 * U/out, nblocks outside 0..1024), NDG_ECUDA (this call's launch failed, or an error of earlier
 * work was already pending: that one is reported and left pending, not cleared). */
int ndg_norms_noalloc(const ndg_config* cfg, const void* U, const void* ref, int nblocks, double* out,
                      void* stream);

/* ---- batching: several independent solves stepped together ------------------------------- */
/* Group `n` contexts (all on the same device) into a batch.  One RK step of the batch is one
 * CUDA-graph replay in which every class of solve (dim, degree, equation, dtype, kernel mapping)
 * is one persistent stage-kernel launch per stage over all of that class's solves, the classes
 * running as parallel branches.  The contexts stay owned by the caller and must outlive the
 * batch; the batch runs on the first context's stream.  Results are bitwise those of ndg_step on
 * each context alone.  A failed bulk-copy wait during a batch step raises the failure flag of
 * every member context (reported by their ndg_synchronize, ndg_get_state and ndg_norms). */
int ndg_batch_create(ndg_ctx* const* ctxs, int n, ndg_batch** out);
/* dts[i] is the step of context i; every context advances nsteps steps of scheme rk. */
int ndg_batch_step(ndg_batch* b, const double* dts, int nsteps, int rk_scheme);
int ndg_batch_destroy(ndg_batch* b);

/* ---- domain decomposition: one solve split into rectangular partitions --------------------- */
/* The paper distributes the element grid over rectangular/cuboid subdomains and exchanges the
 * border values every RK sub-step (Sec. 3.2).  ndg_partition emulates that on one GPU: the global
 * problem gcfg (stream ignored) is split into parts[0] x parts[1] x parts[2] blocks (as even as
 * possible; parts[a] in 1..elems[a], axes >= dim ignored); each block is a solve with its own
 * arrays and halo buffers; before every stage a pack kernel writes every block's boundary traces
 * (n^(dim-1) face values per boundary element and variable) into its neighbours' halos -- the
 * buffers a multi-GPU version would send and receive -- and one batched stage launch advances all
 * blocks.  Results are bitwise those of the unpartitioned solve. */
typedef struct ndg_partition ndg_partition;
int ndg_partition_create(const ndg_config* gcfg, const int parts[3], ndg_partition** out);
/* Global state in element layout of the whole problem (host or device source), scattered to the
 * blocks on the device.  Waits for the copy. */
int ndg_partition_set_state(ndg_partition* p, const void* src, size_t nbytes, int src_on_device);
/* Gathers the blocks into the global element layout.  Waits for the copy. */
int ndg_partition_get_state(ndg_partition* p, void* dst, size_t nbytes, int dst_on_device);
/* nsteps steps of scheme rk: one graph replay per step (exchange + stage launch per stage). */
int ndg_partition_step(ndg_partition* p, double dt, int nsteps, int rk_scheme);
/* Norms of the whole state, combined from the blocks in a fixed order (no reference). */
int ndg_partition_norms(ndg_partition* p, ndg_norms_t* out);
/* Element offset and element counts of block `part` (blocks numbered x fastest). */
int ndg_partition_info(const ndg_partition* p, int part, int offset[3], int elems[3]);
int ndg_partition_destroy(ndg_partition* p);

/* ---- serving: continuous batching of independent solves under a memory budget -------------- */
typedef struct {
  double submit_s;    /* host time of submission (seconds, steady clock) */
  double admit_s;     /* host time the solve was admitted to the GPU */
  double done_s;      /* host time the result was ready on the host */
  double latency_s;   /* done_s - submit_s */
  double t;           /* simulated time reached */
  int64_t steps;      /* RK steps taken */
  size_t device_bytes;/* device memory the solve held */
} ndg_solve_stats_t;

/* Create a pool that admits solves while their device memory stays within budget_bytes and
 * steps all admitted solves together, one batched graph replay per RK step; solves join and
 * leave at step boundaries.  A host worker thread drives the GPU on a stream of its own. */
int ndg_pool_create(size_t budget_bytes, int device, ndg_pool** out);
/* Queue a solve: cfg describes it (stream ignored), u0 is a host array in element layout of
 * cfg->dtype (copied before return), run nsteps steps of size dt with scheme rk.  *ticket
 * identifies it.  NDG_ENOMEM if the solve alone exceeds the budget. */
int ndg_pool_submit(ndg_pool* p, const ndg_config* cfg, const void* u0, size_t nbytes, int rk,
                    double dt, int nsteps, uint64_t* ticket);
/* Wait up to timeout_s (0: do not wait) for the solve.  When done, copies the final state to
 * result (host, element layout; NULL to skip), fills stats (may be NULL) and forgets the ticket.
 * NDG_EAGAIN (timeout 0, not done), NDG_ETIMEOUT (waited, not done), NDG_EINVAL (unknown),
 * NDG_ECUDA (a stage kernel that stepped this solve gave up waiting for its bulk copies: the
 * result is not valid; or a CUDA call of the pool failed). */
int ndg_pool_poll(ndg_pool* p, uint64_t ticket, void* result, size_t nbytes,
                  ndg_solve_stats_t* stats, double timeout_s);
/* Counters: solves queued, running, finished; device bytes in use; peak device bytes. */
int ndg_pool_status(ndg_pool* p, int64_t* queued, int64_t* running, int64_t* finished,
                    size_t* bytes_in_use, size_t* peak_bytes);
/* Stops the worker after the solves already admitted finish; queued ones are dropped. */
int ndg_pool_destroy(ndg_pool* p);

#ifdef __cplusplus
}
#endif
#endif /* NDG_H */
