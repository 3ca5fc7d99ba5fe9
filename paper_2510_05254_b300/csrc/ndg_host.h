// Host-side helpers of libndg shared by the C-ABI implementation (api.cu) and the serving pool
// (pool.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/ndg.h"
#include "ndg_internal.h"

namespace ndg {

// error reporting (thread-local message for ndg_last_error)
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// device memory through the optional allocator hook
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t stream);
void dev_free(void* p, cudaStream_t stream);

const std::vector<StagePlan>& stage_plans(int rk);
int num_roles_for(int rk);
bool valid_rk(int rk);

// Launch resources of one kernel class over a set of solves (one persistent launch per stage).
struct Group {
  KernelClass kc{};
  int variant = 0;  // kLineKernel / kLineVarKernel
  int epb = 0;
  int grid = 0;
  int ntiles = 0;
  std::vector<SolveDesc> h_desc;
  SolveDesc* d_desc = nullptr;
  GroupHeader* d_hdr = nullptr;
  size_t cap = 0;
};
// Upload the work list and the header fields before `err` (the flag is zeroed only when the
// header is allocated).  The bulk-copy wait limit and the test switch that stalls the copies
// come from ndg_debug_stall_copies().
int group_upload(Group& g, cudaStream_t stream);
int group_check(const Group& g);  // after a stream sync: a stage kernel's wait that ran out
// After a stream sync: NDG_ECUDA if the device status word a stage kernel sets when its
// bulk-copy wait runs out (SolveDesc::status) is set, else NDG_OK.
int status_check(const int* d_status);
void group_free(Group& g, cudaStream_t stream);
// Capture one RK step of scheme rk (all stages) of the groups, as parallel branches.
int capture_step(const std::vector<Group*>& groups, int rk, cudaStream_t cap, cudaGraphExec_t* out);

int num_sms(int device);
// Stage-kernel tile: elements per CTA and thread mapping.
struct TileConfig {
  int epb = 0;
  int variant = 0;
};
TileConfig default_tile(const KernelClass& kc);
TileConfig tuned_tile(const KernelClass& kc);  // epb == 0 when the class was never tuned

// Accessors of a context for the partition emulation: its descriptor (buffers, geometry, dt),
// its RK buffers for scheme rk, and marking its state as set by a device-side copy.
SolveDesc ndg_ctx_desc(const ndg_ctx* c);
int ndg_ctx_ensure_buffers(ndg_ctx* c, int rk);
// Marks the state as set and clears the context's status word (stream-ordered on `stream`).
void ndg_ctx_mark_state(ndg_ctx* c, cudaStream_t stream);

// Geometry part of a solve descriptor (scales, lift coefficients, element counts).
void fill_solve_geometry(const ndg_config& cfg, const Basis& b, SolveDesc* d);
// Validate a configuration (no device access); NDG_OK or NDG_EINVAL with a message.
int check_config(const ndg_config& k);

}  // namespace ndg
