// C ABI of libndg (include/ndg.h): solve contexts, graph-replayed RK stepping, norms, state I/O,
// batching of several solves into one graph per RK step, and the tile-size autotuner.
#include <cuda_runtime.h>

#include <cstdint>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ndg.h"
#include "ndg_host.h"
#include "ndg_internal.h"

namespace ndg {
// per-(dtype, dim) dispatch tables from stage_<dtype>_d<dim>.cu
using LaunchFn = int (*)(int, int, int, const SolveDesc*, const GroupHeader*, const StagePlan&, void*);
using PrepareFn = int (*)(int, int, int*);
using ShapeFn = void (*)(int, int, int*, size_t*);
#define NDG_DECL(tag)                         \
  LaunchFn tag##_launch(int degree, int eq);  \
  PrepareFn tag##_prepare(int degree, int eq); \
  ShapeFn tag##_shape(int degree, int eq);
NDG_DECL(stage_f64_d1)
NDG_DECL(stage_f64_d2)
NDG_DECL(stage_f64_d3)
NDG_DECL(stage_f32_d1)
NDG_DECL(stage_f32_d2)
NDG_DECL(stage_f32_d3)
NDG_DECL(stage_f64ff_d1)
NDG_DECL(stage_f64ff_d2)
NDG_DECL(stage_f64ff_d3)
NDG_DECL(stage_f64x_d1)
NDG_DECL(stage_f64x_d2)
NDG_DECL(stage_f64x_d3)
NDG_DECL(stage_f32x_d1)
NDG_DECL(stage_f32x_d2)
NDG_DECL(stage_f32x_d3)
#undef NDG_DECL

namespace {
// Tables by [dtype][dim - 1]; the exact-mass classes (FP64 and FP32 only) by [dtype][dim - 1]
// of the second table.
LaunchFn pick_launch(const KernelClass& k) {
  static LaunchFn (*t[3][3])(int, int) = {{stage_f64_d1_launch, stage_f64_d2_launch, stage_f64_d3_launch},
                                          {stage_f32_d1_launch, stage_f32_d2_launch, stage_f32_d3_launch},
                                          {stage_f64ff_d1_launch, stage_f64ff_d2_launch, stage_f64ff_d3_launch}};
  static LaunchFn (*x[2][3])(int, int) = {{stage_f64x_d1_launch, stage_f64x_d2_launch, stage_f64x_d3_launch},
                                          {stage_f32x_d1_launch, stage_f32x_d2_launch, stage_f32x_d3_launch}};
  if (k.mass == NDG_MASS_EXACT) return k.dtype < 2 ? x[k.dtype][k.dim - 1](k.degree, k.equation) : nullptr;
  return t[k.dtype][k.dim - 1](k.degree, k.equation);
}
PrepareFn pick_prepare(const KernelClass& k) {
  static PrepareFn (*t[3][3])(int, int) = {
      {stage_f64_d1_prepare, stage_f64_d2_prepare, stage_f64_d3_prepare},
      {stage_f32_d1_prepare, stage_f32_d2_prepare, stage_f32_d3_prepare},
      {stage_f64ff_d1_prepare, stage_f64ff_d2_prepare, stage_f64ff_d3_prepare}};
  static PrepareFn (*x[2][3])(int, int) = {
      {stage_f64x_d1_prepare, stage_f64x_d2_prepare, stage_f64x_d3_prepare},
      {stage_f32x_d1_prepare, stage_f32x_d2_prepare, stage_f32x_d3_prepare}};
  if (k.mass == NDG_MASS_EXACT) return k.dtype < 2 ? x[k.dtype][k.dim - 1](k.degree, k.equation) : nullptr;
  return t[k.dtype][k.dim - 1](k.degree, k.equation);
}
ShapeFn pick_shape(const KernelClass& k) {
  static ShapeFn (*t[3][3])(int, int) = {{stage_f64_d1_shape, stage_f64_d2_shape, stage_f64_d3_shape},
                                         {stage_f32_d1_shape, stage_f32_d2_shape, stage_f32_d3_shape},
                                         {stage_f64ff_d1_shape, stage_f64ff_d2_shape, stage_f64ff_d3_shape}};
  static ShapeFn (*x[2][3])(int, int) = {{stage_f64x_d1_shape, stage_f64x_d2_shape, stage_f64x_d3_shape},
                                         {stage_f32x_d1_shape, stage_f32x_d2_shape, stage_f32x_d3_shape}};
  if (k.mass == NDG_MASS_EXACT && k.dtype < 2) return x[k.dtype][k.dim - 1](k.degree, k.equation);
  return t[k.dtype][k.dim - 1](k.degree, k.equation);
}
}  // namespace

int launch_stage(const KernelClass& kc, int variant, int grid, int epb, const SolveDesc* solves,
                 const GroupHeader* header, const StagePlan& plan, void* stream) {
  LaunchFn f = pick_launch(kc);
  if (!f) return (int)cudaErrorInvalidValue;
  return f(variant, grid, epb, solves, header, plan, stream);
}

void stage_launch_shape(const KernelClass& kc, int variant, int epb, int* threads, size_t* smem) {
  pick_shape(kc)(variant, epb, threads, smem);
}

int prepare_stage_kernel(const KernelClass& kc, int variant, int epb, int* max_blocks) {
  PrepareFn f = pick_prepare(kc);
  if (!f) return (int)cudaErrorInvalidValue;
  return f(variant, epb, max_blocks);
}

// ------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------
thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

thread_local std::string g_launch_detail;

void launch_error_detail(int grid, int threads, size_t smem, int max_threads, int regs, size_t local,
                         int max_dyn_smem) {
  char buf[256];
  snprintf(buf, sizeof(buf), " (grid %d, block %d, dynamic smem %zu; kernel: max block %d, %d registers, "
           "%zu B local, max dynamic smem %d)", grid, threads, smem, max_threads, regs, local, max_dyn_smem);
  g_launch_detail = buf;
}

int cuda_fail(cudaError_t e, const char* what) {
  std::string detail;
  detail.swap(g_launch_detail);
  return fail(NDG_ECUDA, "%s: %s%s", what, cudaGetErrorString(e), detail.c_str());
}

// ------------------------------------------------------------------------------------------
// device memory through the optional allocator hook
// ------------------------------------------------------------------------------------------
namespace {
std::mutex g_alloc_mu;
ndg_alloc_fn g_alloc = nullptr;
ndg_free_fn g_free = nullptr;
void* g_alloc_user = nullptr;
std::map<void*, std::pair<ndg_free_fn, void*>> g_hooked;  // ptr -> (free fn, user)
}  // namespace

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t stream) {
  ndg_alloc_fn a;
  ndg_free_fn f;
  void* user;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
    f = g_free;
    user = g_alloc_user;
  }
  if (a) {
    *p = a(bytes, user, (void*)stream);
    if (!*p) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<uintptr_t>(*p) & 255) {
      // the kernels access state arrays 16 bytes at a time: insist on cudaMalloc's alignment
      if (f) f(*p, user, (void*)stream);
      *p = nullptr;
      return cudaErrorInvalidValue;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_hooked[*p] = {f, user};
    return cudaSuccess;
  }
  return cudaMalloc(p, bytes);
}

void dev_free(void* p, cudaStream_t stream) {
  if (!p) return;
  ndg_free_fn f = nullptr;
  void* user = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    auto it = g_hooked.find(p);
    if (it != g_hooked.end()) {
      f = it->second.first;
      user = it->second.second;
      g_hooked.erase(it);
    }
  }
  if (f) f(p, user, (void*)stream);
  else cudaFree(p);
}

// ------------------------------------------------------------------------------------------
// Runge-Kutta stage plans (Eq. (RK3), (RK4), (RK6))
// ------------------------------------------------------------------------------------------
const std::vector<StagePlan>& stage_plans(int rk) {
  static std::vector<StagePlan> p3, p4, p6;
  static std::once_flag once;
  std::call_once(once, [] {
    auto mk = [](int in, int out, double a_self, int acc_mode, double b) {
      StagePlan s;
      std::memset(&s, 0, sizeof(s));
      s.in = in;
      s.out = out;
      s.kwrite = -1;
      s.nread = 0;
      s.a_self = a_self;
      s.acc_mode = acc_mode;
      s.b = b;
      return s;
    };
    // RK3 (Heun's third-order reading of Eq. (RK3)): c = (0, 1/3, 2/3), b = (1/4, 0, 3/4)
    p3 = {mk(kUN, kS0, 1.0 / 3.0, 1, 0.25), mk(kS0, kS1, 2.0 / 3.0, 0, 0.0), mk(kS1, kUN, 0.0, 3, 0.75)};
    // classical RK4, Eq. (RK4)
    p4 = {mk(kUN, kS0, 0.5, 1, 1.0 / 6.0), mk(kS0, kS1, 0.5, 2, 1.0 / 3.0),
          mk(kS1, kS0, 1.0, 2, 1.0 / 3.0), mk(kS0, kUN, 0.0, 3, 1.0 / 6.0)};
    // Luther's sixth-order seven-stage scheme, Eq. (RK6): A strictly lower triangular, rows
    // a[i][j] for stage input i (1-based stage i+1), b weights.
    const double s = std::sqrt(21.0);
    const double A[7][7] = {
        {0},
        {1.0},
        {3.0 / 8.0, 1.0 / 8.0},
        {8.0 / 27.0, 2.0 / 27.0, 8.0 / 27.0},
        {3.0 * (3.0 * s - 7.0) / 392.0, -8.0 * (7.0 - s) / 392.0, 48.0 * (7.0 - s) / 392.0,
         -3.0 * (21.0 - s) / 392.0},
        {-5.0 * (231.0 + 51.0 * s) / 1960.0, -40.0 * (7.0 + s) / 1960.0, -320.0 * s / 1960.0,
         3.0 * (21.0 + 121.0 * s) / 1960.0, 392.0 * (6.0 + s) / 1960.0},
        {15.0 * (22.0 + 7.0 * s) / 180.0, 120.0 / 180.0, 40.0 * (7.0 * s - 5.0) / 180.0,
         -63.0 * (3.0 * s - 2.0) / 180.0, -14.0 * (49.0 + 9.0 * s) / 180.0, 70.0 * (7.0 - s) / 180.0}};
    const double b[7] = {9.0 / 180.0, 0.0, 64.0 / 180.0, 0.0, 49.0 / 180.0, 49.0 / 180.0, 9.0 / 180.0};
    p6.clear();
    for (int st = 0; st < 7; ++st) {
      const int in = st == 0 ? kUN : (st % 2 == 1 ? kS0 : kS1);
      const int out = st == 6 ? kUN : (st % 2 == 0 ? kS0 : kS1);
      int acc_mode;
      if (st == 0) acc_mode = 1;
      else if (st == 6) acc_mode = 3;
      else acc_mode = b[st] != 0.0 ? 2 : 0;
      StagePlan sp = mk(in, out, st < 6 ? A[st + 1][st] : 0.0, acc_mode, b[st]);
      if (st < 6) {
        for (int j = 0; j < st; ++j) {
          if (A[st + 1][j] == 0.0) continue;
          sp.kread[sp.nread] = kK0 + j;
          sp.a_read[sp.nread] = A[st + 1][j];
          sp.a_read_f[sp.nread] = (float)A[st + 1][j];
          ++sp.nread;
        }
        // k_{st+1} is needed later if any later stage input (rows > st+1) uses it
        bool needed = false;
        for (int r = st + 2; r < 7; ++r) needed = needed || A[r][st] != 0.0;
        sp.kwrite = needed ? kK0 + st : -1;
      }
      p6.push_back(sp);
    }
  });
  return rk == 3 ? p3 : (rk == 4 ? p4 : p6);
}

int num_roles_for(int rk) { return rk == 6 ? kK0 + 5 : kK0; }

}  // namespace ndg

using namespace ndg;

// ------------------------------------------------------------------------------------------
// contexts
// ------------------------------------------------------------------------------------------
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

namespace ndg {

namespace {
// ndg_debug_stall_copies: the wait limit and the stall switch written into every header upload
std::atomic<int> g_debug_wait_polls{0};
}  // namespace

int group_upload(Group& g, cudaStream_t stream) {
  if (g.h_desc.size() > g.cap || !g.d_desc) {
    if (g.d_desc) dev_free(g.d_desc, stream);
    if (!g.d_hdr) {
      cudaError_t e = dev_alloc((void**)&g.d_hdr, sizeof(GroupHeader), stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(g.d_hdr, 0, sizeof(GroupHeader), stream);
      if (e != cudaSuccess) return cuda_fail(e, "alloc group header");
    }
    size_t cap = std::max<size_t>(1, g.h_desc.size());
    cudaError_t e = dev_alloc((void**)&g.d_desc, cap * sizeof(SolveDesc), stream);
    if (e != cudaSuccess) return cuda_fail(e, "alloc solve descriptors");
    g.cap = cap;
  }
  const int polls = g_debug_wait_polls.load();
  GroupHeader h{(int)g.h_desc.size(), g.ntiles, g.epb, g.variant, polls, polls > 0 ? 1 : 0, 0, 0};
  // the fields before `err` only: a flag raised by an earlier launch stays until it is read
  cudaError_t e = cudaMemcpyAsync(g.d_hdr, &h, kGroupHeaderUpload, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess && !g.h_desc.empty())
    e = cudaMemcpyAsync(g.d_desc, g.h_desc.data(), g.h_desc.size() * sizeof(SolveDesc),
                        cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return cuda_fail(e, "upload work list");
  return NDG_OK;
}

// After the stream has been synchronised: NDG_ECUDA if a stage kernel of the group flagged a
// bulk-copy wait that ran out (the state is then not valid), else NDG_OK.
int group_check(const Group& g) {
  if (!g.d_hdr) return NDG_OK;
  int err = 0;
  cudaError_t e = cudaMemcpy(&err, &g.d_hdr->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "group status");
  if (err == kStageErrBulkWait)
    return fail(NDG_ECUDA, "stage kernel: a bulk copy into shared memory did not complete within the wait limit");
  return NDG_OK;
}

int status_check(const int* d_status) {
  if (!d_status) return NDG_OK;
  int st = 0;
  cudaError_t e = cudaMemcpy(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "solve status");
  if (st == kStageErrBulkWait)
    return fail(NDG_ECUDA, "stage kernel: a bulk copy into shared memory did not complete within the wait limit "
                           "(the state is not valid until a new one is set)");
  return NDG_OK;
}

void group_free(Group& g, cudaStream_t stream) {
  dev_free(g.d_desc, stream);
  dev_free(g.d_hdr, stream);
  g.d_desc = nullptr;
  g.d_hdr = nullptr;
  g.cap = 0;
}

int num_sms(int device) {
  static int cached[64] = {0};
  if (device < 0 || device >= 64) return 148;
  if (!cached[device]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    cached[device] = v > 0 ? v : 148;
  }
  return cached[device];
}

int default_epb_for(const KernelClass& kc, int variant) {
  const int n = kc.degree + 1;
  // about 128-256 threads per CTA (threads per element = n^(dim-1), times nvar for the
  // (line, variable) mapping), and at most ~100 KB of shared memory so that two CTAs fit on an SM
  int L = 1;
  for (int d = 1; d < kc.dim; ++d) L *= n;
  if (variant == kLineVarKernel) L *= kc.equation == NDG_ADVECTION ? 1 : kc.dim + 1;
  int epb = std::max(1, 256 / L);
  if (kc.dim == 3) epb = std::max(1, 192 / L);
  epb = std::min(epb, 64);
  while (epb > 1) {
    int threads;
    size_t smem;
    stage_launch_shape(kc, variant, epb, &threads, &smem);
    if (smem <= 100 * 1024) break;
    --epb;
  }
  return epb;
}

// Untuned choice: one thread per line (measured faster on B300 than one thread per line and
// variable for every class tried; the autotuner still tries both).
TileConfig default_tile(const KernelClass& kc) {
  TileConfig t;
  t.variant = kLineKernel;
  t.epb = default_epb_for(kc, t.variant);
  return t;
}

// Autotuned tiles per class for this process.
std::mutex g_tune_mu;
std::map<long long, TileConfig> g_tuned;
long long class_key(const KernelClass& k) {
  return ((((long long)k.dim * 16 + k.degree) * 2 + k.equation) * 4 + k.dtype) * 2 + k.mass;
}
// Optional persistent cache: NDG_AUTOTUNE_CACHE names a text file of lines
// "dim degree equation dtype mass epb variant", read once per process, rewritten after each
// autotune (lines of another form are skipped).
bool g_tune_loaded = false;
void load_tune_cache_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("NDG_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[256];
  while (std::fgets(line, sizeof(line), f)) {
    int d, n, e, t, m, epb, var;
    if (std::sscanf(line, "%d %d %d %d %d %d %d", &d, &n, &e, &t, &m, &epb, &var) != 7) continue;
    if (epb > 0 && epb <= 1024 && (var == kLineKernel || var == kLineVarKernel) && (m == 0 || m == 1))
      g_tuned.emplace(class_key(KernelClass{d, n, e, t, m}), TileConfig{epb, var});
  }
  std::fclose(f);
}
void save_tune_cache_locked() {
  const char* path = std::getenv("NDG_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  for (auto& kv : g_tuned) {
    long long key = kv.first;
    const int mass = (int)(key % 2);
    key /= 2;
    const int dtype = (int)(key % 4), eq = (int)((key / 4) % 2), deg = (int)((key / 8) % 16), dim = (int)(key / 128);
    std::fprintf(f, "%d %d %d %d %d %d %d\n", dim, deg, eq, dtype, mass, kv.second.epb, kv.second.variant);
  }
  std::fclose(f);
  std::rename(tmp.c_str(), path);
}
TileConfig tuned_tile(const KernelClass& k) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  load_tune_cache_locked();
  auto it = g_tuned.find(class_key(k));
  return it == g_tuned.end() ? TileConfig{} : it->second;
}

}  // namespace ndg

struct ndg_ctx {
  ndg_config cfg;
  KernelClass kc;
  int n = 0, npe = 0, nvar = 0;
  long long nelem = 0, ndof = 0;
  size_t esize = 0, state_bytes = 0, device_bytes = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t capture_stream = nullptr;
  void* buf[kNumRoles] = {nullptr};
  bool have_state = false;
  double t = 0.0;
  long long steps = 0;
  TileConfig tile;
  Basis basis;
  SolveDesc desc;  // this solve's descriptor (buffers, geometry, dt)
  Group group;     // the solve alone as a launch group
  cudaGraphExec_t graph[7] = {nullptr};
  TileConfig graph_tile[7];
  double* d_partials = nullptr;
  double* d_result = nullptr;
  double* h_result = nullptr;  // pinned
  void* d_scratch = nullptr;   // state-sized scratch (host refs, grid layout)
  int* d_status = nullptr;     // set by a stage kernel whose bulk-copy wait ran out; cleared by set_state
  std::mutex mu;
};

namespace ndg {

int ensure_buffers(ndg_ctx* c, int rk) {
  const int roles = num_roles_for(rk);
  for (int r = 0; r < roles; ++r) {
    if (c->buf[r]) continue;
    cudaError_t e = dev_alloc(&c->buf[r], c->state_bytes, c->stream);
    if (e != cudaSuccess) {
      return fail(NDG_ENOMEM, "device allocation of %zu bytes failed: %s", c->state_bytes,
                  cudaGetErrorString(e));
    }
    c->device_bytes += c->state_bytes;
    c->desc.buf[r] = c->buf[r];
  }
  return NDG_OK;
}

void fill_solve_geometry(const ndg_config& cfg, const Basis& b, SolveDesc* dp) {
  SolveDesc& d = *dp;
  long long nelem = 1;
  for (int a = 0; a < 3; ++a) {
    d.E[a] = a < cfg.dim ? cfg.elems[a] : 1;
    nelem *= d.E[a];
  }
  d.nelem = nelem;
  const int N = cfg.degree;
  const double w0 = b.w[0], wN = b.w[N];
  for (int a = 0; a < 3; ++a) {
    d.vol_scale[a] = d.lift_lo[a] = d.lift_hi[a] = 0.0;
    if (a >= cfg.dim) continue;
    const double h = cfg.length[a] / cfg.elems[a];
    if (cfg.equation == NDG_ADVECTION) {
      const double va = cfg.velocity[a];
      d.vol_scale[a] = -2.0 * va / h;
      d.lift_lo[a] = (2.0 / h) / w0 * 0.5 * (va + std::fabs(va));
      d.lift_hi[a] = (2.0 / h) / wN * 0.5 * (va - std::fabs(va));
    } else {
      d.vol_scale[a] = -2.0 / h;
      d.lift_lo[a] = (1.0 / h) / w0;
      d.lift_hi[a] = (1.0 / h) / wN;
    }
  }
  d.c = cfg.sound_speed;
  d.c2 = cfg.sound_speed * cfg.sound_speed;
  d.rhs_scale = d.vol_scale[0] != 0.0 ? d.vol_scale[0] : 1.0;
  for (int a = 0; a < 3; ++a) {
    d.vol_scale[a] /= d.rhs_scale;
    d.lift_lo[a] /= d.rhs_scale;
    d.lift_hi[a] /= d.rhs_scale;
    d.f_vol_scale[a] = (float)d.vol_scale[a];
    d.f_lift_lo[a] = (float)d.lift_lo[a];
    d.f_lift_hi[a] = (float)d.lift_hi[a];
  }
  d.f_c = (float)d.c;
  d.f_c2 = (float)d.c2;
}

void fill_desc_geometry(ndg_ctx* c) { fill_solve_geometry(c->cfg, c->basis, &c->desc); }

void drop_graphs(ndg_ctx* c) {
  for (int i = 0; i < 7; ++i)
    if (c->graph[i]) {
      cudaGraphExecDestroy(c->graph[i]);
      c->graph[i] = nullptr;
    }
}

int set_group_tile(ndg_ctx* c, TileConfig t) {
  int maxb = 0;
  int e = prepare_stage_kernel(c->kc, t.variant, t.epb, &maxb);
  if (e != 0 || maxb < 1)
    return fail(NDG_EINVAL, "elems_per_block %d does not fit this kernel class (%s)", t.epb,
                e ? cudaGetErrorString((cudaError_t)e) : "no resident CTA");
  c->tile = t;
  Group& g = c->group;
  g.kc = c->kc;
  g.epb = t.epb;
  g.variant = t.variant;
  g.ntiles = (int)((c->nelem + t.epb - 1) / t.epb);
  c->desc.tile_begin = 0;
  g.grid = std::min(g.ntiles, maxb * num_sms(c->cfg.device));
  g.h_desc.assign(1, c->desc);
  drop_graphs(c);
  return group_upload(g, c->stream);
}

// Capture one RK step (all stages) of the given groups, classes as parallel branches.
int capture_step(const std::vector<Group*>& groups, int rk, cudaStream_t cap, cudaGraphExec_t* out) {
  const auto& plans = stage_plans(rk);
  std::vector<cudaStream_t> side(groups.size(), nullptr);
  std::vector<cudaEvent_t> ev(groups.size() + 1, nullptr);
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < groups.size() && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[groups.size()], cudaEventDisableTiming);
  cudaGraph_t graph = nullptr;
  int rc = NDG_OK;
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaEventRecord(ev[groups.size()], cap);
    for (size_t i = 0; i < groups.size(); ++i) {
      Group* g = groups[i];
      cudaStream_t s = side[i];
      cudaStreamWaitEvent(s, ev[groups.size()], 0);
      for (const StagePlan& p : plans) {
        int le = launch_stage(g->kc, g->variant, std::max(1, g->grid), g->epb, g->d_desc, g->d_hdr, p, s);
        if (le != 0 && rc == NDG_OK) rc = cuda_fail((cudaError_t)le, "stage launch");
      }
      cudaEventRecord(ev[i], s);
      cudaStreamWaitEvent(cap, ev[i], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e2 != cudaSuccess && rc == NDG_OK) rc = cuda_fail(e2, "end capture");
  } else {
    rc = cuda_fail(e, "begin capture");
  }
  if (rc == NDG_OK) {
    e = cudaGraphInstantiate(out, graph, 0);
    if (e != cudaSuccess) rc = cuda_fail(e, "graph instantiate");
  }
  if (graph) cudaGraphDestroy(graph);
  for (auto s : side)
    if (s) cudaStreamDestroy(s);
  for (auto x : ev)
    if (x) cudaEventDestroy(x);
  return rc;
}

bool valid_rk(int rk) { return rk == 3 || rk == 4 || rk == 6; }

SolveDesc ndg_ctx_desc(const ndg_ctx* c) { return c->desc; }
int ndg_ctx_ensure_buffers(ndg_ctx* c, int rk) { return ensure_buffers(c, rk); }
void ndg_ctx_mark_state(ndg_ctx* c, cudaStream_t stream) {
  cudaMemsetAsync(c->d_status, 0, sizeof(int), stream);
  c->have_state = true;
  c->t = 0.0;
  c->steps = 0;
}

int check_config(const ndg_config& k) {
  if (k.dim < 1 || k.dim > 3) return fail(NDG_EINVAL, "dim must be 1, 2 or 3 (got %d)", k.dim);
  if (k.degree < 1 || k.degree > kMaxDegree)
    return fail(NDG_EINVAL, "degree must be in 1..%d (got %d)", kMaxDegree, k.degree);
  if (k.equation != NDG_ADVECTION && k.equation != NDG_ISO_EULER)
    return fail(NDG_EINVAL, "unknown equation %d", k.equation);
  if (k.flux != NDG_FLUX_UPWIND && k.flux != NDG_FLUX_LLF)
    return fail(NDG_EINVAL, "unknown flux %d", k.flux);
  if (k.equation == NDG_ISO_EULER && k.flux != NDG_FLUX_LLF)
    return fail(NDG_EINVAL, "isothermal Euler takes the local Lax-Friedrichs flux");
  if (k.dtype != NDG_F64 && k.dtype != NDG_F32 && k.dtype != NDG_F64_FF)
    return fail(NDG_EINVAL, "unknown dtype %d", k.dtype);
  for (int a = 0; a < k.dim; ++a) {
    if (k.elems[a] < 1) return fail(NDG_EINVAL, "elems[%d] must be >= 1", a);
    if (!(k.length[a] > 0.0) || !std::isfinite(k.length[a]))
      return fail(NDG_EINVAL, "length[%d] must be positive", a);
    if (!std::isfinite(k.velocity[a])) return fail(NDG_EINVAL, "velocity must be finite");
  }
  if (k.equation == NDG_ISO_EULER && !(k.sound_speed > 0.0 && std::isfinite(k.sound_speed)))
    return fail(NDG_EINVAL, "sound speed must be positive");
  if (k.elems_per_block < 0) return fail(NDG_EINVAL, "elems_per_block must be >= 0");
  if (k.kernel != NDG_KERNEL_AUTO && k.kernel != NDG_KERNEL_LINE && k.kernel != NDG_KERNEL_LINE_VAR)
    return fail(NDG_EINVAL, "unknown kernel mapping %d", k.kernel);
  if (k.mass != NDG_MASS_LUMPED && k.mass != NDG_MASS_EXACT) return fail(NDG_EINVAL, "unknown mass matrix %d", k.mass);
  if (k.mass == NDG_MASS_EXACT && k.dtype == NDG_F64_FF)
    return fail(NDG_EINVAL, "the exact mass matrix is built for NDG_F64 and NDG_F32");
  return NDG_OK;
}


}  // namespace ndg

// ------------------------------------------------------------------------------------------
// public entry points
// ------------------------------------------------------------------------------------------
extern "C" {

const char* ndg_last_error(void) { return g_last_error.c_str(); }

int ndg_config_init(ndg_config* cfg) {
  if (!cfg) return fail(NDG_EINVAL, "cfg is NULL");
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->dim = 2;
  cfg->degree = 7;
  cfg->elems[0] = cfg->elems[1] = cfg->elems[2] = 16;
  cfg->equation = NDG_ADVECTION;
  cfg->flux = NDG_FLUX_UPWIND;
  cfg->dtype = NDG_F64;
  cfg->length[0] = cfg->length[1] = cfg->length[2] = 1.0;
  cfg->velocity[0] = 1.0;
  cfg->sound_speed = 1.0;
  return NDG_OK;
}

int ndg_set_allocator(ndg_alloc_fn alloc, ndg_free_fn free_fn, void* user) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(NDG_EINVAL, "allocator and free function must both be set or both be NULL");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_user = user;
  return NDG_OK;
}

int ndg_destroy(ndg_ctx* c) {
  if (!c) return NDG_OK;
  {
    DeviceGuard dg(c->cfg.device);
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    for (int r = 0; r < kNumRoles; ++r) dev_free(c->buf[r], c->stream);
    group_free(c->group, c->stream);
    dev_free(c->d_partials, c->stream);
    dev_free(c->d_result, c->stream);
    dev_free(c->d_scratch, c->stream);
    dev_free(c->d_status, c->stream);
    if (c->h_result) cudaFreeHost(c->h_result);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    if (c->own_stream) cudaStreamDestroy(c->stream);
  }
  delete c;
  return NDG_OK;
}

int ndg_create_ex(const ndg_config* cfg, ndg_ctx** out) {
  if (!cfg || !out) return fail(NDG_EINVAL, "NULL argument");
  const ndg_config& k = *cfg;
  {
    int vr = check_config(k);
    if (vr) return vr;
  }
  long long nelem = 1;
  for (int a = 0; a < k.dim; ++a) nelem *= k.elems[a];
  if (nelem > 0x7fffffffLL) return fail(NDG_EINVAL, "more than 2^31 - 1 elements");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1)
    return fail(NDG_ECUDA, "no CUDA device available");
  if (k.device < 0 || k.device >= ndev) return fail(NDG_EINVAL, "bad device %d", k.device);

  DeviceGuard dg(k.device);
  ndg_ctx* c = new ndg_ctx();
  c->cfg = k;
  for (int a = k.dim; a < 3; ++a) {
    c->cfg.elems[a] = 1;
    c->cfg.velocity[a] = 0.0;
  }
  c->kc = KernelClass{k.dim, k.degree, k.equation, k.dtype, k.mass};
  c->n = k.degree + 1;
  c->npe = 1;
  for (int a = 0; a < k.dim; ++a) c->npe *= c->n;
  c->nvar = k.equation == NDG_ADVECTION ? 1 : k.dim + 1;
  c->nelem = nelem;
  c->ndof = nelem * c->npe * c->nvar;
  c->esize = dtype_bytes(k.dtype);
  c->state_bytes = (size_t)c->ndof * c->esize;
  if (!build_basis(k.degree, &c->basis)) {
    delete c;
    return fail(NDG_EINVAL, "basis construction failed");
  }
  std::memset(&c->desc, 0, sizeof(c->desc));
  fill_desc_geometry(c);
  cudaError_t e;
  if (k.stream) {
    c->stream = (cudaStream_t)k.stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "stream create");
    }
    c->own_stream = true;
  }
  e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
  int rc = e == cudaSuccess ? NDG_OK : cuda_fail(e, "capture stream");
  if (rc == NDG_OK) rc = ensure_buffers(c, NDG_RK4);
  if (rc == NDG_OK) {
    e = dev_alloc((void**)&c->d_partials, kNormBlocks * kNormFields * sizeof(double), c->stream);
    if (e == cudaSuccess) e = dev_alloc((void**)&c->d_result, kNormFields * sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_result, kNormFields * sizeof(double));
    if (e == cudaSuccess) e = dev_alloc((void**)&c->d_status, 256, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) rc = fail(NDG_ENOMEM, "norm buffers: %s", cudaGetErrorString(e));
    c->desc.status = c->d_status;
  }
  if (rc == NDG_OK) {
    TileConfig t = tuned_tile(c->kc);
    if (!t.epb) t = default_tile(c->kc);
    if (k.kernel == NDG_KERNEL_LINE) t.variant = kLineKernel;
    if (k.kernel == NDG_KERNEL_LINE_VAR) t.variant = kLineVarKernel;
    if (k.kernel != NDG_KERNEL_AUTO && !k.elems_per_block) t.epb = default_epb_for(c->kc, t.variant);
    if (k.elems_per_block) t.epb = k.elems_per_block;
    t.epb = (int)std::min<long long>(t.epb, nelem);
    rc = set_group_tile(c, t);
  }
  if (rc != NDG_OK) {
    std::string msg = g_last_error;
    ndg_destroy(c);
    g_last_error = msg;
    return rc;
  }
  *out = c;
  return NDG_OK;
}

int ndg_create(int dim, int degree, const int elems[3], int equation, int flux, ndg_ctx** out) {
  if (!elems) return fail(NDG_EINVAL, "elems is NULL");
  ndg_config cfg;
  ndg_config_init(&cfg);
  cfg.dim = dim;
  cfg.degree = degree;
  for (int a = 0; a < 3; ++a) cfg.elems[a] = a < dim ? elems[a] : 1;
  cfg.equation = equation;
  cfg.flux = flux;
  return ndg_create_ex(&cfg, out);
}

int ndg_info(const ndg_ctx* c, ndg_info_t* o) {
  if (!c || !o) return fail(NDG_EINVAL, "NULL argument");
  o->nvar = c->nvar;
  o->nodes_per_elem = c->npe;
  o->nelem = c->nelem;
  o->ndof = c->ndof;
  o->state_bytes = c->state_bytes;
  o->device_bytes = c->device_bytes;
  o->elems_per_block = c->tile.epb;
  o->kernel = c->tile.variant == kLineVarKernel ? NDG_KERNEL_LINE_VAR : NDG_KERNEL_LINE;
  return NDG_OK;
}

int ndg_lgl(int degree, double* xi, double* w) {
  if (!xi || !w) return fail(NDG_EINVAL, "NULL argument");
  Basis b;
  if (degree < 1 || degree > kMaxDegree || !build_basis(degree, &b))
    return fail(NDG_EINVAL, "degree must be in 1..%d", kMaxDegree);
  for (int i = 0; i <= degree; ++i) {
    xi[i] = b.xi[i];
    w[i] = b.w[i];
  }
  return NDG_OK;
}

void* ndg_stream(const ndg_ctx* c) { return c ? (void*)c->stream : nullptr; }

int ndg_synchronize(ndg_ctx* c) {
  if (!c) return fail(NDG_EINVAL, "NULL context");
  DeviceGuard dg(c->cfg.device);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  return status_check(c->d_status);
}

static int ensure_scratch(ndg_ctx* c) {
  if (c->d_scratch) return NDG_OK;
  cudaError_t e = dev_alloc(&c->d_scratch, c->state_bytes, c->stream);
  if (e != cudaSuccess) return fail(NDG_ENOMEM, "scratch allocation failed");
  c->device_bytes += c->state_bytes;
  return NDG_OK;
}

int ndg_set_state(ndg_ctx* c, const void* src, size_t nbytes, int src_on_device, int layout) {
  if (!c || !src) return fail(NDG_EINVAL, "NULL argument");
  if (nbytes != c->state_bytes)
    return fail(NDG_EINVAL, "state size mismatch: got %zu bytes, expected %zu", nbytes, c->state_bytes);
  if (layout != NDG_LAYOUT_ELEMENT && layout != NDG_LAYOUT_GRID) return fail(NDG_EINVAL, "bad layout");
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard dg(c->cfg.device);
  cudaError_t e;
  const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (layout == NDG_LAYOUT_ELEMENT) {
    e = cudaMemcpyAsync(c->buf[kUN], src, nbytes, kind, c->stream);
  } else {
    int rc = ensure_scratch(c);
    if (rc) return rc;
    e = cudaMemcpyAsync(c->d_scratch, src, nbytes, kind, c->stream);
    if (e == cudaSuccess)
      e = (cudaError_t)launch_relayout(c->kc.dtype, c->cfg.dim, c->cfg.degree, c->nvar, c->cfg.elems,
                                       c->d_scratch, c->buf[kUN], true, c->stream);
  }
  // a new state: a flag raised by earlier steps no longer applies
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
  if (e == cudaSuccess && !src_on_device) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_state copy");
  c->have_state = true;
  c->t = 0.0;
  c->steps = 0;
  return NDG_OK;
}

int ndg_get_state(ndg_ctx* c, void* dst, size_t nbytes, int dst_on_device, int layout) {
  if (!c || !dst) return fail(NDG_EINVAL, "NULL argument");
  if (nbytes != c->state_bytes)
    return fail(NDG_EINVAL, "state size mismatch: got %zu bytes, expected %zu", nbytes, c->state_bytes);
  if (layout != NDG_LAYOUT_ELEMENT && layout != NDG_LAYOUT_GRID) return fail(NDG_EINVAL, "bad layout");
  if (!c->have_state) return fail(NDG_ESTATE, "no state has been set");
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard dg(c->cfg.device);
  cudaError_t e;
  const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (layout == NDG_LAYOUT_ELEMENT) {
    e = cudaMemcpyAsync(dst, c->buf[kUN], nbytes, kind, c->stream);
  } else {
    int rc = ensure_scratch(c);
    if (rc) return rc;
    e = (cudaError_t)launch_relayout(c->kc.dtype, c->cfg.dim, c->cfg.degree, c->nvar, c->cfg.elems,
                                     c->buf[kUN], c->d_scratch, false, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, c->d_scratch, nbytes, kind, c->stream);
  }
  if (e == cudaSuccess && !dst_on_device) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "get_state copy");
  return dst_on_device ? NDG_OK : status_check(c->d_status);
}

int ndg_step(ndg_ctx* c, double dt, int nsteps, int rk) {
  if (!c) return fail(NDG_EINVAL, "NULL context");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(NDG_EINVAL, "dt must be positive and finite");
  if (nsteps < 0) return fail(NDG_EINVAL, "nsteps must be >= 0");
  if (!valid_rk(rk)) return fail(NDG_EINVAL, "rk_scheme must be 3, 4 or 6 (got %d)", rk);
  if (!c->have_state) return fail(NDG_ESTATE, "no state has been set");
  if (nsteps == 0) return NDG_OK;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard dg(c->cfg.device);
  int rc = ensure_buffers(c, rk);
  if (rc) return rc;
  Group& g = c->group;
  bool dirty = false;
  if (g.h_desc[0].dt != dt || std::memcmp(g.h_desc[0].buf, c->desc.buf, sizeof(c->desc.buf)) != 0) {
    c->desc.dt = dt;
    g.h_desc[0] = c->desc;
    dirty = true;
  }
  if (dirty) {
    rc = group_upload(g, c->stream);
    if (rc) return rc;
  }
  cudaGraphExec_t& ge = c->graph[rk];
  if (!ge || c->graph_tile[rk].epb != c->tile.epb || c->graph_tile[rk].variant != c->tile.variant) {
    if (ge) {
      cudaGraphExecDestroy(ge);
      ge = nullptr;
    }
    std::vector<Group*> groups{&g};
    // the capture stream must see the uploaded work list: order it after the context stream
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, c->stream);
    cudaStreamWaitEvent(c->capture_stream, ev, 0);
    cudaEventDestroy(ev);
    rc = capture_step(groups, rk, c->capture_stream, &ge);
    if (rc) return rc;
    c->graph_tile[rk] = c->tile;
  }
  for (int s = 0; s < nsteps; ++s) {
    cudaError_t e = cudaGraphLaunch(ge, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  }
  c->t += dt * nsteps;
  c->steps += nsteps;
  return NDG_OK;
}

int ndg_step_split(ndg_ctx* c, double dt, int nsteps, int rk) {
  if (!c) return fail(NDG_EINVAL, "NULL context");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(NDG_EINVAL, "dt must be positive and finite");
  if (nsteps < 0) return fail(NDG_EINVAL, "nsteps must be >= 0");
  if (!valid_rk(rk)) return fail(NDG_EINVAL, "rk_scheme must be 3, 4 or 6 (got %d)", rk);
  if (c->kc.dtype == NDG_F64_FF || c->kc.mass == NDG_MASS_EXACT)
    return fail(NDG_EINVAL, "the split stage is built for NDG_F64 and NDG_F32 with the lumped mass");
  if (!c->have_state) return fail(NDG_ESTATE, "no state has been set");
  if (nsteps == 0) return NDG_OK;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard dg(c->cfg.device);
  int rc = ensure_buffers(c, rk);
  if (rc == NDG_OK) rc = ensure_scratch(c);  // the right-hand side between the kernels
  if (rc) return rc;
  SolveDesc d = c->desc;
  d.dt = dt;
  for (int s = 0; s < nsteps; ++s)
    for (const StagePlan& p : stage_plans(rk)) {
      const int e = launch_split_stage(c->kc, d, p, c->d_scratch, c->stream);
      if (e != 0) return cuda_fail((cudaError_t)e, "split stage launch");
    }
  c->t += dt * nsteps;
  c->steps += nsteps;
  return NDG_OK;
}

int ndg_norms(ndg_ctx* c, const void* ref, int ref_on_device, ndg_norms_t* out) {
  if (!c || !out) return fail(NDG_EINVAL, "NULL argument");
  if (!c->have_state) return fail(NDG_ESTATE, "no state has been set");
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard dg(c->cfg.device);
  const void* dref = ref;
  cudaError_t e = cudaSuccess;
  if (ref && !ref_on_device) {
    int rc = ensure_scratch(c);
    if (rc) return rc;
    e = cudaMemcpyAsync(c->d_scratch, ref, c->state_bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reference copy");
    dref = c->d_scratch;
  }
  double jac = 1.0;
  for (int a = 0; a < c->cfg.dim; ++a) jac *= 0.5 * c->cfg.length[a] / c->cfg.elems[a];
  e = (cudaError_t)launch_norms(c->kc.dtype, c->cfg.dim, c->cfg.degree, c->cfg.equation, c->buf[kUN],
                                dref, c->nelem, jac, c->cfg.sound_speed, c->cfg.velocity, kNormBlocks,
                                c->d_partials, c->d_result, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_result, c->d_result, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "norms");
  if (int rc = status_check(c->d_status)) return rc;
  const double* r = c->h_result;
  out->l2 = r[0];
  out->linf = r[1];
  for (int v = 0; v < 4; ++v) out->integral[v] = v < c->nvar ? r[2 + v] : 0.0;
  out->max_speed = r[6];
  out->nonfinite = (int64_t)r[7];
  out->t = c->t;
  out->steps = c->steps;
  if (out->nonfinite > 0) return fail(NDG_ENONFINITE, "state holds %lld non-finite values", (long long)out->nonfinite);
  return NDG_OK;
}

int ndg_stable_dt(ndg_ctx* c, double cfl, double* dt) {
  if (!c || !dt) return fail(NDG_EINVAL, "NULL argument");
  if (!(cfl > 0.0) || !std::isfinite(cfl)) return fail(NDG_EINVAL, "cfl must be positive");
  ndg_norms_t nr;
  int rc = ndg_norms(c, nullptr, 0, &nr);
  if (rc) return rc;
  double gap = 2.0;
  for (int k = 0; k < c->cfg.degree; ++k) gap = std::min(gap, c->basis.xi[k + 1] - c->basis.xi[k]);
  double hmin = 1e300;
  for (int a = 0; a < c->cfg.dim; ++a) hmin = std::min(hmin, 0.5 * c->cfg.length[a] / c->cfg.elems[a] * gap);
  if (!(nr.max_speed > 0.0)) return fail(NDG_EINVAL, "zero wave speed: no CFL limit");
  *dt = cfl * hmin / nr.max_speed;
  return NDG_OK;
}

int ndg_node_coords(ndg_ctx* c, double* X, size_t count) {
  if (!c || !X) return fail(NDG_EINVAL, "NULL argument");
  const size_t need = (size_t)c->cfg.dim * c->nelem * c->npe;
  if (count != need) return fail(NDG_EINVAL, "coords need %zu doubles, got %zu", need, count);
  const int n = c->n;
  const int E0 = c->cfg.elems[0], E1 = c->cfg.elems[1];
  for (int a = 0; a < c->cfg.dim; ++a) {
    const double h = c->cfg.length[a] / c->cfg.elems[a];
    for (long long e = 0; e < c->nelem; ++e) {
      const long long ei[3] = {e % E0, (e / E0) % E1, e / ((long long)E0 * E1)};
      for (int node = 0; node < c->npe; ++node) {
        const int ii[3] = {node % n, (node / n) % n, node / (n * n)};
        X[((size_t)a * c->nelem + e) * c->npe + node] = ei[a] * h + 0.5 * h * (c->basis.xi[ii[a]] + 1.0);
      }
    }
  }
  return NDG_OK;
}

int ndg_debug_stall_copies(int polls) {
  if (polls < 0) return fail(NDG_EINVAL, "polls must be >= 0");
  g_debug_wait_polls.store(polls);
  return NDG_OK;
}

int ndg_autotune(ndg_ctx* c, int rk, int* best_epb, double* best_ms) {
  if (!c) return fail(NDG_EINVAL, "NULL context");
  if (!valid_rk(rk)) return fail(NDG_EINVAL, "bad rk scheme");
  if (!c->have_state) return fail(NDG_ESTATE, "no state has been set");
  DeviceGuard dg(c->cfg.device);
  int rc = ensure_buffers(c, rk);
  if (rc) return rc;
  // save the state, time candidates on a few steps each, restore
  void* save = nullptr;
  cudaError_t e = dev_alloc(&save, c->state_bytes, c->stream);
  if (e != cudaSuccess) return fail(NDG_ENOMEM, "autotune needs one state-sized buffer");
  cudaMemcpyAsync(save, c->buf[kUN], c->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
  const double t0 = c->t;
  const long long s0 = c->steps;
  // a tiny step keeps the state bounded while timing
  double dt = 1e-6;
  const int cands[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64};
  TileConfig best = c->tile;
  double best_t = 1e300;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const TileConfig orig = c->tile;
  for (int variant : {kLineKernel, kLineVarKernel}) {
    if (c->cfg.kernel == NDG_KERNEL_LINE && variant != kLineKernel) continue;
    if (c->cfg.kernel == NDG_KERNEL_LINE_VAR && variant != kLineVarKernel) continue;
    if (variant == kLineVarKernel && c->nvar == 1) continue;  // same kernel as kLineKernel
    for (int epb : cands) {
      if (epb > c->nelem) break;
      int threads;
      size_t smem;
      stage_launch_shape(c->kc, variant, epb, &threads, &smem);
      if (threads > 1024 || threads < 32 || smem > 220 * 1024) continue;
      {
        std::lock_guard<std::mutex> lk(c->mu);
        if (set_group_tile(c, TileConfig{epb, variant}) != NDG_OK) continue;
      }
      const long long dofs = c->ndof;
      const int reps = (int)std::max<long long>(2, std::min<long long>(50, 400000000LL / std::max<long long>(1, dofs)));
      if (ndg_step(c, dt, 1, rk) != NDG_OK) continue;  // warm-up + capture
      cudaEventRecord(a, c->stream);
      ndg_step(c, dt, reps, rk);
      cudaEventRecord(b, c->stream);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      const double per = ms / reps;
      if (per < best_t) {
        best_t = per;
        best = TileConfig{epb, variant};
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  {
    std::lock_guard<std::mutex> lk(c->mu);
    rc = set_group_tile(c, best.epb ? best : orig);
    cudaMemcpyAsync(c->buf[kUN], save, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
    cudaStreamSynchronize(c->stream);
  }
  dev_free(save, c->stream);
  c->t = t0;
  c->steps = s0;
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_tune_cache_locked();
    g_tuned[class_key(c->kc)] = best;
    save_tune_cache_locked();
  }
  if (best_epb) *best_epb = best.epb;
  if (best_ms) *best_ms = best_t;
  return NDG_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// batching
// ------------------------------------------------------------------------------------------
struct ndg_batch {
  std::vector<ndg_ctx*> ctxs;
  std::vector<Group> groups;
  std::vector<std::vector<int>> members;  // context indices per group
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  int device = 0;
  cudaGraphExec_t graph[7] = {nullptr};
  std::vector<double> last_dt;
};

namespace ndg {

int batch_rebuild(ndg_batch* b, const double* dts, int rk) {
  bool changed = false;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    Group& g = b->groups[gi];
    int tile = 0;
    g.h_desc.clear();
    for (int idx : b->members[gi]) {
      ndg_ctx* c = b->ctxs[idx];
      int rc = ensure_buffers(c, rk);
      if (rc) return rc;
      SolveDesc d = c->desc;
      d.dt = dts[idx];
      d.tile_begin = tile;
      tile += (int)((c->nelem + g.epb - 1) / g.epb);
      g.h_desc.push_back(d);
      if (b->last_dt[idx] != dts[idx]) changed = true;
    }
    g.ntiles = tile;
  }
  (void)changed;
  for (Group& g : b->groups) {
    int rc = group_upload(g, b->stream);
    if (rc) return rc;
  }
  for (size_t i = 0; i < b->ctxs.size(); ++i) b->last_dt[i] = dts[i];
  return NDG_OK;
}

}  // namespace ndg

extern "C" {

int ndg_batch_create(ndg_ctx* const* ctxs, int n, ndg_batch** out) {
  if (!ctxs || n < 1 || !out) return fail(NDG_EINVAL, "need at least one context");
  ndg_batch* b = new ndg_batch();
  b->device = ctxs[0]->cfg.device;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) {
      delete b;
      return fail(NDG_EINVAL, "context %d is NULL", i);
    }
    if (ctxs[i]->cfg.device != b->device) {
      delete b;
      return fail(NDG_EINVAL, "all contexts of a batch must be on one device");
    }
    b->ctxs.push_back(ctxs[i]);
  }
  DeviceGuard dg(b->device);
  b->stream = ctxs[0]->stream;
  cudaError_t e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "stream create");
  }
  // group by kernel class; each class uses the largest tuned/default tile that fits
  for (int i = 0; i < n; ++i) {
    const KernelClass& kc = ctxs[i]->kc;
    size_t gi = 0;
    for (; gi < b->groups.size(); ++gi)
      if (b->groups[gi].kc == kc && b->groups[gi].variant == ctxs[i]->tile.variant) break;
    if (gi == b->groups.size()) {
      Group g;
      g.kc = kc;
      g.epb = ctxs[i]->tile.epb;
      g.variant = ctxs[i]->tile.variant;
      b->groups.push_back(g);
      b->members.push_back({});
    }
    b->members[gi].push_back(i);
  }
  for (Group& g : b->groups) {
    int maxb = 0;
    int pe = prepare_stage_kernel(g.kc, g.variant, g.epb, &maxb);
    if (pe != 0 || maxb < 1) {
      ndg_batch_destroy(b);
      return fail(NDG_EINVAL, "tile does not fit");
    }
    g.grid = maxb * num_sms(b->device);
  }
  b->last_dt.assign(n, -1.0);
  *out = b;
  return NDG_OK;
}

int ndg_batch_step(ndg_batch* b, const double* dts, int nsteps, int rk) {
  if (!b || !dts) return fail(NDG_EINVAL, "NULL argument");
  if (!valid_rk(rk)) return fail(NDG_EINVAL, "bad rk scheme");
  if (nsteps < 0) return fail(NDG_EINVAL, "nsteps must be >= 0");
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    if (!(dts[i] > 0.0) || !std::isfinite(dts[i])) return fail(NDG_EINVAL, "dt[%zu] invalid", i);
    if (!b->ctxs[i]->have_state) return fail(NDG_ESTATE, "context %zu has no state", i);
  }
  if (nsteps == 0) return NDG_OK;
  DeviceGuard dg(b->device);
  // the contexts' own streams may hold pending work (set_state): order the batch after them
  for (ndg_ctx* c : b->ctxs)
    if (c->stream != b->stream) {
      cudaEvent_t ev;
      cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      cudaEventRecord(ev, c->stream);
      cudaStreamWaitEvent(b->stream, ev, 0);
      cudaEventDestroy(ev);
    }
  int rc = batch_rebuild(b, dts, rk);
  if (rc) return rc;
  if (!b->graph[rk]) {
    std::vector<Group*> gs;
    for (Group& g : b->groups) gs.push_back(&g);
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, b->stream);
    cudaStreamWaitEvent(b->capture_stream, ev, 0);
    cudaEventDestroy(ev);
    rc = capture_step(gs, rk, b->capture_stream, &b->graph[rk]);
    if (rc) return rc;
  }
  for (int s = 0; s < nsteps; ++s) {
    cudaError_t e = cudaGraphLaunch(b->graph[rk], b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  }
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    ndg_ctx* c = b->ctxs[i];
    c->t += dts[i] * nsteps;
    c->steps += nsteps;
    if (c->stream != b->stream) {  // later work on the context's stream sees the batch's result
      cudaEvent_t ev;
      cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      cudaEventRecord(ev, b->stream);
      cudaStreamWaitEvent(c->stream, ev, 0);
      cudaEventDestroy(ev);
    }
  }
  return NDG_OK;
}

int ndg_batch_destroy(ndg_batch* b) {
  if (!b) return NDG_OK;
  DeviceGuard dg(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int i = 0; i < 7; ++i)
    if (b->graph[i]) cudaGraphExecDestroy(b->graph[i]);
  for (Group& g : b->groups) group_free(g, b->stream);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  delete b;
  return NDG_OK;
}

}  // extern "C"
