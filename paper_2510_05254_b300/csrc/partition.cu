// Domain decomposition with a face-trace halo exchange, emulated with P partitions on one GPU.
//
// The paper distributes the element grid over rectangular/cuboid subdomains and exchanges the
// border values with non-blocking MPI every RK sub-step (Sec. 3.2).  Here every partition is a
// solve of its own (own arrays), and before every stage a pack kernel writes each partition's
// boundary traces -- the n^(d-1) face values per boundary element and variable -- into the halo
// buffers of its neighbours; the stage kernel reads a partition-boundary neighbour's trace from
// the halo instead of wrapping around.  On one GPU the pack writes the neighbour's halo directly;
// with several GPUs the same buffers would be the send/receive buffers of a peer copy or NCCL
// send/recv.  The arithmetic is unchanged, so results are bitwise those of the unpartitioned
// solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ndg.h"
#include "ndg_host.h"
#include "ndg_internal.h"

using namespace ndg;

namespace {

// One face of one partition: its boundary traces go to one halo buffer of a neighbour.
struct PackItem {
  int src;         // source partition (index into the descriptor array)
  int axis;
  int side;        // 0: low boundary (node 0 along axis), 1: high boundary (node N)
  int pad;
  void* dst;       // neighbour's halo buffer, layout [v][te][face node]
  long long begin; // first value of this item in the launch's flat numbering
  long long count; // nvar * transverse elements * n^(dim-1)
};

template <typename real>
__global__ void pack_traces(const SolveDesc* parts, const PackItem* items, int nitems, long long total,
                            int role, int dim, int n, int nvar) {
  int npe = 1, L = 1;
  for (int d = 0; d < dim; ++d) npe *= n;
  for (int d = 1; d < dim; ++d) L *= n;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].begin <= q) lo = mid; else hi = mid - 1;
    }
    const PackItem& it = items[lo];
    const SolveDesc& sd = parts[it.src];
    const long long r = q - it.begin;
    const long long te_count = it.count / ((long long)nvar * L);
    const int f = (int)(r % L);
    const long long te = (r / L) % te_count;
    const int v = (int)(r / ((long long)L * te_count));
    const int a = it.axis;
    const long long E0 = sd.E[0], E1 = sd.E[1];
    const long long Ea = sd.E[a];
    const long long ca = it.side == 0 ? 0 : Ea - 1;
    const int ia = it.side == 0 ? 0 : n - 1;
    long long e;
    int node;
    if (a == 0) {
      e = ca + E0 * te;
      node = ia + n * f;
    } else if (a == 1) {
      e = te % E0 + E0 * (ca + E1 * (te / E0));
      node = f % n + n * ia + n * n * (f / n);
    } else {
      e = te + E0 * E1 * ca;
      node = f + n * n * ia;
    }
    const real* src = static_cast<const real*>(sd.buf[role]);
    static_cast<real*>(it.dst)[r] = src[(long long)v * sd.nelem * npe + e * npe + node];
  }
}

// Copy between the global element-layout array and one partition's (to_part: global -> part).
template <typename real>
__global__ void subbox_copy(real* __restrict__ global, real* __restrict__ part, int to_part, int npe, int nvar,
                            int GE0, int GE1, int GE2, int o0, int o1, int o2, int PE0, int PE1, int PE2) {
  const long long pn = (long long)PE0 * PE1 * PE2;
  const long long gn = (long long)GE0 * GE1 * GE2;
  const long long total = pn * npe * nvar;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int node = (int)(q % npe);
    const long long e = (q / npe) % pn;
    const long long v = q / (npe * pn);
    const long long lx = e % PE0, ly = (e / PE0) % PE1, lz = e / ((long long)PE0 * PE1);
    const long long ge = (o0 + lx) + GE0 * ((o1 + ly) + (long long)GE1 * (o2 + lz));
    const long long gq = (v * gn + ge) * npe + node;
    if (to_part) part[q] = global[gq];
    else global[gq] = part[q];
  }
  (void)GE2;
}

}  // namespace

struct ndg_partition {
  ndg_config global{};
  int parts[3] = {1, 1, 1};
  int nparts = 0;
  int n = 0, npe = 0, nvar = 0;
  size_t esize = 0, global_bytes = 0;
  std::vector<ndg_ctx*> ctx;            // one solve per partition
  std::vector<int> off;                 // 3 offsets per partition (element coordinates)
  std::vector<int> cnt;                 // 3 element counts per partition
  std::vector<void*> halos;             // device buffers
  Group group;                          // the partitions as one launch group
  std::vector<PackItem> h_items;
  PackItem* d_items = nullptr;
  long long pack_total = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph[7] = {nullptr};
  void* d_global = nullptr;             // global-layout staging for set/get state
  double t = 0.0;
  long long steps = 0;
  bool have_state = false;
};

namespace {

int part_index(const ndg_partition* P, int px, int py, int pz) {
  return px + P->parts[0] * (py + P->parts[1] * pz);
}

void split(int E, int P, int p, int* off, int* cnt) {
  const int base = E / P, extra = E % P;
  *cnt = base + (p < extra ? 1 : 0);
  *off = p * base + std::min(p, extra);
}

int launch_pack(ndg_partition* P, int role, cudaStream_t s) {
  if (P->pack_total == 0) return NDG_OK;
  long long blocks = (P->pack_total + 255) / 256;
  blocks = std::min<long long>(blocks, 148 * 8);
  if (dtype_bytes(P->global.dtype) == 8)
    pack_traces<double><<<(int)blocks, 256, 0, s>>>(P->group.d_desc, P->d_items, (int)P->h_items.size(),
                                                     P->pack_total, role, P->global.dim, P->n, P->nvar);
  else
    pack_traces<float><<<(int)blocks, 256, 0, s>>>(P->group.d_desc, P->d_items, (int)P->h_items.size(),
                                                    P->pack_total, role, P->global.dim, P->n, P->nvar);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NDG_OK : cuda_fail(e, "pack launch");
}

int copy_parts(ndg_partition* P, bool to_part) {
  for (int p = 0; p < P->nparts; ++p) {
    const long long total = (long long)P->cnt[3 * p] * P->cnt[3 * p + 1] * P->cnt[3 * p + 2] * P->npe * P->nvar;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 148 * 8);
    void* part = P->group.h_desc[p].buf[kUN];
    const int* o = &P->off[3 * p];
    const int* c = &P->cnt[3 * p];
    if (dtype_bytes(P->global.dtype) == 8)
      subbox_copy<double><<<blocks, 256, 0, P->stream>>>((double*)P->d_global, (double*)part, to_part, P->npe,
                                                         P->nvar, P->global.elems[0], P->global.elems[1],
                                                         P->global.elems[2], o[0], o[1], o[2], c[0], c[1], c[2]);
    else
      subbox_copy<float><<<blocks, 256, 0, P->stream>>>((float*)P->d_global, (float*)part, to_part, P->npe,
                                                        P->nvar, P->global.elems[0], P->global.elems[1],
                                                        P->global.elems[2], o[0], o[1], o[2], c[0], c[1], c[2]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sub-box copy");
  }
  return NDG_OK;
}

}  // namespace

extern "C" {

int ndg_partition_create(const ndg_config* gcfg, const int parts[3], ndg_partition** out) {
  if (!gcfg || !parts || !out) return fail(NDG_EINVAL, "NULL argument");
  int rc = check_config(*gcfg);
  if (rc) return rc;
  ndg_partition* P = new ndg_partition();
  P->global = *gcfg;
  for (int a = gcfg->dim; a < 3; ++a) P->global.elems[a] = 1;
  P->nparts = 1;
  for (int a = 0; a < 3; ++a) {
    P->parts[a] = a < gcfg->dim ? parts[a] : 1;
    if (P->parts[a] < 1 || P->parts[a] > P->global.elems[a]) {
      delete P;
      return fail(NDG_EINVAL, "parts[%d] must be in 1..elems[%d]", a, a);
    }
    P->nparts *= P->parts[a];
  }
  P->n = gcfg->degree + 1;
  P->npe = 1;
  for (int a = 0; a < gcfg->dim; ++a) P->npe *= P->n;
  P->nvar = gcfg->equation == NDG_ADVECTION ? 1 : gcfg->dim + 1;
  P->esize = dtype_bytes(gcfg->dtype);
  long long gel = (long long)P->global.elems[0] * P->global.elems[1] * P->global.elems[2];
  P->global_bytes = (size_t)gel * P->npe * P->nvar * P->esize;
  cudaSetDevice(gcfg->device);
  cudaError_t e = cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete P;
    return cuda_fail(e, "partition streams");
  }
  // one solve per partition, on the partition's stream
  for (int pz = 0; pz < P->parts[2]; ++pz)
    for (int py = 0; py < P->parts[1]; ++py)
      for (int px = 0; px < P->parts[0]; ++px) {
        int o[3], c[3];
        const int pp[3] = {px, py, pz};
        ndg_config lc = P->global;
        for (int a = 0; a < 3; ++a) {
          split(P->global.elems[a], P->parts[a], pp[a], &o[a], &c[a]);
          lc.elems[a] = c[a];
          if (a < gcfg->dim) lc.length[a] = gcfg->length[a] * c[a] / P->global.elems[a];
        }
        lc.stream = P->stream;
        ndg_ctx* cx = nullptr;
        rc = ndg_create_ex(&lc, &cx);
        if (rc) {
          std::string m = ndg_last_error();
          ndg_partition_destroy(P);
          return fail(rc, "partition create: %s", m.c_str());
        }
        P->ctx.push_back(cx);
        for (int a = 0; a < 3; ++a) {
          P->off.push_back(o[a]);
          P->cnt.push_back(c[a]);
        }
      }
  // the partitions' descriptors as one group, with halo buffers on every partition boundary
  ndg_info_t info;
  ndg_info(P->ctx[0], &info);
  P->group.kc = KernelClass{gcfg->dim, gcfg->degree, gcfg->equation, gcfg->dtype, gcfg->mass};
  P->group.epb = info.elems_per_block;
  P->group.variant = info.kernel == NDG_KERNEL_LINE_VAR ? kLineVarKernel : kLineKernel;
  int L = 1;
  for (int a = 1; a < gcfg->dim; ++a) L *= P->n;
  // the coefficients depend only on the element size, velocity and c: take them from the global
  // problem, so that a partition's (length * count / E) / count rounding cannot change a bit
  SolveDesc gd;
  std::memset(&gd, 0, sizeof(gd));
  {
    Basis b;
    build_basis(gcfg->degree, &b);
    fill_solve_geometry(P->global, b, &gd);
  }
  int tile = 0;
  for (int p = 0; p < P->nparts; ++p) {
    SolveDesc d = ndg_ctx_desc(P->ctx[p]);
    d.rhs_scale = gd.rhs_scale;
    for (int a = 0; a < 3; ++a) {
      d.vol_scale[a] = gd.vol_scale[a];
      d.lift_lo[a] = gd.lift_lo[a];
      d.lift_hi[a] = gd.lift_hi[a];
      d.f_vol_scale[a] = gd.f_vol_scale[a];
      d.f_lift_lo[a] = gd.f_lift_lo[a];
      d.f_lift_hi[a] = gd.f_lift_hi[a];
    }
    d.c = gd.c;
    d.c2 = gd.c2;
    d.f_c = gd.f_c;
    d.f_c2 = gd.f_c2;
    d.tile_begin = tile;
    tile += (int)((d.nelem + P->group.epb - 1) / P->group.epb);
    P->group.h_desc.push_back(d);
  }
  P->group.ntiles = tile;
  const int pz_n = P->parts[2], py_n = P->parts[1], px_n = P->parts[0];
  for (int p = 0; p < P->nparts; ++p) {
    const int pp[3] = {p % px_n, (p / px_n) % py_n, p / (px_n * py_n)};
    SolveDesc& d = P->group.h_desc[p];
    for (int a = 0; a < gcfg->dim; ++a) {
      if (P->parts[a] == 1) continue;  // this axis is not cut: periodic wrap inside the solve
      const long long te = d.nelem / d.E[a];
      const size_t bytes = (size_t)P->nvar * te * L * P->esize;
      for (int side = 0; side < 2; ++side) {
        void* h = nullptr;
        e = dev_alloc(&h, bytes, P->stream);
        if (e != cudaSuccess) {
          ndg_partition_destroy(P);
          return fail(NDG_ENOMEM, "halo allocation failed");
        }
        P->halos.push_back(h);
        if (side == 0) d.halo_lo[a] = h; else d.halo_hi[a] = h;
        // who fills it: the neighbour across this side sends its opposite boundary
        int q[3] = {pp[0], pp[1], pp[2]};
        q[a] = side == 0 ? (pp[a] + P->parts[a] - 1) % P->parts[a] : (pp[a] + 1) % P->parts[a];
        PackItem it{};
        it.src = part_index(P, q[0], q[1], q[2]);
        it.axis = a;
        it.side = side == 0 ? 1 : 0;  // low halo holds the low neighbour's high boundary
        it.dst = h;
        it.count = (long long)P->nvar * te * L;
        it.begin = P->pack_total;
        P->pack_total += it.count;
        P->h_items.push_back(it);
      }
    }
  }
  (void)pz_n;
  int maxb = 0;
  int pe = prepare_stage_kernel(P->group.kc, P->group.variant, P->group.epb, &maxb);
  if (pe != 0 || maxb < 1) {
    ndg_partition_destroy(P);
    return fail(NDG_EINVAL, "stage kernel does not fit");
  }
  P->group.grid = maxb * num_sms(gcfg->device);
  rc = group_upload(P->group, P->stream);
  if (rc == NDG_OK && !P->h_items.empty()) {
    e = dev_alloc((void**)&P->d_items, P->h_items.size() * sizeof(PackItem), P->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(P->d_items, P->h_items.data(), P->h_items.size() * sizeof(PackItem),
                          cudaMemcpyHostToDevice, P->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "pack list");
  }
  if (rc == NDG_OK) {
    e = dev_alloc(&P->d_global, P->global_bytes, P->stream);
    if (e != cudaSuccess) rc = fail(NDG_ENOMEM, "global staging allocation failed");
  }
  if (rc) {
    std::string m = ndg_last_error();
    ndg_partition_destroy(P);
    return fail(rc, "%s", m.c_str());
  }
  *out = P;
  return NDG_OK;
}

int ndg_partition_set_state(ndg_partition* P, const void* src, size_t nbytes, int src_on_device) {
  if (!P || !src) return fail(NDG_EINVAL, "NULL argument");
  if (nbytes != P->global_bytes) return fail(NDG_EINVAL, "state size mismatch");
  cudaSetDevice(P->global.device);
  cudaError_t e = cudaMemcpyAsync(P->d_global, src, nbytes,
                                  src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, P->stream);
  if (e != cudaSuccess) return cuda_fail(e, "state copy");
  int rc = copy_parts(P, true);
  if (rc) return rc;
  // a new state: flags raised by earlier steps no longer apply
  for (ndg_ctx* c : P->ctx) ndg_ctx_mark_state(c, P->stream);
  e = cudaMemsetAsync(&P->group.d_hdr->err, 0, sizeof(int), P->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) return cuda_fail(e, "state copy");
  P->have_state = true;
  P->t = 0.0;
  P->steps = 0;
  return NDG_OK;
}

int ndg_partition_get_state(ndg_partition* P, void* dst, size_t nbytes, int dst_on_device) {
  if (!P || !dst) return fail(NDG_EINVAL, "NULL argument");
  if (nbytes != P->global_bytes) return fail(NDG_EINVAL, "state size mismatch");
  if (!P->have_state) return fail(NDG_ESTATE, "no state has been set");
  cudaSetDevice(P->global.device);
  int rc = copy_parts(P, false);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(dst, P->d_global, nbytes,
                                  dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, P->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) return cuda_fail(e, "state copy");
  return group_check(P->group);
}

int ndg_partition_step(ndg_partition* P, double dt, int nsteps, int rk) {
  if (!P) return fail(NDG_EINVAL, "NULL argument");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(NDG_EINVAL, "dt must be positive and finite");
  if (!valid_rk(rk)) return fail(NDG_EINVAL, "bad rk scheme");
  if (nsteps < 0) return fail(NDG_EINVAL, "nsteps must be >= 0");
  if (!P->have_state) return fail(NDG_ESTATE, "no state has been set");
  if (nsteps == 0) return NDG_OK;
  cudaSetDevice(P->global.device);
  bool changed = false;
  for (int p = 0; p < P->nparts; ++p) {
    int rc = ndg_ctx_ensure_buffers(P->ctx[p], rk);
    if (rc) return rc;
    SolveDesc fresh = ndg_ctx_desc(P->ctx[p]);
    SolveDesc& d = P->group.h_desc[p];
    if (d.dt != dt || std::memcmp(d.buf, fresh.buf, sizeof(d.buf)) != 0) {
      std::memcpy(d.buf, fresh.buf, sizeof(d.buf));
      d.dt = dt;
      changed = true;
    }
  }
  if (changed) {
    int rc = group_upload(P->group, P->stream);
    if (rc) return rc;
  }
  if (!P->graph[rk]) {
    // one RK step: for every stage, the exchange of the stage input's traces, then the stage
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, P->stream);
    cudaStreamWaitEvent(P->cap, ev, 0);
    cudaEventDestroy(ev);
    cudaError_t e = cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    int rc = NDG_OK;
    for (const StagePlan& sp : stage_plans(rk)) {
      if (rc == NDG_OK) rc = launch_pack(P, sp.in, P->cap);
      int le = launch_stage(P->group.kc, P->group.variant, std::max(1, P->group.grid), P->group.epb, P->group.d_desc,
                            P->group.d_hdr, sp, P->cap);
      if (le && rc == NDG_OK) rc = cuda_fail((cudaError_t)le, "stage launch");
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(P->cap, &g);
    if (e != cudaSuccess && rc == NDG_OK) rc = cuda_fail(e, "end capture");
    if (rc == NDG_OK) {
      e = cudaGraphInstantiate(&P->graph[rk], g, 0);
      if (e != cudaSuccess) rc = cuda_fail(e, "graph instantiate");
    }
    if (g) cudaGraphDestroy(g);
    if (rc) return rc;
  }
  for (int s = 0; s < nsteps; ++s) {
    cudaError_t e = cudaGraphLaunch(P->graph[rk], P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  }
  P->t += dt * nsteps;
  P->steps += nsteps;
  return NDG_OK;
}

int ndg_partition_norms(ndg_partition* P, ndg_norms_t* out) {
  if (!P || !out) return fail(NDG_EINVAL, "NULL argument");
  if (!P->have_state) return fail(NDG_ESTATE, "no state has been set");
  std::memset(out, 0, sizeof(*out));
  double l2sq = 0.0;
  int status = NDG_OK;
  for (ndg_ctx* c : P->ctx) {  // partitions in a fixed order: deterministic
    ndg_norms_t r;
    int rc = ndg_norms(c, nullptr, 0, &r);
    if (rc != NDG_OK && rc != NDG_ENONFINITE) return rc;
    if (rc == NDG_ENONFINITE) status = rc;
    l2sq += r.l2 * r.l2;
    out->linf = std::max(out->linf, r.linf);
    for (int v = 0; v < 4; ++v) out->integral[v] += r.integral[v];
    out->max_speed = std::max(out->max_speed, r.max_speed);
    out->nonfinite += r.nonfinite;
  }
  if (int rc = group_check(P->group)) return rc;
  out->l2 = std::sqrt(l2sq);
  out->t = P->t;
  out->steps = P->steps;
  return status == NDG_OK ? NDG_OK : fail(status, "state holds non-finite values");
}

int ndg_partition_info(const ndg_partition* P, int part, int offset[3], int elems[3]) {
  if (!P || !offset || !elems) return fail(NDG_EINVAL, "NULL argument");
  if (part < 0 || part >= P->nparts) return fail(NDG_EINVAL, "no partition %d", part);
  for (int a = 0; a < 3; ++a) {
    offset[a] = P->off[3 * part + a];
    elems[a] = P->cnt[3 * part + a];
  }
  return NDG_OK;
}

int ndg_partition_destroy(ndg_partition* P) {
  if (!P) return NDG_OK;
  cudaSetDevice(P->global.device);
  if (P->stream) cudaStreamSynchronize(P->stream);
  for (int i = 0; i < 7; ++i)
    if (P->graph[i]) cudaGraphExecDestroy(P->graph[i]);
  for (void* h : P->halos) dev_free(h, P->stream);
  dev_free(P->d_items, P->stream);
  dev_free(P->d_global, P->stream);
  group_free(P->group, P->stream);
  for (ndg_ctx* c : P->ctx) ndg_destroy(c);
  if (P->cap) cudaStreamDestroy(P->cap);
  if (P->stream) cudaStreamDestroy(P->stream);
  delete P;
  return NDG_OK;
}

}  // extern "C"
