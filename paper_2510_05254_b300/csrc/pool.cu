// Serving pool: continuous batching of independent solves under a device-memory budget.
//
// Three host threads cooperate:
//   - callers: ndg_pool_submit copies the initial state into host memory and queues the solve;
//   - the worker: admits queued solves first-in first-out while the budget allows, and steps
//     every running solve together, one CUDA-graph replay per RK step.  Solves of one kernel
//     class (dim, degree, equation, dtype, mass matrix, RK scheme) share one persistent stage launch per
//     stage; classes are parallel branches of the graph.  The graph reads its work lists from
//     device memory, so solves join and leave at step boundaries by rewriting those lists; it
//     is captured again only when a class first appears or a list outgrows its capacity;
//   - the io thread: uploads admitted solves' initial states and downloads finished results on
//     its own stream, so the worker never blocks on a host copy.
// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync): admitting and retiring a
// solve does not synchronise the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <cmath>
#include <thread>
#include <vector>

#include "ndg_host.h"
#include "ndg_internal.h"

using namespace ndg;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum SolveState { kQueued, kUploading, kReady, kRunning, kRetiring, kDone };

struct PoolSolve {
  uint64_t ticket = 0;
  ndg_config cfg{};
  KernelClass kc{};
  int rk = 4;
  double dt = 0.0;
  int nsteps = 0;
  int steps_done = 0;
  size_t state_bytes = 0;
  size_t need = 0;  // device bytes while admitted
  std::vector<char> host;  // initial state, then the result
  void* buf[kNumRoles] = {nullptr};
  int* d_status = nullptr;  // set by a stage kernel whose bulk-copy wait ran out (SolveDesc::status)
  int h_status = 0;         // its value, read back when the solve retires
  SolveDesc desc{};
  SolveState state = kQueued;
  cudaEvent_t ev = nullptr;  // upload done / last step done
  double submit_s = 0, admit_s = 0, done_s = 0;
};

long long pool_class_key(const KernelClass& k, int rk) {
  return (((((long long)k.dim * 16 + k.degree) * 2 + k.equation) * 4 + k.dtype) * 2 + k.mass) * 8 + rk;
}

struct PoolClass {
  Group group;
  int rk = 4;
  std::vector<PoolSolve*> members;
};

}  // namespace

struct ndg_pool {
  size_t budget = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work;  // worker: new submissions / uploads done / memory freed
  std::condition_variable cv_io;    // io thread: new tasks
  std::condition_variable cv_done;  // pollers
  std::deque<PoolSolve*> queue;
  std::deque<PoolSolve*> io_tasks;
  std::map<uint64_t, std::unique_ptr<PoolSolve>> solves;
  std::vector<PoolSolve*> running;
  uint64_t next_ticket = 1;
  size_t in_use = 0, peak = 0;
  int64_t finished = 0;
  bool stop = false;
  std::thread worker, io;
  cudaStream_t stream = nullptr;     // compute
  cudaStream_t io_stream = nullptr;  // uploads / downloads
  cudaStream_t cap_stream = nullptr;
  std::string worker_error;
  // batching state (worker thread only)
  std::map<long long, PoolClass> classes;
  cudaGraphExec_t graph = nullptr;
  bool graph_dirty = true;
  std::deque<cudaEvent_t> inflight;  // events of launched steps (bounded look-ahead)
};

namespace {

// Worker: rebuild the work lists of every class from the running set.
int rebuild_lists(ndg_pool* p) {
  for (auto& kv : p->classes) {
    kv.second.members.clear();
    kv.second.group.h_desc.clear();
    kv.second.group.ntiles = 0;
  }
  for (PoolSolve* s : p->running) {
    const long long key = pool_class_key(s->kc, s->rk);
    auto it = p->classes.find(key);
    if (it == p->classes.end()) {
      PoolClass pc;
      pc.rk = s->rk;
      pc.group.kc = s->kc;
      TileConfig t = tuned_tile(s->kc);
      if (!t.epb) t = default_tile(s->kc);
      int maxb = 0;
      int e = prepare_stage_kernel(s->kc, t.variant, t.epb, &maxb);
      if (e != 0 || maxb < 1) return fail(NDG_ECUDA, "stage kernel does not fit");
      pc.group.epb = t.epb;
      pc.group.variant = t.variant;
      pc.group.grid = maxb * num_sms(p->device);
      it = p->classes.emplace(key, std::move(pc)).first;
      p->graph_dirty = true;
    }
    PoolClass& pc = it->second;
    SolveDesc d = s->desc;
    d.tile_begin = pc.group.ntiles;
    pc.group.ntiles += (int)((d.nelem + pc.group.epb - 1) / pc.group.epb);
    pc.group.h_desc.push_back(d);
    pc.members.push_back(s);
  }
  for (auto& kv : p->classes) {
    Group& g = kv.second.group;
    const size_t before = g.cap;
    const void* before_ptr = g.d_desc;
    if (g.h_desc.size() > g.cap) {
      // grow geometrically so that membership changes rarely force a new graph
      std::vector<SolveDesc> keep = g.h_desc;
      g.h_desc.resize(std::max<size_t>(g.h_desc.size(), 2 * g.cap + 8));
      int rc = group_upload(g, p->stream);  // reallocates with the larger capacity
      g.h_desc = keep;
      if (rc) return rc;
    }
    int rc = group_upload(g, p->stream);
    if (rc) return rc;
    if (g.cap != before || g.d_desc != before_ptr) p->graph_dirty = true;
  }
  return NDG_OK;
}

int launch_step(ndg_pool* p) {
  if (p->graph_dirty) {
    if (p->graph) {
      cudaGraphExecDestroy(p->graph);
      p->graph = nullptr;
    }
    // one graph over every class seen so far; classes with an empty list exit immediately.
    // Classes with different RK schemes get their own stage sequences as parallel branches.
    std::map<int, std::vector<Group*>> by_rk;
    for (auto& kv : p->classes) by_rk[kv.second.rk].push_back(&kv.second.group);
    cudaGraph_t whole = nullptr;
    cudaError_t e = cudaGraphCreate(&whole, 0);
    if (e != cudaSuccess) return cuda_fail(e, "graph create");
    for (auto& kv : by_rk) {
      cudaGraphExec_t part = nullptr;
      cudaEvent_t ev;
      cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      cudaEventRecord(ev, p->stream);
      cudaStreamWaitEvent(p->cap_stream, ev, 0);
      cudaEventDestroy(ev);
      // capture this scheme's classes into a child graph of the step graph
      cudaGraph_t g = nullptr;
      cudaError_t ce = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (ce != cudaSuccess) return cuda_fail(ce, "begin capture");
      const auto& plans = stage_plans(kv.first);
      std::vector<cudaStream_t> side(kv.second.size());
      std::vector<cudaEvent_t> evs(kv.second.size() + 1);
      for (auto& x : evs) cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
      for (auto& s : side) cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
      cudaEventRecord(evs.back(), p->cap_stream);
      int rc = NDG_OK;
      for (size_t i = 0; i < kv.second.size(); ++i) {
        Group* gr = kv.second[i];
        cudaStreamWaitEvent(side[i], evs.back(), 0);
        for (const StagePlan& sp : plans) {
          int le = launch_stage(gr->kc, gr->variant, std::max(1, gr->grid), gr->epb, gr->d_desc, gr->d_hdr, sp,
                                side[i]);
          if (le && rc == NDG_OK) rc = cuda_fail((cudaError_t)le, "stage launch");
        }
        cudaEventRecord(evs[i], side[i]);
        cudaStreamWaitEvent(p->cap_stream, evs[i], 0);
      }
      ce = cudaStreamEndCapture(p->cap_stream, &g);
      for (auto& x : evs) cudaEventDestroy(x);
      for (auto& s : side) cudaStreamDestroy(s);
      if (ce != cudaSuccess && rc == NDG_OK) rc = cuda_fail(ce, "end capture");
      if (rc) {
        if (g) cudaGraphDestroy(g);
        cudaGraphDestroy(whole);
        return rc;
      }
      cudaGraphNode_t node;
      e = cudaGraphAddChildGraphNode(&node, whole, nullptr, 0, g);
      cudaGraphDestroy(g);
      (void)part;
      if (e != cudaSuccess) {
        cudaGraphDestroy(whole);
        return cuda_fail(e, "child graph");
      }
    }
    e = cudaGraphInstantiate(&p->graph, whole, 0);
    cudaGraphDestroy(whole);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    p->graph_dirty = false;
  }
  cudaError_t e = cudaGraphLaunch(p->graph, p->stream);
  return e == cudaSuccess ? NDG_OK : cuda_fail(e, "graph launch");
}

void worker_main(ndg_pool* p) {
  cudaSetDevice(p->device);
  bool membership_changed = false;
  while (true) {
    std::vector<PoolSolve*> to_upload, to_retire;
    {
      std::unique_lock<std::mutex> lk(p->mu);
      // admission, first in first out, while the budget allows
      while (!p->stop && !p->queue.empty() && p->in_use + p->queue.front()->need <= p->budget) {
        PoolSolve* s = p->queue.front();
        p->queue.pop_front();
        s->state = kUploading;
        s->admit_s = now_s();
        p->in_use += s->need;
        p->peak = std::max(p->peak, p->in_use);
        to_upload.push_back(s);
      }
      // uploads finished by the io thread join at this step boundary
      for (auto& kv : p->solves) {
        PoolSolve* s = kv.second.get();
        if (s->state == kReady) {
          s->state = kRunning;
          cudaStreamWaitEvent(p->stream, s->ev, 0);
          p->running.push_back(s);
          membership_changed = true;
        }
      }
      // solves that reached their step count leave
      for (size_t i = 0; i < p->running.size();) {
        PoolSolve* s = p->running[i];
        if (s->steps_done >= s->nsteps) {
          s->state = kRetiring;
          cudaEventRecord(s->ev, p->stream);
          to_retire.push_back(s);
          p->running.erase(p->running.begin() + i);
          membership_changed = true;
        } else {
          ++i;
        }
      }
      for (PoolSolve* s : to_upload) p->io_tasks.push_back(s);
      for (PoolSolve* s : to_retire) p->io_tasks.push_back(s);
      if (!to_upload.empty() || !to_retire.empty()) p->cv_io.notify_one();
      if (p->running.empty()) {
        bool busy = !p->queue.empty() || !p->io_tasks.empty();
        for (auto& kv : p->solves) busy = busy || kv.second->state == kUploading || kv.second->state == kReady;
        if (p->stop && !busy) break;
        p->cv_work.wait_for(lk, std::chrono::milliseconds(busy ? 1 : 20));
        continue;
      }
    }
    if (membership_changed) {
      int rc = rebuild_lists(p);
      if (rc) {
        std::lock_guard<std::mutex> lk(p->mu);
        p->worker_error = ndg_last_error();
      }
      membership_changed = false;
    }
    if (launch_step(p) != NDG_OK) {
      std::lock_guard<std::mutex> lk(p->mu);
      p->worker_error = ndg_last_error();
    }
    for (PoolSolve* s : p->running) ++s->steps_done;
    // bound the look-ahead: at most two steps queued ahead of the GPU
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, p->stream);
    p->inflight.push_back(ev);
    while (p->inflight.size() > 2) {
      cudaEventSynchronize(p->inflight.front());
      cudaEventDestroy(p->inflight.front());
      p->inflight.pop_front();
    }
  }
  while (!p->inflight.empty()) {
    cudaEventSynchronize(p->inflight.front());
    cudaEventDestroy(p->inflight.front());
    p->inflight.pop_front();
  }
}

void io_main(ndg_pool* p) {
  cudaSetDevice(p->device);
  while (true) {
    PoolSolve* s = nullptr;
    {
      std::unique_lock<std::mutex> lk(p->mu);
      p->cv_io.wait(lk, [&] { return !p->io_tasks.empty() || p->stop; });
      if (p->io_tasks.empty()) {
        if (p->stop) {
          bool pending = false;
          for (auto& kv : p->solves)
            pending = pending || kv.second->state == kRunning || kv.second->state == kUploading ||
                      kv.second->state == kReady;
          if (!pending) break;
          p->cv_io.wait_for(lk, std::chrono::milliseconds(2));
        }
        continue;
      }
      s = p->io_tasks.front();
      p->io_tasks.pop_front();
    }
    if (s->state == kUploading) {
      const int roles = num_roles_for(s->rk);
      cudaError_t e = cudaSuccess;
      for (int r = 0; r < roles && e == cudaSuccess; ++r) e = cudaMallocAsync(&s->buf[r], s->state_bytes, p->io_stream);
      if (e == cudaSuccess) e = cudaMallocAsync((void**)&s->d_status, 256, p->io_stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(s->d_status, 0, sizeof(int), p->io_stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->buf[kUN], s->host.data(), s->state_bytes, cudaMemcpyHostToDevice, p->io_stream);
      for (int r = 0; r < kNumRoles; ++r) s->desc.buf[r] = s->buf[r];
      s->desc.status = s->d_status;
      if (e == cudaSuccess) e = cudaEventRecord(s->ev, p->io_stream);
      std::lock_guard<std::mutex> lk(p->mu);
      if (e != cudaSuccess) {
        p->worker_error = cudaGetErrorString(e);
        s->state = kDone;  // reported through poll as a CUDA error
        s->done_s = now_s();
        p->in_use -= s->need;
        p->cv_done.notify_all();
      } else {
        s->state = kReady;
      }
      p->cv_work.notify_one();
    } else if (s->state == kRetiring) {
      cudaStreamWaitEvent(p->io_stream, s->ev, 0);
      cudaError_t e = cudaMemcpyAsync(s->host.data(), s->buf[kUN], s->state_bytes, cudaMemcpyDeviceToHost,
                                      p->io_stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&s->h_status, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, p->io_stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(p->io_stream);
      for (int r = 0; r < kNumRoles; ++r)
        if (s->buf[r]) {
          cudaFreeAsync(s->buf[r], p->io_stream);
          s->buf[r] = nullptr;
        }
      if (s->d_status) {
        cudaFreeAsync(s->d_status, p->io_stream);
        s->d_status = nullptr;
      }
      std::lock_guard<std::mutex> lk(p->mu);
      if (e != cudaSuccess) p->worker_error = cudaGetErrorString(e);
      s->state = kDone;
      s->done_s = now_s();
      p->in_use -= s->need;
      ++p->finished;
      p->cv_done.notify_all();
      p->cv_work.notify_one();
    }
  }
}

}  // namespace

extern "C" {

int ndg_pool_create(size_t budget_bytes, int device, ndg_pool** out) {
  if (!out || budget_bytes == 0) return fail(NDG_EINVAL, "need an output pointer and a non-zero budget");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return fail(NDG_ECUDA, "no CUDA device available");
  if (device < 0 || device >= ndev) return fail(NDG_EINVAL, "bad device %d", device);
  cudaSetDevice(device);
  ndg_pool* p = new ndg_pool();
  p->budget = budget_bytes;
  p->device = device;
  cudaError_t e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->io_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "pool streams");
  }
  // keep freed blocks in the stream-ordered pool instead of returning them to the driver
  cudaMemPool_t mp;
  if (cudaDeviceGetDefaultMemPool(&mp, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  p->worker = std::thread(worker_main, p);
  p->io = std::thread(io_main, p);
  *out = p;
  return NDG_OK;
}

int ndg_pool_submit(ndg_pool* p, const ndg_config* cfg, const void* u0, size_t nbytes, int rk, double dt,
                    int nsteps, uint64_t* ticket) {
  if (!p || !cfg || !u0 || !ticket) return fail(NDG_EINVAL, "NULL argument");
  int rc = check_config(*cfg);
  if (rc) return rc;
  if (!valid_rk(rk)) return fail(NDG_EINVAL, "rk_scheme must be 3, 4 or 6");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(NDG_EINVAL, "dt must be positive and finite");
  if (nsteps < 0) return fail(NDG_EINVAL, "nsteps must be >= 0");
  if (cfg->device != p->device) return fail(NDG_EINVAL, "solve device differs from the pool's");
  auto s = std::make_unique<PoolSolve>();
  s->cfg = *cfg;
  s->cfg.stream = nullptr;
  for (int a = cfg->dim; a < 3; ++a) {
    s->cfg.elems[a] = 1;
    s->cfg.velocity[a] = 0.0;
  }
  s->kc = KernelClass{cfg->dim, cfg->degree, cfg->equation, cfg->dtype, cfg->mass};
  s->rk = rk;
  s->dt = dt;
  s->nsteps = nsteps;
  const int n = cfg->degree + 1;
  long long ndof = cfg->equation == NDG_ADVECTION ? 1 : cfg->dim + 1;
  for (int a = 0; a < cfg->dim; ++a) ndof *= (long long)cfg->elems[a] * n;
  long long nelem = 1;
  for (int a = 0; a < cfg->dim; ++a) nelem *= cfg->elems[a];
  if (nelem > 0x7fffffffLL) return fail(NDG_EINVAL, "more than 2^31 - 1 elements");
  s->state_bytes = (size_t)ndof * dtype_bytes(cfg->dtype);
  if (nbytes != s->state_bytes)
    return fail(NDG_EINVAL, "state size mismatch: got %zu bytes, expected %zu", nbytes, s->state_bytes);
  s->need = s->state_bytes * num_roles_for(rk);
  if (s->need > p->budget)
    return fail(NDG_ENOMEM, "solve needs %zu bytes, more than the pool budget %zu", s->need, p->budget);
  Basis b;
  build_basis(cfg->degree, &b);
  std::memset(&s->desc, 0, sizeof(s->desc));
  fill_solve_geometry(s->cfg, b, &s->desc);
  s->desc.dt = dt;
  s->host.assign((const char*)u0, (const char*)u0 + nbytes);
  {
    cudaSetDevice(p->device);
    cudaError_t e = cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "event create");
  }
  s->submit_s = now_s();
  std::lock_guard<std::mutex> lk(p->mu);
  if (p->stop) return fail(NDG_ESTATE, "pool is shutting down");
  s->ticket = p->next_ticket++;
  *ticket = s->ticket;
  if (nsteps == 0) {  // nothing to run: the result is the input
    s->state = kDone;
    s->done_s = s->admit_s = now_s();
    ++p->finished;
  } else {
    p->queue.push_back(s.get());
  }
  p->solves.emplace(s->ticket, std::move(s));
  p->cv_work.notify_one();
  return NDG_OK;
}

int ndg_pool_poll(ndg_pool* p, uint64_t ticket, void* result, size_t nbytes, ndg_solve_stats_t* stats,
                  double timeout_s) {
  if (!p) return fail(NDG_EINVAL, "NULL pool");
  std::unique_lock<std::mutex> lk(p->mu);
  auto it = p->solves.find(ticket);
  if (it == p->solves.end()) return fail(NDG_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  PoolSolve* s = it->second.get();
  if (s->state != kDone) {
    if (timeout_s <= 0.0) return NDG_EAGAIN;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    if (!p->cv_done.wait_until(lk, deadline, [&] { return s->state == kDone; })) {
      return fail(NDG_ETIMEOUT, "solve %llu not finished within %.3f s", (unsigned long long)ticket, timeout_s);
    }
  }
  if (result) {
    if (nbytes != s->state_bytes) return fail(NDG_EINVAL, "result buffer size mismatch");
    std::memcpy(result, s->host.data(), nbytes);
  }
  if (stats) {
    stats->submit_s = s->submit_s;
    stats->admit_s = s->admit_s;
    stats->done_s = s->done_s;
    stats->latency_s = s->done_s - s->submit_s;
    stats->t = s->dt * s->steps_done;
    stats->steps = s->steps_done;
    stats->device_bytes = s->need;
  }
  if (s->ev) cudaEventDestroy(s->ev);
  const int st = s->h_status;
  p->solves.erase(it);
  if (st == kStageErrBulkWait)
    return fail(NDG_ECUDA, "solve %llu: a stage kernel's bulk copy into shared memory did not complete within "
                "the wait limit (the result is not valid)", (unsigned long long)ticket);
  if (!p->worker_error.empty()) {
    std::string m = p->worker_error;
    return fail(NDG_ECUDA, "pool worker: %s", m.c_str());
  }
  return NDG_OK;
}

int ndg_pool_status(ndg_pool* p, int64_t* queued, int64_t* running, int64_t* finished, size_t* bytes,
                    size_t* peak) {
  if (!p) return fail(NDG_EINVAL, "NULL pool");
  std::lock_guard<std::mutex> lk(p->mu);
  if (queued) *queued = (int64_t)p->queue.size();
  if (running) {
    int64_t r = 0;
    for (auto& kv : p->solves)
      r += kv.second->state == kRunning || kv.second->state == kUploading || kv.second->state == kReady ||
           kv.second->state == kRetiring;
    *running = r;
  }
  if (finished) *finished = p->finished;
  if (bytes) *bytes = p->in_use;
  if (peak) *peak = p->peak;
  return NDG_OK;
}

int ndg_pool_destroy(ndg_pool* p) {
  if (!p) return NDG_OK;
  {
    std::lock_guard<std::mutex> lk(p->mu);
    p->stop = true;
    p->queue.clear();  // never admitted: dropped
    p->cv_work.notify_all();
    p->cv_io.notify_all();
  }
  if (p->worker.joinable()) p->worker.join();
  {
    std::lock_guard<std::mutex> lk(p->mu);
    p->cv_io.notify_all();
  }
  if (p->io.joinable()) p->io.join();
  cudaSetDevice(p->device);
  cudaStreamSynchronize(p->stream);
  cudaStreamSynchronize(p->io_stream);
  if (p->graph) cudaGraphExecDestroy(p->graph);
  for (auto& kv : p->classes) group_free(kv.second.group, p->stream);
  for (auto& kv : p->solves) {
    PoolSolve* s = kv.second.get();
    for (int r = 0; r < kNumRoles; ++r)
      if (s->buf[r]) cudaFreeAsync(s->buf[r], p->io_stream);
    if (s->d_status) cudaFreeAsync(s->d_status, p->io_stream);
    if (s->ev) cudaEventDestroy(s->ev);
  }
  cudaStreamSynchronize(p->io_stream);
  cudaStreamDestroy(p->stream);
  cudaStreamDestroy(p->io_stream);
  cudaStreamDestroy(p->cap_stream);
  delete p;
  return NDG_OK;
}

}  // extern "C"
