// Serving loop: continuous batching of TR-ALS decompositions on one GPU.
//
// Requests (tensors of different orders, sizes and ranks) are submitted from any host thread and
// queue in arrival order.  A worker thread admits queued requests in order whenever their kind of
// slot is free and the request's device footprint fits in what is left of the HBM budget (a request
// whose footprint does not fit holds back the ones behind it).  There are two kinds of slot:
//  - small requests (order <= 5, ranks <= 8, few entries; see grp_eligible) join the grouped step
//    engine (group.cu): every step advances all of them by one core update through one graph of
//    grouped kernels over a device table of the active slots, so their launch cost is shared;
//  - the others get a resident plan on their slot's own non-blocking stream; their sweeps are
//    enqueued at once as replays of the plan's captured per-sweep CUDA graph, and the tensor-core
//    MTTSP of the large tensors keeps the device busy meanwhile.
// The plans are started and retired by a worker thread and the grouped engine is driven by a thread of
// its own: a plan's set-up and tear-down take up to tens of milliseconds of host time (graph
// instantiation and destruction wait on the device), which must not hold up the engine's steps.
// Footprints are computed on the host (the plan's counting pass, or the engine's carve-up, plus a
// device copy of X when X is on the host).  Plans and workspaces allocate stream-ordered, so admitting
// and retiring requests never synchronises the device.  A plan request computes exactly what
// trals_decompose computes for it alone; a grouped request computes the same method in the same
// precisions with the engine's own kernels.  Either way the kernels are deterministic and slots share
// no device state, so a result does not depend on what else was in flight.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "group.cuh"
#include "trals_internal.cuh"
#include "../../include/trals_testing.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int N = 0;
  int64_t I[TRALS_MAX_ORDER] = {};
  int32_t R[TRALS_MAX_ORDER] = {};
  const void* X = nullptr;
  int xt = 0;
  int x_on_host = 0;
  size_t x_bytes = 0;
  int sweeps = 0;
  trals_opts opts{};
  std::vector<std::vector<double>> cores;   // initial cores at submit, fitted cores when done
  std::vector<double> res;                  // relative residual per sweep
  size_t footprint = 0;
  bool grouped = false;                     // served by the grouped step engine
  double t_submit = 0, t_admit = -1, t_done = -1;
  trals_status status = TRALS_E_PENDING;
  std::string error;
};

struct Slot {
  cudaStream_t stream = nullptr;
  trals_ctx* ctx = nullptr;
  cudaEvent_t done = nullptr;
  Request* req = nullptr;
  trals_plan* plan = nullptr;
  void* Xdev = nullptr;
  // pinned landing buffers for the results, so that collecting them never blocks the worker
  double* h_res = nullptr;
  size_t res_cap = 0;
  double* h_cores = nullptr;
  size_t cores_cap = 0;
  void* h_status = nullptr;
};

// Grow a pinned host buffer to hold at least `need` doubles.
cudaError_t reserve_pinned(double** buf, size_t* cap, size_t need) {
  if (*cap >= need) return cudaSuccess;
  if (*buf) cudaFreeHost(*buf);
  *buf = nullptr;
  *cap = 0;
  const size_t c = std::max<size_t>(need, 4096);
  cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(buf), c * sizeof(double), cudaHostAllocDefault);
  if (e == cudaSuccess) *cap = c;
  return e;
}

}  // namespace

struct trals_server {
  int device = 0;
  size_t budget = 0;
  size_t used = 0;
  int max_slots = 0;
  std::vector<Slot> slots;
  trals_ctx* sizing = nullptr;     // context for footprint counts (no work is ever enqueued on it)
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> tickets;
  uint64_t next_ticket = 1;
  uint64_t completed = 0;
  size_t peak_used = 0;
  int peak_active = 0;
  std::mutex mu;
  std::condition_variable cv;      // submit / stop -> worker
  std::condition_variable done_cv; // worker -> waiters
  std::thread worker;                   // admission and the plan requests
  std::thread engine;                   // the grouped step engine
  bool stopping = false;
  trals::GroupEngine* grp = nullptr;    // grouped step engine (small requests), driven by its own thread
  std::deque<Request*> ginbox;          // admitted grouped requests not yet taken by the engine thread
  std::condition_variable gcv;          // worker / stop -> engine thread
  // requests up to 2^18 entries (every order-3 tensor of sizes <= 64): larger ones run their MTTSP faster on
  // the tensor cores of a plan than in the grouped CUDA-core kernel
  int64_t grp_max_elems = (int64_t)1 << 18;
  int grp_active = 0;                   // engine slots holding a request
  uint64_t grouped_completed = 0;
  uint64_t grouped_steps = 0;
  int withhold_steps = 0;               // testing: steps whose descriptor table is withheld
  long long withhold_spin = 0;
  double host_start_s = 0;         // host time spent starting requests (plan set-up, graph capture, launches)
  cudaMemPool_t pool = nullptr;    // the device's default pool and its release threshold before the server
  uint64_t pool_threshold = 0;
  Clock::time_point t0;
  std::string last_error;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

size_t x_elem_bytes(int xt) { return xt == TRALS_X_F64 ? 8 : xt == TRALS_X_F32 ? 4 : 2; }

// Admitted request: everything it needs is enqueued on the slot's stream without waiting: the copy
// of X (host X only), the plan set-up, all its sweeps (graph replays), the final explicit residual
// where the per-sweep one is not computed, and the copies of its results into the slot's pinned
// buffers; the slot's event marks the end.
trals_status start_request(Slot& sl) {
  Request* r = sl.req;
  const void* X = r->X;
  if (r->x_on_host) {
    cudaError_t e = cudaMallocAsync(&sl.Xdev, r->x_bytes, sl.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.Xdev, r->X, r->x_bytes, cudaMemcpyHostToDevice, sl.stream);
    if (e != cudaSuccess) {
      r->error = std::string("device copy of X: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? TRALS_E_OOM : TRALS_E_CUDA;
    }
    X = sl.Xdev;
  }
  trals_status st = trals::plan_create_async(sl.ctx, r->N, r->I, r->R, X, r->xt, &r->opts, &sl.plan);
  if (st == TRALS_OK) {
    std::vector<const double*> ptrs(r->N);
    for (int n = 0; n < r->N; ++n) ptrs[n] = r->cores[n].data();
    st = trals::plan_set_cores_async(sl.plan, ptrs.data());
  }
  if (st == TRALS_OK) st = trals_plan_run(sl.plan, r->sweeps, 1);
  if (st == TRALS_OK) {
    cudaError_t e = reserve_pinned(&sl.h_res, &sl.res_cap, (size_t)std::max(r->sweeps, 1));
    if (e == cudaSuccess) e = reserve_pinned(&sl.h_cores, &sl.cores_cap, trals::plan_core_elems(sl.plan));
    if (e != cudaSuccess) {
      r->error = std::string("pinned result buffers: ") + cudaGetErrorString(e);
      return TRALS_E_CUDA;
    }
    const bool final_explicit = r->sweeps > 0 && r->opts.mode != TRALS_MODE_FP64 && !r->opts.explicit_residual;
    st = trals::plan_enqueue_results(sl.plan, r->sweeps, final_explicit, sl.h_res, sl.h_cores, sl.h_status);
  }
  if (st == TRALS_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = TRALS_E_CUDA;
  if (st != TRALS_OK && r->error.empty()) r->error = trals_last_error(sl.ctx);
  return st;
}

// Request whose event has completed (or that failed to start): take its results from the pinned
// buffers and release its device memory.  Only the slot's own (finished) stream is waited on.
void finish_request(trals_server* S, Slot& sl, trals_status st) {
  Request* r = sl.req;
  if (st == TRALS_OK && sl.plan) {
    const int code = trals::status_code(sl.h_status);
    if (code != TRALS_OK) {
      st = (trals_status)code;
      r->error = trals::status_message(sl.h_status);
    } else {
      std::memcpy(r->res.data(), sl.h_res, r->sweeps * sizeof(double));
      size_t off = 0;
      for (int n = 0; n < r->N; ++n) {
        std::memcpy(r->cores[n].data(), sl.h_cores + off, r->cores[n].size() * sizeof(double));
        off += r->cores[n].size();
      }
    }
  }
  if (sl.plan) trals_plan_destroy(sl.plan);
  sl.plan = nullptr;
  if (sl.Xdev) cudaFreeAsync(sl.Xdev, sl.stream);
  sl.Xdev = nullptr;
  std::lock_guard<std::mutex> lk(S->mu);
  r->status = st;
  r->t_done = S->now();
  S->used -= r->footprint;
  sl.req = nullptr;
  ++S->completed;
  S->done_cv.notify_all();
}

// A grouped request's outcome: results from the engine's pinned buffers, then its slot is released.
void finish_grouped(trals_server* S, Request* r, int gslot, trals_status st, const std::string& err) {
  if (st == TRALS_OK) {
    const double* cores = nullptr;
    double res = 0.0;
    std::string msg;
    const int code = trals::grp_result(S->grp, gslot, &cores, &res, &msg);
    if (code != TRALS_OK) {
      st = (trals_status)code;
      r->error = msg;
    } else {
      size_t off = 0;
      for (int n = 0; n < r->N; ++n) {
        std::memcpy(r->cores[n].data(), cores + off, r->cores[n].size() * sizeof(double));
        off += r->cores[n].size();
      }
      // as the reduced-precision plans: no per-sweep residual, the explicit one after the last sweep
      for (int k = 0; k + 1 < r->sweeps; ++k) r->res[k] = std::nan("");
      r->res[r->sweeps - 1] = res;
    }
  } else {
    r->error = err;
  }
  if (gslot >= 0) trals::grp_release(S->grp, gslot);
  std::lock_guard<std::mutex> lk(S->mu);
  r->status = st;
  r->t_done = S->now();
  S->used -= r->footprint;
  if (gslot >= 0) --S->grp_active;
  ++S->completed;
  ++S->grouped_completed;
  S->done_cv.notify_all();
}

void worker_main(trals_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<int> admitted;
    int active = 0, handed = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (const Slot& sl : S->slots) active += sl.req != nullptr;
      if (S->stopping && active == 0) break;
      // admission in arrival order: a request waits for a slot of its kind (those behind it may pass),
      // and one whose footprint does not fit holds back the rest
      int gfree = S->grp ? trals::kGrpMaxSlots - S->grp_active : 0;
      for (auto it = S->queue.begin(); !S->stopping && it != S->queue.end();) {
        Request* r = *it;
        if (S->used + r->footprint > S->budget) break;
        int free_slot = -1;
        if (r->grouped) {
          if (gfree == 0) {
            ++it;
            continue;
          }
          --gfree;
          S->ginbox.push_back(r);
          ++S->grp_active;
          ++handed;
        } else {
          for (int k = 0; k < (int)S->slots.size(); ++k)
            if (!S->slots[k].req) {
              free_slot = k;
              break;
            }
          if (free_slot < 0) {
            ++it;
            continue;
          }
          S->slots[free_slot].req = r;
          admitted.push_back(free_slot);
          ++active;
        }
        it = S->queue.erase(it);
        S->used += r->footprint;
        S->peak_used = std::max(S->peak_used, S->used);
        r->t_admit = S->now();
      }
      S->peak_active = std::max(S->peak_active, active + S->grp_active);
    }
    if (handed) S->gcv.notify_all();
    bool progress = !admitted.empty() || handed > 0;
    const auto t0 = Clock::now();
    for (int k : admitted) {
      const trals_status st = start_request(S->slots[k]);
      if (st != TRALS_OK) finish_request(S, S->slots[k], st);
    }
    if (!admitted.empty()) {
      const double dt = std::chrono::duration<double>(Clock::now() - t0).count();
      std::lock_guard<std::mutex> lk(S->mu);
      S->host_start_s += dt;
    }
    for (Slot& sl : S->slots) {
      if (!sl.req || !sl.plan) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      progress = true;
      if (q != cudaSuccess) {
        sl.req->error = std::string("stream error: ") + cudaGetErrorString(q);
        finish_request(S, sl, TRALS_E_CUDA);
      } else {
        finish_request(S, sl, TRALS_OK);
      }
    }
    if (!progress) {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait_for(lk, std::chrono::microseconds(active > 0 ? 20 : 2000));
    }
  }
}

// The grouped engine: takes the requests the worker admitted, launches steps while any is active and
// hands back the finished ones.
void engine_main(trals_server* S) {
  cudaSetDevice(S->device);
  std::vector<Request*> gslot_req(trals::kGrpMaxSlots, nullptr);
  for (;;) {
    std::vector<Request*> take;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stopping && S->grp_active == 0 && S->ginbox.empty()) break;
      while (!S->ginbox.empty()) {
        take.push_back(S->ginbox.front());
        S->ginbox.pop_front();
      }
      if (S->withhold_steps > 0) {
        trals::grp_withhold(S->grp, S->withhold_steps, S->withhold_spin);
        S->withhold_steps = 0;
      }
    }
    bool progress = !take.empty();
    for (Request* r : take) {
      std::vector<const double*> init(r->N);
      for (int n = 0; n < r->N; ++n) init[n] = r->cores[n].data();
      std::string err;
      const int g = trals::grp_admit(S->grp, r->N, r->I, r->R, static_cast<const float*>(r->X), r->x_on_host != 0,
                                     r->opts.mode, r->sweeps, init.data(), &err);
      if (g < 0) finish_grouped(S, r, -1, TRALS_E_CUDA, err);
      else gslot_req[g] = r;
    }
    std::string err;
    if (trals::grp_step(S->grp, &err)) {
      progress = true;
      std::lock_guard<std::mutex> lk(S->mu);
      S->grouped_steps = trals::grp_steps(S->grp);
    } else if (!err.empty()) {
      std::lock_guard<std::mutex> lk(S->mu);
      S->last_error = err;
    }
    std::vector<int> done;
    trals::grp_poll(S->grp, &done);
    for (int g : done) {
      Request* r = gslot_req[g];
      gslot_req[g] = nullptr;
      finish_grouped(S, r, g, TRALS_OK, std::string());
      progress = true;
    }
    if (!progress) {
      std::unique_lock<std::mutex> lk(S->mu);
      S->gcv.wait_for(lk, std::chrono::microseconds(trals::grp_busy(S->grp) ? 10 : 2000));
    }
  }
}

}  // namespace

extern "C" {

trals_status trals_server_create(trals_server** out, int device, size_t hbm_budget_bytes, int max_slots) {
  if (!out || max_slots < 1 || max_slots > 1024 || hbm_budget_bytes == 0) return TRALS_E_ARG;
  *out = nullptr;
  trals_server* S = new trals_server();
  S->device = device;
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  S->t0 = Clock::now();
  // Plans and workspaces allocate stream-ordered from the device's default pool.  Its release threshold
  // (0 by default) would hand the memory back at every synchronisation, so that each large request
  // maps gigabytes afresh on the worker thread; keep up to the budget in the pool while the server runs.
  if (cudaSetDevice(device) == cudaSuccess && cudaDeviceGetDefaultMemPool(&S->pool, device) == cudaSuccess) {
    cudaMemPoolGetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &S->pool_threshold);
    uint64_t keep = std::max<uint64_t>(S->pool_threshold, hbm_budget_bytes);
    cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  } else {
    S->pool = nullptr;
  }
  trals_status st = trals_create(&S->sizing, device, nullptr);
  if (st == TRALS_OK) {
    S->slots.resize(max_slots);
    for (Slot& sl : S->slots) {
      if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
        st = TRALS_E_CUDA;
        break;
      }
      st = trals_create(&sl.ctx, device, sl.stream);
      if (st != TRALS_OK) break;
      if (cudaHostAlloc(&sl.h_status, 64, cudaHostAllocDefault) != cudaSuccess ||
          reserve_pinned(&sl.h_res, &sl.res_cap, 1024) != cudaSuccess ||
          reserve_pinned(&sl.h_cores, &sl.cores_cap, 1 << 16) != cudaSuccess) {
        st = TRALS_E_CUDA;
        break;
      }
    }
  }
  if (st == TRALS_OK) {
    std::string err;
    S->grp = trals::grp_create(device, &err);
    if (!S->grp) {
      S->last_error = err;
      st = TRALS_E_CUDA;
    }
  }
  if (st != TRALS_OK) {
    trals_server_destroy(S);
    return st;
  }
  S->worker = std::thread(worker_main, S);
  S->engine = std::thread(engine_main, S);
  *out = S;
  return TRALS_OK;
}

void trals_server_destroy(trals_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
    for (Request* r : S->queue) {   // never admitted: dropped
      r->status = TRALS_E_REJECTED;
      r->error = "server destroyed before admission";
    }
    S->queue.clear();
  }
  S->cv.notify_all();
  S->gcv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  if (S->engine.joinable()) S->engine.join();
  for (auto& kv : S->tickets) delete kv.second;
  for (Slot& sl : S->slots) {
    if (sl.ctx) trals_destroy(sl.ctx);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.h_res) cudaFreeHost(sl.h_res);
    if (sl.h_cores) cudaFreeHost(sl.h_cores);
    if (sl.h_status) cudaFreeHost(sl.h_status);
  }
  if (S->grp) trals::grp_destroy(S->grp);
  if (S->sizing) trals_destroy(S->sizing);
  if (S->pool) {
    cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &S->pool_threshold);
    cudaMemPoolTrimTo(S->pool, 0);
  }
  delete S;
}

trals_status trals_server_submit(trals_server* S, const trals_request* q, uint64_t* ticket) {
  if (!S || !q || !ticket || !q->X || !q->init_cores || q->sweeps < 0 || q->N < 3 || q->N > TRALS_MAX_ORDER ||
      !q->I || !q->R)
    return TRALS_E_ARG;
  Request* r = new Request();
  r->N = q->N;
  int64_t numel = 1;
  for (int n = 0; n < q->N; ++n) {
    r->I[n] = q->I[n];
    r->R[n] = q->R[n];
    numel *= q->I[n] > 0 ? q->I[n] : 1;
  }
  r->X = q->X;
  r->xt = q->xt;
  r->x_on_host = q->x_on_host;
  r->x_bytes = (size_t)numel * x_elem_bytes(q->xt);
  r->sweeps = q->sweeps;
  r->opts = q->opts;
  r->res.assign(std::max(q->sweeps, 1), 0.0);
  size_t fp = 0;
  trals_status st;
  {
    std::lock_guard<std::mutex> lk(S->mu);   // the sizing context's error string is shared
    // a host X is inspected for alignment only; the device copy will be 256-byte aligned
    const void* xprobe = q->x_on_host ? reinterpret_cast<const void*>(uintptr_t(1) << 40) : q->X;
    st = trals_plan_footprint(S->sizing, r->N, r->I, r->R, xprobe, r->xt, &r->opts, &fp);
    if (st != TRALS_OK) S->last_error = trals_last_error(S->sizing);
    r->grouped = st == TRALS_OK && S->grp &&
                 trals::grp_eligible(r->N, r->I, r->R, r->xt, r->opts, r->sweeps, S->grp_max_elems);
  }
  if (st != TRALS_OK) {
    delete r;
    return st;
  }
  if (r->grouped)
    r->footprint = trals::grp_footprint(r->N, r->I, r->R, r->opts.mode, r->x_on_host != 0);
  else
    r->footprint = fp + (r->x_on_host ? ((r->x_bytes + 255) & ~(size_t)255) : 0);
  if (r->footprint > S->budget) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->last_error = "request footprint " + std::to_string(r->footprint) + " B exceeds the HBM budget " +
                    std::to_string(S->budget) + " B";
    delete r;
    return TRALS_E_REJECTED;
  }
  r->cores.resize(r->N);
  for (int n = 0; n < r->N; ++n) {
    if (!q->init_cores[n]) {
      delete r;
      return TRALS_E_ARG;
    }
    const size_t cnt = (size_t)r->R[n] * r->I[n] * r->R[(n + 1) % r->N];
    r->cores[n].assign(q->init_cores[n], q->init_cores[n] + cnt);
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) {
      delete r;
      return TRALS_E_REJECTED;
    }
    r->ticket = S->next_ticket++;
    r->t_submit = S->now();
    S->tickets[r->ticket] = r;
    S->queue.push_back(r);
    *ticket = r->ticket;
  }
  S->cv.notify_all();
  return TRALS_OK;
}

static trals_status take_result(trals_server* S, Request* r, trals_result* res, double* const* cores_out,
                                double* rel_res_out) {
  if (res) {
    res->status = r->status;
    res->sweeps = r->sweeps;
    res->submit_s = r->t_submit;
    res->admit_s = r->t_admit;
    res->done_s = r->t_done;
    res->footprint_bytes = r->footprint;
  }
  if (cores_out)
    for (int n = 0; n < r->N; ++n)
      if (cores_out[n]) std::memcpy(cores_out[n], r->cores[n].data(), r->cores[n].size() * sizeof(double));
  if (rel_res_out && r->sweeps > 0) std::memcpy(rel_res_out, r->res.data(), r->sweeps * sizeof(double));
  if (r->status != TRALS_OK) S->last_error = r->error;
  S->tickets.erase(r->ticket);
  delete r;
  return TRALS_OK;
}

trals_status trals_server_poll(trals_server* S, uint64_t ticket, trals_result* res, double* const* cores_out,
                               double* rel_res_out) {
  if (!S) return TRALS_E_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return TRALS_E_ARG;
  if (it->second->status == TRALS_E_PENDING) return TRALS_E_PENDING;
  return take_result(S, it->second, res, cores_out, rel_res_out);
}

trals_status trals_server_wait(trals_server* S, uint64_t ticket, double timeout_s, trals_result* res,
                               double* const* cores_out, double* rel_res_out) {
  if (!S) return TRALS_E_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return TRALS_E_ARG;
  Request* r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(
                                           timeout_s < 0 ? 1e9 : timeout_s));
  while (r->status == TRALS_E_PENDING)
    if (S->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && r->status == TRALS_E_PENDING)
      return TRALS_E_PENDING;
  return take_result(S, r, res, cores_out, rel_res_out);
}

trals_status trals_server_stats(trals_server* S, trals_server_info* out) {
  if (!S || !out) return TRALS_E_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  int active = 0;
  for (const Slot& sl : S->slots) active += sl.req != nullptr;
  out->queued = (int)S->queue.size();
  out->active = active;
  out->completed = S->completed;
  out->used_bytes = S->used;
  out->peak_used_bytes = S->peak_used;
  out->peak_active = S->peak_active;
  out->host_start_s = S->host_start_s;
  out->grouped_completed = S->grouped_completed;
  out->grouped_steps = S->grouped_steps;
  return TRALS_OK;
}

trals_status trals_server_set_group_limit(trals_server* S, int64_t max_elems) {
  if (!S || max_elems < 0) return TRALS_E_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  S->grp_max_elems = max_elems;
  return TRALS_OK;
}

trals_status trals_testing_server_withhold_steps(trals_server* S, int steps, long long spin_cycles) {
  if (!S || steps < 0 || spin_cycles <= 0) return TRALS_E_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  S->withhold_steps = steps;
  S->withhold_spin = spin_cycles;
  return TRALS_OK;
}

const char* trals_server_last_error(const trals_server* S) { return S ? S->last_error.c_str() : "null server"; }

}  // extern "C"
