// fsa_serve_*: a continuous-batching serving loop over the apply path.
//
// One host thread owns the device side.  Each turn of its loop it
//   1. retires in-flight requests whose completion event has fired (their
//      workspace goes back to the stream-ordered pool, their ticket -> DONE);
//   2. admits queued requests in arrival order while fewer than max_inflight
//      are on the GPU and the bytes the server holds (resident plans plus
//      in-flight workspaces) plus the request's need fit the HBM budget:
//      hbm_fraction x (device memory free now + what the server holds),
//      re-read from the driver before each admission round so that memory
//      taken or returned by other users of the device counts, capped by
//      hbm_budget_bytes; idle plans are evicted LRU-first, and workspace the
//      pool keeps but no request uses is trimmed, to make room;
//   3. enqueues each admitted request's five passes on one of its streams
//      (round robin) with a workspace from cudaMallocAsync, so requests that
//      arrive while others run start as soon as a slot and memory free up
//      and their kernels overlap on the device.
// A request's result never depends on the mix: it runs the same kernels on
// its own workspace with its plan's spectrum; nothing is reduced across
// requests.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fsa_internal.h"

namespace fsa {
fsa_status plan_create_internal(fsa_plan** out, fsa_kernel kernel, const double* L, const int* n, fsa_dtype dtype,
                                double eps, double eps_tol, bool with_workspace, double param);
cudaError_t plan_generate_into(fsa_plan* p, void* scratch, cudaStream_t s);
size_t plan_workspace_bytes(const int* n, fsa_dtype dt);
size_t plan_gen_scratch_bytes(const int* n, fsa_dtype dt, int d);
size_t plan_resident_bytes(const int* n, fsa_dtype dt, int d);
}  // namespace fsa

using namespace fsa;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct PlanKey {
  int n[3];
  int kernel;
  double L[3];
  int dt;
  double eps;
  double param;
  bool operator<(const PlanKey& o) const {
    return std::memcmp(this, &o, sizeof(PlanKey)) < 0;
  }
};

struct CachedPlan {
  fsa_plan* plan = nullptr;
  cudaEvent_t ready = nullptr;  // recorded after generation, on the generating stream
  int refs = 0;
  size_t bytes = 0;
  std::list<PlanKey>::iterator lru;
};

struct Req {
  fsa_request r{};
  fsa_req_state state = FSA_REQ_QUEUED;
  fsa_req_times t{};
  PlanKey key{};
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaEvent_t done = nullptr;
  cudaStream_t stream = nullptr;
  int lane = -1;        // index into the server's streams
  double work = 0;      // estimated work (size_aware_work)
};

// Estimated work of a request in relative units: grid points, times 5 for the
// FP64 tier (its double-word passes run about 5x longer than FP32 ones).
double size_aware_work(const fsa_request& r) {
  const double V = (double)r.n[0] * r.n[1] * (r.d == 2 ? 1 : r.n[2]);
  return V * (r.dtype == FSA_F64 ? 5.0 : 1.0);
}
// Requests at least this large (about a 384^3 FP32 or a 256^3 FP64 solve,
// 2 ms and more on GB300) go to the bulk lane.
constexpr double kBulkWork = 4.0e7;

}  // namespace

struct fsa_server {
  fsa_serve_opts o{};
  int device = 0;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  std::vector<uint64_t> inflight;
  uint64_t next = 1;
  bool stop = false;
  std::thread worker;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> free_events;
  size_t rr = 0;
  int nbulk = 0;                 // size-aware policy: the last nbulk streams are the bulk lane
  std::vector<double> lane_work;  // estimated work in flight per stream
  cudaMemPool_t pool = nullptr;
  std::map<PlanKey, CachedPlan> plans;
  std::list<PlanKey> plan_lru;  // front = most recent
  size_t held = 0;              // plan bytes + in-flight workspace bytes
  size_t ws_inflight = 0;       // the in-flight workspace part of held
  size_t budget_cap = 0;        // hbm_budget_bytes (0 = none)
  fsa_serve_stats st{};
};

namespace {

// Evict idle plans (LRU) other than `keep` until `need` more bytes fit, or
// nothing idle is left.
void make_room(fsa_server* s, size_t need, const PlanKey& keep) {
  auto it = s->plan_lru.end();
  while (s->held + need > s->budget && it != s->plan_lru.begin()) {
    --it;
    auto pit = s->plans.find(*it);
    if (pit->second.refs == 0 && std::memcmp(&pit->first, &keep, sizeof keep) != 0) {
      s->held -= pit->second.bytes;
      fsa_plan_destroy(pit->second.plan);
      cudaEventDestroy(pit->second.ready);
      s->plans.erase(pit);
      it = s->plan_lru.erase(it);
    }
  }
}

// Evict the least recently used idle plan other than `keep`, if any.
void evict_one(fsa_server* s, const PlanKey& keep) {
  for (auto it = s->plan_lru.end(); it != s->plan_lru.begin();) {
    --it;
    auto pit = s->plans.find(*it);
    if (pit->second.refs == 0 && std::memcmp(&pit->first, &keep, sizeof keep) != 0) {
      s->held -= pit->second.bytes;
      fsa_plan_destroy(pit->second.plan);
      cudaEventDestroy(pit->second.ready);
      s->plans.erase(pit);
      s->plan_lru.erase(it);
      return;
    }
  }
}

// Bytes the workspace pool keeps reserved on the device (in use or idle).
size_t pool_reserved(fsa_server* s) {
  uint64_t r = 0;
  if (cudaMemPoolGetAttribute(s->pool, cudaMemPoolAttrReservedMemCurrent, &r) != cudaSuccess) {
    cudaGetLastError();
    return s->ws_inflight;
  }
  return (size_t)r;
}

// Re-read the device's free memory: the budget is hbm_fraction x (free now +
// what this server holds on the device), so that memory other users take or
// return since the server started counts.  Capped by hbm_budget_bytes.
void refresh_budget(fsa_server* s) {
  size_t freeb = 0, total = 0;
  if (cudaMemGetInfo(&freeb, &total) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const size_t mine = (s->held - s->ws_inflight) + std::max(pool_reserved(s), s->ws_inflight);
  size_t b = (size_t)(s->o.hbm_fraction * (double)(freeb + mine));
  if (s->budget_cap && s->budget_cap < b) b = s->budget_cap;
  s->budget = b;
}

// Try to start request `id`; returns false if it must wait for room.
bool try_admit(fsa_server* s, uint64_t id) {
  Req& q = s->reqs[id];
  const size_t ws = plan_workspace_bytes(q.r.n, q.r.dtype);
  const bool hit = s->plans.count(q.key) != 0;
  size_t plan_bytes = 0, gen_scratch = 0;
  if (!hit) {
    plan_bytes = plan_resident_bytes(q.r.n, q.r.dtype, q.r.d);
    gen_scratch = plan_gen_scratch_bytes(q.r.n, q.r.dtype, q.r.d);
  }
  const size_t need = ws + plan_bytes + gen_scratch;
  // make_room never evicts this request's own plan, so `hit` stays valid
  if (s->held + need > s->budget) make_room(s, need, q.key);
  if ((int)s->plans.size() >= s->o.plan_cache_max && !hit) evict_one(s, q.key);
  if (s->held + need > s->budget && !(s->inflight.empty() && s->held == 0)) return false;
  // Workspace the pool keeps from finished requests is reused first; when the
  // pool holds more idle memory than the new request can reuse and the total
  // would pass the budget, give the idle part back before allocating.
  if (s->held - s->ws_inflight + pool_reserved(s) + plan_bytes + gen_scratch + ws > s->budget) {
    cudaMemPoolTrimTo(s->pool, s->ws_inflight);
    cudaGetLastError();
  }
  auto pit = s->plans.find(q.key);

  // stream: round robin (policy 1), or (policy 0) the least loaded stream of
  // the request's lane -- large requests on low-priority bulk streams, the
  // rest on high-priority streams -- so no request queues behind a long
  // solve on its own stream
  int lane = 0;
  const double work = size_aware_work(q.r);
  const bool bulk = s->nbulk > 0 && work >= kBulkWork;
  if (s->nbulk == 0) {
    lane = (int)(s->rr++ % s->streams.size());
  } else {
    const int nfast = (int)s->streams.size() - s->nbulk;
    const int lo = bulk ? nfast : 0, hi = bulk ? (int)s->streams.size() : nfast;
    lane = lo;
    for (int i = lo + 1; i < hi; ++i)
      if (s->lane_work[i] < s->lane_work[lane]) lane = i;
  }
  cudaStream_t stream = s->streams[lane];
  fsa_status status = FSA_OK;
  cudaError_t e = cudaSuccess;
  if (!hit) {
    fsa_plan* p = nullptr;
    status = plan_create_internal(&p, q.r.kernel, q.r.L, q.r.n, q.r.dtype, q.r.eps, 0.0, false, q.r.kernel_param);
    if (status == FSA_OK)  // charge what the plan really holds
      plan_bytes = p->spectrum_bytes + (p->spectrum_dw ? p->spectrum_bytes : 0);
    // server plans have no workspace of their own; FP64 arithmetic follows the
    // per-shape choice made by earlier plans (double-word by default)
    if (status == FSA_OK) {
      void* scratch = nullptr;
      cudaEvent_t ready = nullptr;
      if (gen_scratch) e = cudaMallocFromPoolAsync(&scratch, gen_scratch, s->pool, stream);
      if (e == cudaSuccess) e = plan_generate_into(p, scratch, stream);
      if (scratch) cudaFreeAsync(scratch, stream);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(ready, stream);
      if (e != cudaSuccess) {
        fsa_plan_destroy(p);
        if (ready) cudaEventDestroy(ready);
        status = cuda_error(e, "serve: tensor generation");
      } else {
        s->plan_lru.push_front(q.key);
        CachedPlan cp;
        cp.plan = p;
        cp.ready = ready;
        cp.bytes = plan_bytes;
        cp.lru = s->plan_lru.begin();
        pit = s->plans.emplace(q.key, cp).first;
        s->held += plan_bytes;
      }
    }
    s->st.plan_misses++;
  } else {
    s->plan_lru.erase(pit->second.lru);
    s->plan_lru.push_front(q.key);
    pit->second.lru = s->plan_lru.begin();
    s->st.plan_hits++;
  }
  q.t.admit_s = now_s();
  q.t.plan_hit = hit ? 1 : 0;
  if (status != FSA_OK) {
    q.state = FSA_REQ_FAILED;
    q.t.status = status;
    q.t.done_s = now_s();
    s->st.failed++;
    return true;
  }
  fsa_plan* p = pit->second.plan;
  // the spectrum may still be generating on another stream
  e = cudaStreamWaitEvent(stream, pit->second.ready, 0);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&q.ws, ws, s->pool, stream);
  if (e == cudaSuccess) {
    const void* rho[1] = {q.r.rho};
    void* phi[1] = {q.r.phi};
    void* X[1] = {q.ws};
    const size_t xb = (size_t)(q.r.n[0] + 1) * q.r.n[1] * q.r.n[2] * 2 * (q.r.dtype == FSA_F32 ? 4 : 8);
    void* Y[1] = {(char*)q.ws + xb};
    const void* S[1] = {plan_apply_spectrum(p)};
    // bulk requests launch one CTA per tile: their blocks retire as they go,
    // so kernels of the high-priority streams get SMs in between
    launch_grid_mode() = bulk ? 1 : 0;
    e = run_group(p, 1, rho, phi, X, Y, S, stream);
    launch_grid_mode() = 0;
    cudaFreeAsync(q.ws, stream);
  }
  if (e == cudaSuccess) {
    if (!s->free_events.empty()) {
      q.done = s->free_events.back();
      s->free_events.pop_back();
    } else {
      e = cudaEventCreateWithFlags(&q.done, cudaEventDisableTiming);
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(q.done, stream);
  if (e != cudaSuccess) {
    q.state = FSA_REQ_FAILED;
    q.t.status = cuda_error(e, "serve: launch");
    q.t.done_s = now_s();
    s->st.failed++;
    cudaGetLastError();
    return true;
  }
  pit->second.refs++;
  q.ws_bytes = ws;
  q.stream = stream;
  q.lane = lane;
  q.work = work;
  s->lane_work[lane] += work;
  s->held += ws;
  s->ws_inflight += ws;
  q.state = FSA_REQ_RUNNING;
  s->inflight.push_back(id);
  return true;
}

void retire(fsa_server* s) {
  for (size_t i = 0; i < s->inflight.size();) {
    Req& q = s->reqs[s->inflight[i]];
    cudaError_t e = cudaEventQuery(q.done);
    if (e == cudaErrorNotReady) {
      ++i;
      continue;
    }
    q.t.done_s = now_s();
    if (e == cudaSuccess) {
      q.state = FSA_REQ_DONE;
      q.t.status = FSA_OK;
      s->st.completed++;
    } else {
      q.state = FSA_REQ_FAILED;
      q.t.status = cuda_error(e, "serve: device");
      s->st.failed++;
    }
    s->free_events.push_back(q.done);
    q.done = nullptr;
    s->held -= q.ws_bytes;
    s->ws_inflight -= q.ws_bytes;
    if (q.lane >= 0) s->lane_work[q.lane] -= q.work;
    auto pit = s->plans.find(q.key);
    if (pit != s->plans.end()) pit->second.refs--;
    s->inflight[i] = s->inflight.back();
    s->inflight.pop_back();
  }
}

void loop(fsa_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    const size_t before = s->inflight.size();
    retire(s);
    bool changed = s->inflight.size() != before;
    if (!s->queue.empty() && (int)s->inflight.size() < s->o.max_inflight) refresh_budget(s);
    while (!s->queue.empty() && (int)s->inflight.size() < s->o.max_inflight) {
      const uint64_t id = s->queue.front();
      if (!try_admit(s, id)) break;
      s->queue.pop_front();
      changed = true;
    }
    if (changed) s->cv_done.notify_all();
    if (s->stop && s->queue.empty() && s->inflight.empty()) break;
    if (!s->inflight.empty())
      s->cv_work.wait_for(lk, std::chrono::microseconds(20));
    else
      s->cv_work.wait_for(lk, std::chrono::milliseconds(50), [&] { return s->stop || !s->queue.empty(); });
  }
}

bool valid_request(const fsa_request* r) {
  if (!r || r->kernel < FSA_KERNEL_COULOMB3D || r->kernel > FSA_KERNEL_YUKAWA2D) return false;
  if (r->kernel == FSA_KERNEL_DDI3D) return false;  // DDI plans need dipoles: fsa_plan_create_ddi3d
  if (!(r->kernel_param >= 0) || !std::isfinite(r->kernel_param)) return false;
  if (r->d != kernel_dim(r->kernel)) return false;
  if (r->dtype != FSA_F32 && r->dtype != FSA_F64) return false;
  if (!r->rho || !r->phi || (((uintptr_t)r->rho | (uintptr_t)r->phi) & 15u)) return false;
  if (!(r->eps >= 0)) return false;
  for (int j = 0; j < r->d; ++j)
    if (!supported_n(r->n[j]) || !(r->L[j] > 0)) return false;
  return true;
}

}  // namespace

extern "C" {

fsa_status fsa_serve_create(fsa_server** out, const fsa_serve_opts* opts) {
  if (!out) return set_error(FSA_ERR_INVALID_ARG, "fsa_serve_create: out is NULL");
  *out = nullptr;
  fsa_serve_opts o{};
  o.device = -1;
  if (opts) o = *opts;
  if (o.max_inflight <= 0) o.max_inflight = 64;
  if (o.streams <= 0) o.streams = 8;
  if (!(o.hbm_fraction > 0 && o.hbm_fraction <= 1)) o.hbm_fraction = 0.9;
  if (o.plan_cache_max <= 0) o.plan_cache_max = 64;
  if (o.queue_max <= 0) o.queue_max = 1 << 20;
  if (o.policy != 1) o.policy = 0;
  int dev = o.device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return set_error(FSA_ERR_CUDA, "fsa_serve_create: no device");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(dev);
  fsa_server* s = new fsa_server();
  s->o = o;
  s->device = dev;
  size_t freeb = 0, total = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&freeb, &total);
  s->budget = (size_t)(o.hbm_fraction * (double)freeb);
  s->budget_cap = o.hbm_budget_bytes;
  if (o.hbm_budget_bytes && o.hbm_budget_bytes < s->budget) s->budget = o.hbm_budget_bytes;
  // policy 0 (size-aware): a quarter of the streams (at least one) form the
  // bulk lane at the lowest priority, the others run at the highest
  int prio_lo = 0, prio_hi = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  s->nbulk = (o.policy == 0 && o.streams >= 2) ? std::max(1, o.streams / 4) : 0;
  for (int i = 0; e == cudaSuccess && i < o.streams; ++i) {
    cudaStream_t st;
    const bool bulk_lane = s->nbulk > 0 && i >= o.streams - s->nbulk;
    e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, s->nbulk == 0 ? 0 : (bulk_lane ? prio_lo : prio_hi));
    if (e == cudaSuccess) s->streams.push_back(st);
  }
  s->lane_work.assign(s->streams.size(), 0.0);
  if (e == cudaSuccess) {
    cudaMemPoolProps pp{};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = dev;
    e = cudaMemPoolCreate(&s->pool, &pp);
  }
  if (e == cudaSuccess) {
    uint64_t keep = UINT64_MAX;  // keep freed workspace in the pool
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    int no = 0;  // no hidden cross-stream dependencies from reuse
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
  }
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    for (auto st : s->streams) cudaStreamDestroy(st);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return cuda_error(e, "fsa_serve_create");
  }
  s->worker = std::thread(loop, s);
  *out = s;
  return FSA_OK;
}

fsa_status fsa_serve_submit(fsa_server* s, const fsa_request* req, uint64_t* ticket) {
  if (!s || !ticket) return set_error(FSA_ERR_INVALID_ARG, "fsa_serve_submit: NULL argument");
  if (!valid_request(req)) return set_error(FSA_ERR_INVALID_ARG, "fsa_serve_submit: invalid request");
  std::lock_guard<std::mutex> lk(s->mu);
  if ((int)s->queue.size() >= s->o.queue_max) return set_error(FSA_ERR_BUSY, "fsa_serve_submit: queue full");
  const uint64_t id = s->next++;
  Req& q = s->reqs[id];
  q.r = *req;
  if (q.r.d == 2) {  // a plane is held as three axes with n[2] = 1
    q.r.n[2] = 1;
    q.r.L[2] = 1.0;
  }
  q.t.submit_s = now_s();
  std::memset(&q.key, 0, sizeof q.key);
  for (int j = 0; j < 3; ++j) {
    q.key.n[j] = q.r.n[j];
    q.key.L[j] = q.r.L[j];
  }
  q.key.kernel = req->kernel;
  q.key.dt = req->dtype;
  q.key.eps = req->eps;
  // Yukawa: 0 selects lam = 1, so both spellings share a plan; other kernels
  // ignore the parameter
  const bool yuk = req->kernel == FSA_KERNEL_YUKAWA3D || req->kernel == FSA_KERNEL_YUKAWA2D;
  q.r.kernel_param = yuk ? (req->kernel_param > 0 ? req->kernel_param : 1.0) : 0.0;
  q.key.param = q.r.kernel_param;
  s->queue.push_back(id);
  s->st.submitted++;
  *ticket = id;
  s->cv_work.notify_one();
  return FSA_OK;
}

fsa_status fsa_serve_poll(fsa_server* s, uint64_t ticket, double timeout_s, fsa_req_state* state,
                          fsa_req_times* times) {
  if (!s) return set_error(FSA_ERR_INVALID_ARG, "fsa_serve_poll: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(FSA_ERR_NOT_FOUND, "fsa_serve_poll: unknown ticket");
  auto finished = [&] {
    auto i = s->reqs.find(ticket);
    return i->second.state == FSA_REQ_DONE || i->second.state == FSA_REQ_FAILED;
  };
  if (timeout_s > 0 && !finished()) {
    if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), finished)) {
      it = s->reqs.find(ticket);
      if (state) *state = it->second.state;
      if (times) *times = it->second.t;
      return set_error(FSA_ERR_TIMEOUT, "fsa_serve_poll: timed out");
    }
  }
  it = s->reqs.find(ticket);
  if (state) *state = it->second.state;
  if (times) *times = it->second.t;
  if (finished()) s->reqs.erase(it);
  return FSA_OK;
}

fsa_status fsa_serve_stats_get(fsa_server* s, fsa_serve_stats* out) {
  if (!s || !out) return set_error(FSA_ERR_INVALID_ARG, "fsa_serve_stats_get: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->device_bytes_held = s->held;
  out->inflight = (int)s->inflight.size();
  out->queued = (int)s->queue.size();
  return FSA_OK;
}

fsa_status fsa_serve_destroy(fsa_server* s) {
  if (!s) return FSA_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (auto st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (auto& kv : s->plans) {
    fsa_plan_destroy(kv.second.plan);
    cudaEventDestroy(kv.second.ready);
  }
  for (auto ev : s->free_events) cudaEventDestroy(ev);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  cudaSetDevice(prev);
  delete s;
  return FSA_OK;
}

}  // extern "C"
