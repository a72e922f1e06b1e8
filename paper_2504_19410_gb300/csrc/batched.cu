// fsa_apply_batched: many solves of uneven size in one launch sequence.
//
// The FP32 3-D solves whose transform lengths the mixed-length kernels carry
// (2n in {128, 192, 256, 384, 512}: the 64^3 ... 256^3 grids of the batched
// workload) run as five launches in all: each pass is ONE persistent launch
// over the concatenated tile lists of all of them, whatever their sizes
// (mixed.cu, passes_mix.cuh).  The other solves (FP64, planes, DDI, other
// lengths) form groups of one grid and dtype; each pass of a group is
// one persistent launch that walks the tiles of all the group's solves (the
// kernels take a by-value job table), and the groups run on forked streams so
// their passes overlap on the device.  Either sequence is captured once per
// batch signature (plans, buffers) into a CUDA graph and replayed, so a
// repeated batch costs one graph launch on the caller's stream.  The
// signature includes the kernel-selection generation, so a batch replayed
// after fsa_autotune_set, fsa_fused_select or fsa_pipe_select is captured
// again with the new kernels.
#include <algorithm>
#include <tuple>
#include <list>
#include <map>
#include <mutex>
#include <set>
#include <vector>

#include "fsa_internal.h"

namespace fsa {
namespace {

struct GroupKey {
  int n0, n1, n2, dt, dw, ddi;
  bool operator<(const GroupKey& o) const {
    return std::tie(n0, n1, n2, dt, dw, ddi) < std::tie(o.n0, o.n1, o.n2, o.dt, o.dw, o.ddi);
  }
};

struct Sig {
  std::vector<const void*> v;
  bool operator<(const Sig& o) const { return v < o.v; }
  bool operator==(const Sig& o) const { return v == o.v; }
};

struct DeviceCtx {
  cudaStream_t capture = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;
  std::map<Sig, cudaGraphExec_t> graphs;
  std::list<Sig> lru;  // front = most recent
};

std::mutex g_mu;
std::map<int, DeviceCtx> g_ctx;
constexpr size_t kMaxGraphs = 32;

cudaError_t ensure_ctx(DeviceCtx& c, size_t groups) {
  cudaError_t e = cudaSuccess;
  if (!c.capture) e = cudaStreamCreateWithFlags(&c.capture, cudaStreamNonBlocking);
  while (e == cudaSuccess && c.side.size() < groups) {
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) c.side.push_back(s);
  }
  while (e == cudaSuccess && c.ev.size() < 2 * groups + 2) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) c.ev.push_back(ev);
  }
  return e;
}

cudaError_t launch_group(const std::vector<int>& idx, const fsa_plan* const* plans, const void* const* rho,
                         void* const* phi, cudaStream_t s) {
  const fsa_plan* p0 = plans[idx[0]];
  std::vector<const void*> r, S;
  std::vector<void*> f, X, Y;
  std::vector<const DdiPar*> par;
  for (int k : idx) {
    const fsa_plan* p = plans[k];
    r.push_back(rho[k]);
    f.push_back(phi[k]);
    X.push_back(p->ws);
    Y.push_back((char*)p->ws + p->x_bytes);
    S.push_back(plan_apply_spectrum(p));
    par.push_back(p->ddi_par);
  }
  return run_group(p0, (int)idx.size(), r.data(), f.data(), X.data(), Y.data(), S.data(), s, nullptr, par.data());
}

// Schedule chosen for a list of plans (auto mode's pick, or the forced one),
// for fsa_apply_batched_launches.
std::map<std::vector<const void*>, int> g_choice;

// Capture one batch into an executable graph.  sched 1: the mixed-length
// requests in one launch per pass (mixed.cu), the rest in shape groups on side
// streams; 3: the same with the mixed requests pipelined in two halves; 2: every
// request in its shape group (one persistent launch per pass per group, the
// groups on concurrent streams).
cudaError_t capture_batch(DeviceCtx& c, int count, const fsa_plan* const* plans, const void* const* rho,
                          void* const* phi, int sched, cudaGraphExec_t* exec) {
  std::map<GroupKey, std::vector<int>> groups;
  std::vector<const fsa_plan*> mplans;
  std::vector<const void*> mrho;
  std::vector<void*> mphi;
  for (int k = 0; k < count; ++k) {
    const fsa_plan* p = plans[k];
    if (sched != 2 && mixed_eligible(p)) {
      mplans.push_back(p);
      mrho.push_back(rho[k]);
      mphi.push_back(phi[k]);
    } else {
      groups[GroupKey{p->n[0], p->n[1], p->n[2], (int)p->dtype, p->f64_dw, p->ddi}].push_back(k);
    }
  }
  const bool mixed = !mplans.empty();
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c.capture, cudaStreamCaptureModeThreadLocal);
  // the mixed launches on the capture stream; every group on a side stream
  size_t g = mixed ? 1 : 0;
  cudaError_t le = e;
  if (mixed && le == cudaSuccess)
    le = mixed_passes((int)mplans.size(), mplans.data(), mrho.data(), mphi.data(), c.capture, sched == 3);
  for (auto& kv : groups) {
    if (le != cudaSuccess) break;
    if (g == 0) {
      le = launch_group(kv.second, plans, rho, phi, c.capture);
    } else {
      cudaStream_t s = c.side[g - 1];
      le = cudaEventRecord(c.ev[2 * g], c.capture);
      if (le == cudaSuccess) le = cudaStreamWaitEvent(s, c.ev[2 * g], 0);
      if (le == cudaSuccess) le = launch_group(kv.second, plans, rho, phi, s);
      if (le == cudaSuccess) le = cudaEventRecord(c.ev[2 * g + 1], s);
      if (le == cudaSuccess) le = cudaStreamWaitEvent(c.capture, c.ev[2 * g + 1], 0);
    }
    ++g;
  }
  if (e == cudaSuccess) e = cudaStreamEndCapture(c.capture, &graph);
  if (e == cudaSuccess) e = le;
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  return e;
}

}  // namespace
}  // namespace fsa

using namespace fsa;

extern "C" fsa_status fsa_apply_batched(const fsa_plan* const* plans, const void* const* rho, void* const* phi,
                                        int count, fsa_stream_t stream) {
  if (count < 0 || (count > 0 && (!plans || !rho || !phi)))
    return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_batched: bad arguments");
  if (count == 0) return FSA_OK;
  const int dev = plans[0] ? plans[0]->device : -1;
  std::vector<const fsa_plan*> seen;
  for (int k = 0; k < count; ++k) {
    const fsa_plan* p = plans[k];
    if (!p || !rho[k] || !phi[k]) return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_batched: NULL entry");
    if (p->device != dev) return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_batched: plans on different devices");
    if (!p->generated) return set_error(FSA_ERR_NOT_GENERATED, "fsa_apply_batched: plan not generated");
    if (((uintptr_t)rho[k] | (uintptr_t)phi[k]) & 15u)
      return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_batched: rho and phi must be 16-byte aligned");
    seen.push_back(p);
  }
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
    return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_batched: a plan appears twice (its workspace is shared)");
  int eligible = 0;
  for (int k = 0; k < count; ++k) eligible += mixed_eligible(plans[k]) ? 1 : 0;
  const int mode = batched_mode();
  // schedules: 1 = mixed, one launch per pass; 2 = shape groups; 3 = mixed,
  // pipelined halves.  Mode 0 (auto) times 1 and 2 on the first call of a
  // batch signature and keeps the faster.
  const int fixed = eligible == 0 ? 2 : (mode == 0 ? 0 : mode);

  Sig sig;
  sig.v.push_back(reinterpret_cast<const void*>((uintptr_t)mode));  // the mode shapes the graph
  // so do the kernels selected for each length: a selection change
  // (fsa_autotune_set, fsa_fused_select, fsa_pipe_select) starts new captures
  sig.v.push_back(reinterpret_cast<const void*>((uintptr_t)(unsigned)apply_graphs_generation()));
  std::vector<const void*> pkey;
  for (int k = 0; k < count; ++k) {
    sig.v.push_back(plans[k]);
    sig.v.push_back(rho[k]);
    sig.v.push_back(phi[k]);
    pkey.push_back(plans[k]);
  }

  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != dev) cudaSetDevice(dev);
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceCtx& c = g_ctx[dev];
  std::set<GroupKey> shapes;  // an upper bound on the groups any schedule forms
  for (int k = 0; k < count; ++k) {
    const fsa_plan* p = plans[k];
    shapes.insert(GroupKey{p->n[0], p->n[1], p->n[2], (int)p->dtype, p->f64_dw, p->ddi});
  }
  cudaError_t e = ensure_ctx(c, shapes.size() + 1);
  cudaGraphExec_t exec = nullptr;
  auto it = c.graphs.find(sig);
  if (e == cudaSuccess && it != c.graphs.end()) {
    exec = it->second;
    c.lru.remove(sig);
    c.lru.push_front(sig);
  } else if (e == cudaSuccess) {
    if (fixed != 0) {
      e = capture_batch(c, count, plans, rho, phi, fixed, &exec);
      if (e == cudaSuccess) g_choice[pkey] = fixed;
    } else {
      // auto: both candidates, each launched twice on the caller's stream (the
      // second launch timed), the faster kept and launched once more below, so
      // this call's results are the kept schedule's
      cudaGraphExec_t cand[2] = {nullptr, nullptr};
      const int sched[2] = {1, 2};
      float ms[2] = {1e30f, 1e30f};
      cudaEvent_t t0 = nullptr, t1 = nullptr;
      e = cudaEventCreate(&t0);
      if (e == cudaSuccess) e = cudaEventCreate(&t1);
      for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = capture_batch(c, count, plans, rho, phi, sched[i], &cand[i]);
        if (e == cudaSuccess) e = cudaGraphLaunch(cand[i], (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaEventRecord(t0, (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(cand[i], (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaEventRecord(t1, (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[i], t0, t1);
      }
      if (t0) cudaEventDestroy(t0);
      if (t1) cudaEventDestroy(t1);
      const int win = ms[0] <= ms[1] ? 0 : 1;
      if (cand[1 - win]) cudaGraphExecDestroy(cand[1 - win]);
      exec = cand[win];
      if (e == cudaSuccess) g_choice[pkey] = sched[win];
    }
    if (e == cudaSuccess) {
      c.graphs[sig] = exec;
      c.lru.push_front(sig);
      while (c.lru.size() > kMaxGraphs) {
        cudaGraphExecDestroy(c.graphs[c.lru.back()]);
        c.graphs.erase(c.lru.back());
        c.lru.pop_back();
      }
    }
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, (cudaStream_t)stream);
  if (prev != dev) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_error(e, "fsa_apply_batched");
  }
  return FSA_OK;
}

extern "C" fsa_status fsa_batched_mode_set(int mode) {
  if (mode < 0 || mode > 3) return set_error(FSA_ERR_INVALID_ARG, "fsa_batched_mode_set: mode must be 0 .. 3");
  batched_mode() = mode;
  return FSA_OK;
}

extern "C" fsa_status fsa_apply_batched_launches(const fsa_plan* const* plans, int count, int* launches) {
  if (!launches || count < 0 || (count > 0 && !plans))
    return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_batched_launches: bad arguments");
  int mixed = 0;
  std::map<GroupKey, std::pair<int, int>> groups;  // members, launches per apply
  // the schedule: forced by the mode, else auto mode's pick for these plans
  // once a batch of them has run, else the mixed path (its first candidate)
  int sched = batched_mode();
  if (sched == 0) {
    std::lock_guard<std::mutex> lk(g_mu);
    std::vector<const void*> pkey(plans, plans + count);
    auto it = g_choice.find(pkey);
    sched = it != g_choice.end() ? it->second : 1;
  }
  for (int k = 0; k < count; ++k) {
    const fsa_plan* p = plans[k];
    if (!p) return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_batched_launches: NULL plan");
    if (sched != 2 && mixed_eligible(p)) {
      ++mixed;
    } else {
      auto& g = groups[GroupKey{p->n[0], p->n[1], p->n[2], (int)p->dtype, p->f64_dw, p->ddi}];
      ++g.first;
      fsa_plan_info info{};
      fsa_plan_info_get(p, &info);
      g.second = info.launches_per_apply;
    }
  }
  int n = mixed_launches(mixed, sched == 3);
  for (auto& kv : groups) n += kv.second.second * ((kv.second.first + kMaxJobs - 1) / kMaxJobs);
  *launches = n;
  return FSA_OK;
}

// Graphs hold plan pointers and workspace addresses: drop any that mention a
// plan about to be destroyed.
namespace fsa {
void batched_forget_plan(const fsa_plan* p) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& dc : g_ctx) {
    DeviceCtx& c = dc.second;
    for (auto it = c.lru.begin(); it != c.lru.end();) {
      bool uses = false;
      for (size_t i = 1; i < it->v.size(); i += 3) uses |= (it->v[i] == p);  // v = mode, then (plan, rho, phi)...
      if (uses) {
        cudaGraphExecDestroy(c.graphs[*it]);
        std::vector<const void*> pkey;
        for (size_t i = 1; i < it->v.size(); i += 3) pkey.push_back(it->v[i]);
        g_choice.erase(pkey);
        c.graphs.erase(*it);
        it = c.lru.erase(it);
      } else {
        ++it;
      }
    }
  }
}
}  // namespace fsa
