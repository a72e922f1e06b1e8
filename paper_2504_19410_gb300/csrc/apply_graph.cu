// Repeated single solves through cached CUDA graphs.
//
// fsa_apply and fsa_apply_host launch the five passes of Sec. 2.3 (three
// for a plane, ten for the DDI grid reading).  Launched one by one, each
// kernel waits for the device front end between passes; replaying the same
// launches as one captured graph cuts that gap (measured on a GB300 at
// 256^3 FP32: 0.453 ms per solve launched directly, 0.442 ms replayed).  A
// solve's launches depend only on its plan, its buffers and the kernels
// selected for its transform lengths, so the graph of a (plan, rho, phi)
// triple is captured on the SECOND call with that triple (a single call
// costs nothing extra) and replayed from then on.  Selection changes
// (fsa_autotune_set, fsa_fused_select, fsa_pipe_select) bump a generation
// that is part of every graph key (here and in fsa_apply_batched), so they
// start new captures; a plan's graphs are dropped when it is destroyed.
#include <atomic>
#include <list>
#include <map>
#include <mutex>
#include <set>
#include <tuple>

#include "fsa_internal.h"

namespace fsa {
namespace {

struct Key {
  const fsa_plan* p;
  const void* rho;
  void* phi;
  int gen;   // selection generation at capture
  int grid;  // the calling thread's launch_grid_mode
  bool operator<(const Key& o) const { return std::tie(p, rho, phi, gen, grid) < std::tie(o.p, o.rho, o.phi, o.gen, o.grid); }
  bool operator==(const Key& o) const { return !(*this < o) && !(o < *this); }
};

struct DeviceCtx {
  cudaStream_t capture = nullptr;
  std::map<Key, cudaGraphExec_t> graphs;
  std::list<Key> lru;  // front = most recent
  std::set<Key> seen;  // triples called once, not captured yet
};

std::mutex g_mu;
std::map<int, DeviceCtx> g_ctx;
std::atomic<int> g_gen{0};
std::atomic<int> g_enabled{1};
constexpr size_t kMaxGraphs = 64;   // per device; the least recently used is dropped
constexpr size_t kMaxSeen = 4096;  // triples remembered before their second call

}  // namespace

void apply_graphs_invalidate() { g_gen.fetch_add(1); }

int apply_graphs_generation() { return g_gen.load(); }

void apply_graphs_forget_plan(const fsa_plan* p) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& kv : g_ctx) {
    DeviceCtx& c = kv.second;
    for (auto it = c.graphs.begin(); it != c.graphs.end();) {
      if (it->first.p == p) {
        // an executable graph still in flight is freed when it completes
        cudaGraphExecDestroy(it->second);
        c.lru.remove(it->first);
        it = c.graphs.erase(it);
      } else {
        ++it;
      }
    }
    for (auto it = c.seen.begin(); it != c.seen.end();) it = it->p == p ? c.seen.erase(it) : std::next(it);
  }
}

// The passes of plan p from rho to phi on stream s: by a graph replay when
// this triple has been seen before, else launched directly.
cudaError_t plan_apply_graph(const fsa_plan* p, const void* rho, void* phi, cudaStream_t s) {
  if (!g_enabled.load()) return plan_apply_passes(p, rho, phi, s);
  // a caller capturing its own stream into a graph gets the launches
  // themselves (no capture or instantiation of ours inside its capture)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return plan_apply_passes(p, rho, phi, s);
  }
  const Key key{p, rho, phi, g_gen.load(), launch_grid_mode()};
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaSuccess;
  {
    // held through the graph launch: another thread's capture may evict
    // (destroy) this executable graph as soon as the lock is released
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceCtx& c = g_ctx[p->device];
    auto it = c.graphs.find(key);
    if (it != c.graphs.end()) {
      exec = it->second;
      c.lru.remove(key);
      c.lru.push_front(key);
    } else if (c.seen.count(key)) {
      // second call: capture the launches (nothing runs during a capture)
      if (!c.capture) e = cudaStreamCreateWithFlags(&c.capture, cudaStreamNonBlocking);
      cudaGraph_t graph = nullptr;
      if (e == cudaSuccess) e = cudaStreamBeginCapture(c.capture, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const cudaError_t le = plan_apply_passes(p, rho, phi, c.capture);
        e = cudaStreamEndCapture(c.capture, &graph);
        if (e == cudaSuccess) e = le;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e == cudaSuccess) {
        c.seen.erase(key);
        c.graphs[key] = exec;
        c.lru.push_front(key);
        while (c.lru.size() > kMaxGraphs) {
          cudaGraphExecDestroy(c.graphs[c.lru.back()]);
          c.graphs.erase(c.lru.back());
          c.lru.pop_back();
        }
      } else {
        cudaGetLastError();
        exec = nullptr;
        e = cudaSuccess;  // fall back to direct launches below
      }
    } else {
      if (c.seen.size() >= kMaxSeen) c.seen.clear();
      c.seen.insert(key);
    }
    if (exec) return cudaGraphLaunch(exec, s);
  }
  return plan_apply_passes(p, rho, phi, s);
}

}  // namespace fsa

extern "C" fsa_status fsa_apply_graphs_set(int enable) {
  if (enable != 0 && enable != 1) return fsa::set_error(FSA_ERR_INVALID_ARG, "fsa_apply_graphs_set: enable must be 0 or 1");
  fsa::g_enabled.store(enable);
  return FSA_OK;
}
