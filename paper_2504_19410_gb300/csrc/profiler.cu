// fsa_profiler_*: per-pass CUDA-event timing of the apply path.
//
// Every launch of a profiled solve is followed by an event on the launching
// stream, tagged with its pass; when the middle passes run in plane slabs a
// pass has several launches and its time is their sum.
#include <vector>

#include "fsa_internal.h"

namespace {
constexpr int kEvPerStep = 512;
}

struct fsa_profiler {
  int max_steps = 0;
  int steps = 0;
  int device = 0;
  std::vector<cudaEvent_t> ev;     // kEvPerStep per step
  std::vector<signed char> kind;   // pass of the interval ending at event i+1
  std::vector<int> used;           // events recorded per step
};

namespace fsa {
cudaError_t plan_apply_passes_trace(const fsa_plan* p, const void* rho, void* phi, cudaStream_t s, PassTrace* tr);
}  // namespace fsa

using namespace fsa;

extern "C" {

fsa_status fsa_profiler_create(fsa_profiler** out, int max_steps) {
  if (!out || max_steps <= 0 || max_steps > 4096)
    return set_error(FSA_ERR_INVALID_ARG, "fsa_profiler_create: max_steps must be in [1, 4096]");
  *out = nullptr;
  fsa_profiler* p = new fsa_profiler();
  p->max_steps = max_steps;
  cudaGetDevice(&p->device);
  p->ev.assign((size_t)kEvPerStep * max_steps, nullptr);
  p->kind.assign((size_t)kEvPerStep * max_steps, -1);
  p->used.assign(max_steps, 0);
  for (auto& e : p->ev) {
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) {
      e = nullptr;
      fsa_profiler_destroy(p);
      return cuda_error(r, "fsa_profiler_create");
    }
  }
  *out = p;
  return FSA_OK;
}

fsa_status fsa_apply_profiled(const fsa_plan* plan, const void* rho, void* phi, fsa_stream_t stream,
                              fsa_profiler* prof) {
  if (!plan || !rho || !phi || !prof) return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_profiled: NULL argument");
  if (!plan->generated) return set_error(FSA_ERR_NOT_GENERATED, "fsa_apply_profiled: not generated");
  if (!plan->ws) return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_profiled: plan has no workspace");
  if (prof->steps >= prof->max_steps) return set_error(FSA_ERR_BUSY, "fsa_apply_profiled: profiler full");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != plan->device) cudaSetDevice(plan->device);
  PassTrace tr;
  tr.ev = &prof->ev[(size_t)kEvPerStep * prof->steps];
  tr.kind = &prof->kind[(size_t)kEvPerStep * prof->steps];
  tr.cap = kEvPerStep;
  cudaError_t e = plan_apply_passes_trace(plan, rho, phi, (cudaStream_t)stream, &tr);
  if (prev != plan->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_error(e, "fsa_apply_profiled");
  prof->used[prof->steps] = tr.used;
  prof->steps++;
  return FSA_OK;
}

fsa_status fsa_profiler_read(fsa_profiler* prof, double* pass_ms, double* step_ms, int* steps) {
  if (!prof) return set_error(FSA_ERR_INVALID_ARG, "fsa_profiler_read: NULL profiler");
  double acc[kNumPass] = {0, 0, 0, 0, 0}, tot = 0;
  const int n = prof->steps;
  for (int k = 0; k < n; ++k) {
    cudaEvent_t* e = &prof->ev[(size_t)kEvPerStep * k];
    const signed char* kd = &prof->kind[(size_t)kEvPerStep * k];
    const int u = prof->used[k];
    if (u < 2) continue;
    cudaError_t r = cudaEventSynchronize(e[u - 1]);
    for (int i = 0; i + 1 < u && r == cudaSuccess; ++i) {
      float ms = 0;
      r = cudaEventElapsedTime(&ms, e[i], e[i + 1]);
      if (kd[i] >= 0 && kd[i] < kNumPass) acc[(int)kd[i]] += ms;
    }
    float all = 0;
    if (r == cudaSuccess) r = cudaEventElapsedTime(&all, e[0], e[u - 1]);
    if (r != cudaSuccess) return cuda_error(r, "fsa_profiler_read");
    tot += all;
  }
  for (int i = 0; i < kNumPass; ++i)
    if (pass_ms) pass_ms[i] = n ? acc[i] / n : 0.0;
  if (step_ms) *step_ms = n ? tot / n : 0.0;
  if (steps) *steps = n;
  prof->steps = 0;
  return FSA_OK;
}

fsa_status fsa_profiler_destroy(fsa_profiler* prof) {
  if (!prof) return FSA_OK;
  for (auto e : prof->ev)
    if (e) cudaEventDestroy(e);
  delete prof;
  return FSA_OK;
}

}  // extern "C"
