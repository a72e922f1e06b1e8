// fsa_profiler_*: per-pass CUDA-event timing of the apply path.
#include <vector>

#include "fsa_internal.h"

struct fsa_profiler {
  int max_steps = 0;
  int steps = 0;
  int device = 0;
  std::vector<cudaEvent_t> ev;  // 6 per step
};

namespace fsa {
// The five passes of one plan with an event before and after each (plan.cu).
cudaError_t plan_apply_passes_events(const fsa_plan* p, const void* rho, void* phi, cudaStream_t s,
                                     cudaEvent_t* ev6);
}  // namespace fsa

using namespace fsa;

extern "C" {

fsa_status fsa_profiler_create(fsa_profiler** out, int max_steps) {
  if (!out || max_steps <= 0) return set_error(FSA_ERR_INVALID_ARG, "fsa_profiler_create: bad arguments");
  *out = nullptr;
  fsa_profiler* p = new fsa_profiler();
  p->max_steps = max_steps;
  cudaGetDevice(&p->device);
  p->ev.resize((size_t)6 * max_steps);
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
  cudaError_t e =
      plan_apply_passes_events(plan, rho, phi, (cudaStream_t)stream, &prof->ev[(size_t)6 * prof->steps]);
  if (prev != plan->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_error(e, "fsa_apply_profiled");
  prof->steps++;
  return FSA_OK;
}

fsa_status fsa_profiler_read(fsa_profiler* prof, double* pass_ms, double* step_ms, int* steps) {
  if (!prof) return set_error(FSA_ERR_INVALID_ARG, "fsa_profiler_read: NULL profiler");
  double acc[5] = {0, 0, 0, 0, 0}, tot = 0;
  const int n = prof->steps;
  for (int k = 0; k < n; ++k) {
    cudaEvent_t* e = &prof->ev[(size_t)6 * k];
    cudaError_t r = cudaEventSynchronize(e[5]);
    for (int i = 0; i < 5 && r == cudaSuccess; ++i) {
      float ms = 0;
      r = cudaEventElapsedTime(&ms, e[i], e[i + 1]);
      acc[i] += ms;
    }
    float all = 0;
    if (r == cudaSuccess) r = cudaEventElapsedTime(&all, e[0], e[5]);
    if (r != cudaSuccess) return cuda_error(r, "fsa_profiler_read");
    tot += all;
  }
  for (int i = 0; i < 5; ++i)
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
