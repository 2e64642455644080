// prof.cu -- launch counting and optional CUDA-event timing per stage of the path.
#include "ctd_internal.cuh"

namespace ctd {

static thread_local ProfState* g_prof = nullptr;

void prof_bind(ProfState* p) { g_prof = p; }
int prof_stage() { return g_prof ? g_prof->stage : STG_MISC; }
void prof_set_stage(int s) {
  if (g_prof) g_prof->stage = s;
}
bool prof_recording() { return g_prof && g_prof->on; }
// kernels launched by a CUDA graph replay, counted like individual launches (current stage)
void prof_count_launches(int64_t k) {
  if (g_prof) g_prof->launches[g_prof->stage] += k;
}

static cudaEvent_t take_event(ProfState* p) {
  if (!p->pool.empty()) {
    cudaEvent_t e = p->pool.back();
    p->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

LaunchScope::LaunchScope(cudaStream_t s) : st(s) {
  if (!g_prof) return;
  g_prof->launches[g_prof->stage]++;
  if (g_prof->on) {
    a = take_event(g_prof);
    cudaEventRecord(a, st);
  }
}

LaunchScope::~LaunchScope() {
  if (!g_prof || !a) return;
  cudaEvent_t b = take_event(g_prof);
  cudaEventRecord(b, st);
  g_prof->pending.push_back({g_prof->stage, a, b});
}

void ProfState::collect() {
  for (const Rec& r : pending) {
    float ms_ = 0.0f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&ms_, r.a, r.b);
    ms[r.stage] += ms_;
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  pending.clear();
}

ProfState::~ProfState() {
  collect();
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

}  // namespace ctd
