// One (precision, cubic edge) instance of the persistent pair engine. The
// build compiles this file once per compiled edge with
// -DACE_EDGE_R=<float|double> -DACE_EDGE_N=<n> -DACE_EDGE_TAG=<f32_n|f64_n>, so
// the instances compile in parallel; pair_dispatch.cu maps n to them.
#include "pair_kernels.cuh"

#if !defined(ACE_EDGE_R) || !defined(ACE_EDGE_N) || !defined(ACE_EDGE_TAG)
#error "pair_edge.cu needs ACE_EDGE_R, ACE_EDGE_N and ACE_EDGE_TAG"
#endif
#define ACE_CAT2(a, b) a##b
#define ACE_CAT(a, b) ACE_CAT2(a, b)

namespace ace {

void ACE_CAT(edge_prepare_, ACE_EDGE_TAG)(EngineInfo& info) { engine_prepare<ACE_EDGE_R, ACE_EDGE_N>(info); }
void ACE_CAT(edge_tasks_, ACE_EDGE_TAG)(const Batch& b, int nt[4]) { engine_tasks<ACE_EDGE_R, ACE_EDGE_N>(b, nt); }
bool ACE_CAT(edge_engine_, ACE_EDGE_TAG)(const PairLaunch& L, const EngineLaunch& E, cudaStream_t st) {
  return launch_engine<ACE_EDGE_R, ACE_EDGE_N>(L, E, st);
}

}  // namespace ace
