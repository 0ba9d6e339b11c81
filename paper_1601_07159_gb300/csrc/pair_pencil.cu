// One (precision, pencil length n_z) instance of pass B, and pass D of the
// cubic grid of that edge. The build compiles
// this file once per compiled length with -DACE_PENCIL_R=<float|double>
// -DACE_PZ=<n_z> -DACE_PENCIL_TAG=<f32_nz|f64_nz> (and again with
// -DACE_RADIX_ORDER=1 -DACE_PENCIL_TAG=f32_nz_r1 for the lengths listed in
// ACE_EDGES_F32_R1); pair_dispatch.cu maps lengths to them.
#include "pair_kernels.cuh"

#if !defined(ACE_PENCIL_R) || !defined(ACE_PZ) || !defined(ACE_PENCIL_TAG)
#error "pair_pencil.cu needs ACE_PENCIL_R, ACE_PZ and ACE_PENCIL_TAG"
#endif
#define ACE_CAT2(a, b) a##b
#define ACE_CAT(a, b) ACE_CAT2(a, b)

namespace ace {

bool ACE_CAT(pencil_launch_, ACE_PENCIL_TAG)(const PairLaunch& L, const Batch& b, cudaStream_t st) {
  return launch_pencil<ACE_PENCIL_R, ACE_PZ>(L, b, st);
}

#if ACE_RADIX_ORDER == 0
// pass D of the cubic grid of this edge (N_g compiled in; no transforms, so
// only the radix-order-0 instance has one)
bool ACE_CAT(point_cube_launch_, ACE_PENCIL_TAG)(const PairLaunch& L, const Batch& b, cudaStream_t st) {
  return launch_point<ACE_PENCIL_R, (long long)ACE_PZ * ACE_PZ * ACE_PZ>(L, b, st);
}
#endif

}  // namespace ace
