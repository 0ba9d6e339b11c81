// One (precision, plane n_x x n_y) instance of the plane passes A and C. The
// build compiles this file once per compiled plane with
// -DACE_PLANE_R=<float|double> -DACE_PX=<n_x> -DACE_PY=<n_y>
// -DACE_PLANE_TAG=<f32_nx_ny|f64_nx_ny> (and FP32 planes again with
// -DACE_RADIX_ORDER=1 -DACE_PLANE_TAG=f32_nx_ny_r1); pair_dispatch.cu maps
// planes to them.
#include "pair_kernels.cuh"

#if !defined(ACE_PLANE_R) || !defined(ACE_PX) || !defined(ACE_PY) || !defined(ACE_PLANE_TAG)
#error "pair_plane.cu needs ACE_PLANE_R, ACE_PX, ACE_PY and ACE_PLANE_TAG"
#endif
#define ACE_CAT2(a, b) a##b
#define ACE_CAT(a, b) ACE_CAT2(a, b)

namespace ace {

bool ACE_CAT(plane_launch_, ACE_PLANE_TAG)(const PairLaunch& L, const Batch& b, int pass, cudaStream_t st) {
  return launch_plane<ACE_PLANE_R, ACE_PX, ACE_PY>(L, b, pass, st);
}

}  // namespace ace
