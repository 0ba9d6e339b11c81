// Pass D (the accumulate pass), which depends on the grid only through N_g:
// one instance per precision for any grid (the cubic ones, with N_g compiled
// in, live beside pass B in pair_pencil.cu).
#include "pair_kernels.cuh"

namespace ace {

bool launch_point_f32(const PairLaunch& L, const Batch& b, cudaStream_t st) { return launch_point<float, 0>(L, b, st); }
bool launch_point_f64(const PairLaunch& L, const Batch& b, cudaStream_t st) { return launch_point<double, 0>(L, b, st); }

}  // namespace ace
