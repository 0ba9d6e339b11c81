// FP32 instantiations of the pair FFT-Poisson passes (complex-float storage).
#include "pair_kernels.cuh"

namespace ace {

bool pair_edge_supported_f32(int n) {
  switch (n) {
    case 8: case 12: case 16: case 20: case 24: case 32: case 36: case 40: case 48: case 64:
      return true;
    default:
      return false;
  }
}

bool launch_pair_batch_f32(const PairLaunch& L, const Batch& b, cudaStream_t st) {
  switch (L.n) {
    case 8: return launch_edge<float, 8>(L, b, st);
    case 12: return launch_edge<float, 12>(L, b, st);
    case 16: return launch_edge<float, 16>(L, b, st);
    case 20: return launch_edge<float, 20>(L, b, st);
    case 24: return launch_edge<float, 24>(L, b, st);
    case 32: return launch_edge<float, 32>(L, b, st);
    case 36: return launch_edge<float, 36>(L, b, st);
    case 40: return launch_edge<float, 40>(L, b, st);
    case 48: return launch_edge<float, 48>(L, b, st);
    case 64: return launch_edge<float, 64>(L, b, st);
    default: return false;
  }
}

}  // namespace ace
