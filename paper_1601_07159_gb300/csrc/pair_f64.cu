// FP64 instantiations of the pair FFT-Poisson passes (complex-double or real
// double storage).
#include "pair_kernels.cuh"

namespace ace {

bool pair_edge_supported_f64(int n) {
  switch (n) {
    case 8: case 12: case 16: case 20: case 24: case 32: case 36: case 40: case 48:
      return true;
    default:
      return false;
  }
}

bool launch_pair_batch_f64(const PairLaunch& L, const Batch& b, cudaStream_t st) {
  switch (L.n) {
    case 8: return launch_edge<double, 8>(L, b, st);
    case 12: return launch_edge<double, 12>(L, b, st);
    case 16: return launch_edge<double, 16>(L, b, st);
    case 20: return launch_edge<double, 20>(L, b, st);
    case 24: return launch_edge<double, 24>(L, b, st);
    case 32: return launch_edge<double, 32>(L, b, st);
    case 36: return launch_edge<double, 36>(L, b, st);
    case 40: return launch_edge<double, 40>(L, b, st);
    case 48: return launch_edge<double, 48>(L, b, st);
    default: return false;
  }
}

int energy_blocks(int n, int npairs, bool f64) {
  (void)f64;
  return (int)(((long long)npairs * n * n + 255) / 256);
}

}  // namespace ace
