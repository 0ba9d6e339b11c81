// FP64 Cholesky factorisation of -M and the in-place triangular inverse
// (Sec. 3: -M = L L^*, then Xi = W L^{-*} of Eq. Wtilde).
//
// One CTA of 1024 threads. The lower triangle is held packed, row-major
// (element (i, k), k <= i, at i(i+1)/2 + k), in shared memory when it fits
// (N <= 159: N(N+1)/2 complex doubles <= 200 KB), else in the plan's global
// work buffer. Both steps are right-looking with one barrier per column:
//   Cholesky  j = 0..N-1: pivot d = A_jj (real), L_jj = sqrt(d), L_ij = A_ij / L_jj,
//             A_ik -= L_ij conj(L_kj) for j < k <= i;
//   inverse   j = N-1..0: X_jj = 1/L_jj, X(j+1:, j) = -X_jj X(j+1:, j+1:) L(j+1:, j)
//             (the trailing block already holds its inverse), the textbook
//             column-by-column form of the inverse of a triangular matrix.
// A non-finite or non-positive pivot writes the status word and stops.
// Output: LinvH[c][i] = conj(X_ic) (row-major N x N, zero above), so that
// Xi_k = sum_i W_i LinvH[i][k].
#include <cmath>

#include "ace_internal.h"

namespace ace {

namespace {

struct Cpx { double x, y; };

__device__ __forceinline__ long long tri(int i, int k) { return (long long)i * (i + 1) / 2 + k; }

template <bool SMEM>
__global__ void __launch_bounds__(1024)
chol_inv_kernel(const double* __restrict__ M, int n, Cpx* __restrict__ gA, double* __restrict__ LinvH,
                int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int fail;
  __shared__ Cpx col[1024];
  Cpx* A = SMEM ? reinterpret_cast<Cpx*>(smem_raw) : gA;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  // A = -M (lower triangle, packed)
  for (long long e = tid; e < (long long)n * n; e += nt) {
    const int i = (int)(e / n), k = (int)(e % n);
    if (k <= i) A[tri(i, k)] = Cpx{-M[2 * e], -M[2 * e + 1]};
  }
  if (tid == 0) fail = 0;
  __syncthreads();
  // ---- Cholesky
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const double d = A[tri(j, j)].x;
      if (!isfinite(d)) {
        fail = 1; status[0] = -3; status[1] = j + 1;
      } else if (!(d > 0.0)) {
        fail = 1; status[0] = -2; status[1] = j + 1;
      } else {
        A[tri(j, j)] = Cpx{sqrt(d), 0.0};
      }
    }
    __syncthreads();
    if (fail) return;
    const double inv = 1.0 / A[tri(j, j)].x;
    for (int i = j + 1 + tid; i < n; i += nt) {
      Cpx v = A[tri(i, j)];
      v.x *= inv; v.y *= inv;
      A[tri(i, j)] = v;
      col[i] = v;
    }
    __syncthreads();
    for (int i = j + 1 + warp; i < n; i += nwarps) {
      const Cpx a = col[i];
      for (int k = j + 1 + lane; k <= i; k += 32) {
        const Cpx b = col[k];
        Cpx& t = A[tri(i, k)];
        t.x -= a.x * b.x + a.y * b.y;     // A_ik -= L_ij conj(L_kj)
        t.y -= a.y * b.x - a.x * b.y;
      }
    }
    __syncthreads();
  }
  // ---- inverse, in place
  for (int j = n - 1; j >= 0; --j) {
    const double xjj = 1.0 / A[tri(j, j)].x;
    for (int i = j + 1 + tid; i < n; i += nt) col[i] = A[tri(i, j)];   // L(j+1:, j)
    __syncthreads();
    for (int i = j + 1 + warp; i < n; i += nwarps) {
      double sr = 0.0, si = 0.0;
      for (int k = j + 1 + lane; k <= i; k += 32) {
        const Cpx x = A[tri(i, k)], l = col[k];
        sr += x.x * l.x - x.y * l.y;
        si += x.x * l.y + x.y * l.x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o);
        si += __shfl_down_sync(0xffffffffu, si, o);
      }
      if (lane == 0) A[tri(i, j)] = Cpx{-xjj * sr, -xjj * si};
    }
    if (tid == 0) A[tri(j, j)] = Cpx{xjj, 0.0};
    __syncthreads();
  }
  // ---- LinvH[c][i] = conj(X_ic)
  for (long long e = tid; e < (long long)n * n; e += nt) {
    const int c = (int)(e / n), i = (int)(e % n);
    Cpx v{0.0, 0.0};
    if (i >= c) v = A[tri(i, c)];
    LinvH[2 * e] = v.x;
    LinvH[2 * e + 1] = -v.y;
  }
}

}  // namespace

void prepare_cholesky(int n) {
  const size_t packed = (size_t)n * (n + 1) / 2 * sizeof(Cpx);
  if (packed <= 200 * 1024)
    cudaFuncSetAttribute(chol_inv_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)packed);
}

__global__ void scale_kernel_f(float* x, long long count, float s) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    x[i] *= s;
}
__global__ void scale_kernel_d(double* x, long long count, double s) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    x[i] *= s;
}

// X *= s over `count` stored vector elements (real and imaginary parts alike).
void launch_scale(bool f64, bool real, void* X, long long count, double s, cudaStream_t st) {
  const long long nreal = real ? count : 2 * count;
  const unsigned grid = (unsigned)((nreal + 255) / 256 < 152 * 16 ? (nreal + 255) / 256 : 152 * 16);
  if (f64) scale_kernel_d<<<grid, 256, 0, st>>>(static_cast<double*>(X), nreal, s);
  else scale_kernel_f<<<grid, 256, 0, st>>>(static_cast<float*>(X), nreal, (float)s);
}

void launch_cholesky_inv(const double* M, int n, double* work, double* LinvH, int* status,
                         cudaStream_t st) {
  const size_t packed = (size_t)n * (n + 1) / 2 * sizeof(Cpx);
  if (n <= 1024 && packed <= 200 * 1024) {
    chol_inv_kernel<true><<<1, 1024, packed, st>>>(M, n, nullptr, LinvH, status);
  } else {
    chol_inv_kernel<false><<<1, 1024, 0, st>>>(M, n, reinterpret_cast<Cpx*>(work), LinvH, status);
  }
}

}  // namespace ace
