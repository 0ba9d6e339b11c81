// FP64 Cholesky factorisation of -M and the inverse of its factor (Sec. 3:
// -M = L L^*, then Xi = W L^{-*} of Eq. Wtilde), blocked so that the FP64 work
// spreads over many SMs (FP64 throughput per SM is low on this part).
//
// Blocks of NB = 32 columns. For panel p (rows/cols [p0, p0 + nb)):
//   diag    one CTA: A_pp -> L_pp (right-looking Cholesky in shared memory,
//           status word on a non-finite or non-positive pivot), D_p = L_pp^{-1}
//           (column-by-column inverse of a triangular matrix); L_pp is stored
//           in A, D_p in the diagonal block of X.
//   panel   L_ip = A_ip D_p^*  for every row i below the panel (one CTA per 16
//           rows, in place: a CTA reads and writes only its own rows).
//   update  A_ik -= sum_l L_il conj(L_kl) over the panel columns l, for the
//           trailing lower triangle i >= k (16 x 16 output tiles).
// Then the block rows of X = L^{-1} below the diagonal, in order q = 1..P-1:
//   T     = L(q, 0:q) X(0:q, 0:q)        (block-row product, X lower triangular)
//   X(q, 0:q) = -D_q T
// and finally LinvH[c][i] = conj(X_ic) (zero above the diagonal), so that
// Xi_k = sum_i W_i LinvH[i][k].
// Every kernel returns at once when the status word already holds a failure.
#include <cmath>

#include "ace_internal.h"

namespace ace {

namespace {

constexpr int NB = 32;   // panel width
constexpr int TT = 16;   // output tile edge of the FP64 tile products

__device__ __forceinline__ double2 zfma(double2 acc, double2 a, double2 b) {   // acc + a b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 zfmac(double2 acc, double2 a, double2 b) {  // acc + a conj(b)
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.y, b.x, acc.y);
  acc.y = fma(-a.x, b.y, acc.y);
  return acc;
}

__global__ void neg_copy_kernel(const double2* __restrict__ M, long long count, double2* __restrict__ A) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) A[i] = make_double2(-M[i].x, -M[i].y);
}

// Factor and invert the diagonal block of panel p (nb <= NB).
__global__ void __launch_bounds__(1024)
diag_kernel(double2* __restrict__ A, double2* __restrict__ X, int n, int p0, int nb, int* status) {
  __shared__ double2 a[NB][NB + 1];
  __shared__ double2 col[NB];
  __shared__ int fail;
  __shared__ double rcp;   // one FP64 reciprocal per step, shared (FP64 division is costly here)
  const int tid = threadIdx.x;
  if (status[0] != 0) return;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int i = e / NB, k = e % NB;
    a[i][k] = (i < nb && k <= i) ? A[(long long)(p0 + i) * n + p0 + k] : make_double2(0.0, 0.0);
  }
  if (tid == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      const double d = a[j][j].x;
      if (!isfinite(d)) {
        fail = 1; status[0] = -3; status[1] = p0 + j + 1;
      } else if (!(d > 0.0)) {
        fail = 1; status[0] = -2; status[1] = p0 + j + 1;
      } else {
        const double l = sqrt(d);
        a[j][j] = make_double2(l, 0.0);
        rcp = 1.0 / l;
      }
    }
    __syncthreads();
    if (fail) return;
    const double inv = rcp;
    if (tid > j && tid < nb) {
      a[tid][j].x *= inv;
      a[tid][j].y *= inv;
      col[tid] = a[tid][j];
    }
    __syncthreads();
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      const int i = e / NB, k = e % NB;
      if (i > j && k > j && k <= i && i < nb) a[i][k] = zfmac(a[i][k], make_double2(-col[i].x, -col[i].y), col[k]);
    }
    __syncthreads();
  }
  // L_pp back to A
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, k = e % nb;
    if (k <= i) A[(long long)(p0 + i) * n + p0 + k] = a[i][k];
  }
  __syncthreads();
  // in-place inverse, columns from the right
  for (int j = nb - 1; j >= 0; --j) {
    if (tid == 0) rcp = 1.0 / a[j][j].x;
    if (tid > j && tid < nb) col[tid] = a[tid][j];
    __syncthreads();
    const double xjj = rcp;
    if (tid > j && tid < nb) {
      double2 s = make_double2(0.0, 0.0);
      for (int k = j + 1; k <= tid; ++k) s = zfma(s, a[tid][k], col[k]);
      a[tid][j] = make_double2(-xjj * s.x, -xjj * s.y);
    }
    if (tid == 0) a[j][j] = make_double2(xjj, 0.0);
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, k = e % nb;
    X[(long long)(p0 + i) * n + p0 + k] = (k <= i) ? a[i][k] : make_double2(0.0, 0.0);
  }
}

// L_ip = A_ip D_p^* for rows i in [r0, n): one CTA per TT rows, all nb columns.
__global__ void __launch_bounds__(256)
panel_kernel(double2* __restrict__ A, const double2* __restrict__ X, int n, int p0, int nb, int r0,
             const int* status) {
  __shared__ double2 rows[TT][NB + 1];
  __shared__ double2 d[NB][NB + 1];
  if (status[0] != 0) return;
  const int tid = threadIdx.x;
  const int i0 = r0 + blockIdx.x * TT;
  for (int e = tid; e < TT * NB; e += blockDim.x) {
    const int i = e / NB, k = e % NB;
    rows[i][k] = (i0 + i < n && k < nb) ? A[(long long)(i0 + i) * n + p0 + k] : make_double2(0.0, 0.0);
  }
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int i = e / NB, k = e % NB;
    d[i][k] = (i < nb && k < nb) ? X[(long long)(p0 + i) * n + p0 + k] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int e = tid; e < TT * NB; e += blockDim.x) {
    const int i = e / NB, c = e % NB;
    if (i0 + i >= n || c >= nb) continue;
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < nb; ++k) s = zfmac(s, rows[i][k], d[c][k]);   // sum_k A_ik conj(D_ck)
    A[(long long)(i0 + i) * n + p0 + c] = s;
  }
}

// A_ik -= sum_{l in panel} L_il conj(L_kl), trailing lower triangle i >= k >= r0.
// Grid: one CTA per lower 16 x 16 tile (bi >= bk) of the trailing block.
__global__ void __launch_bounds__(256)
update_kernel(double2* __restrict__ A, int n, int p0, int nb, int r0, const int* status) {
  __shared__ double2 li[TT][NB + 1];
  __shared__ double2 lk[TT][NB + 1];
  if (status[0] != 0) return;
  int t = blockIdx.x, bi = 0;
  while (t > bi) { t -= bi + 1; ++bi; }
  const int bk = t;
  const int i0 = r0 + bi * TT, k0 = r0 + bk * TT;
  const int tid = threadIdx.x;
  for (int e = tid; e < TT * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    const bool okc = c < nb;
    li[r][c] = (okc && i0 + r < n) ? A[(long long)(i0 + r) * n + p0 + c] : make_double2(0.0, 0.0);
    lk[r][c] = (okc && k0 + r < n) ? A[(long long)(k0 + r) * n + p0 + c] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int r = tid / TT, c = tid % TT;
  const int i = i0 + r, k = k0 + c;
  if (i >= n || k >= n || k > i) return;
  double2 s = make_double2(0.0, 0.0);
  for (int l = 0; l < nb; ++l) s = zfmac(s, li[r][l], lk[c][l]);
  double2& out = A[(long long)i * n + k];
  out = make_double2(out.x - s.x, out.y - s.y);
}

// T(r, j) = sum_{k = j}^{q0 - 1} L(q0 + r, k) X(k, j), r < nb, j < q0 (X lower triangular).
__global__ void __launch_bounds__(256)
inv_row_kernel(const double2* __restrict__ A, const double2* __restrict__ X, double2* __restrict__ T,
               int n, int q0, int nb, const int* status) {
  if (status[0] != 0) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nb * q0) return;
  const int r = idx / q0, j = idx % q0;
  double2 s = make_double2(0.0, 0.0);
  for (int k = j; k < q0; ++k) s = zfma(s, A[(long long)(q0 + r) * n + k], X[(long long)k * n + j]);
  T[(long long)r * q0 + j] = s;
}

// X(q0 + r, j) = -sum_c D_q(r, c) T(c, j), r < nb, j < q0.
__global__ void __launch_bounds__(256)
inv_apply_kernel(const double2* __restrict__ T, double2* __restrict__ X, int n, int q0, int nb,
                 const int* status) {
  if (status[0] != 0) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nb * q0) return;
  const int r = idx / q0, j = idx % q0;
  double2 s = make_double2(0.0, 0.0);
  for (int c = 0; c <= r; ++c) s = zfma(s, X[(long long)(q0 + r) * n + q0 + c], T[(long long)c * q0 + j]);
  X[(long long)(q0 + r) * n + j] = make_double2(-s.x, -s.y);
}

__global__ void linvh_kernel(const double2* __restrict__ X, int n, double* __restrict__ LinvH,
                             const int* status) {
  if (status[0] != 0) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int c = (int)(e / n), i = (int)(e % n);
  double2 v = make_double2(0.0, 0.0);
  if (i >= c) v = X[(long long)i * n + c];
  LinvH[2 * e] = v.x;
  LinvH[2 * e + 1] = -v.y;
}

}  // namespace

void prepare_cholesky(int) {}

size_t cholesky_work_doubles(int n) { return 2 * ((size_t)2 * n * n + (size_t)NB * n); }

int launch_cholesky_inv(const double* M, int n, double* work, double* LinvH, int* status, cudaStream_t st) {
  double2* A = reinterpret_cast<double2*>(work);
  double2* X = A + (size_t)n * n;
  double2* T = X + (size_t)n * n;
  int launches = 0;
  const long long nn = (long long)n * n;
  neg_copy_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(reinterpret_cast<const double2*>(M), nn, A);
  ++launches;
  for (int p0 = 0; p0 < n; p0 += NB) {
    const int nb = (p0 + NB <= n) ? NB : n - p0;
    diag_kernel<<<1, 1024, 0, st>>>(A, X, n, p0, nb, status);
    ++launches;
    const int r0 = p0 + nb;
    if (r0 >= n) break;
    const int rows = n - r0;
    panel_kernel<<<(rows + TT - 1) / TT, 256, 0, st>>>(A, X, n, p0, nb, r0, status);
    const int bt = (rows + TT - 1) / TT;
    update_kernel<<<bt * (bt + 1) / 2, 256, 0, st>>>(A, n, p0, nb, r0, status);
    launches += 2;
  }
  for (int q0 = NB; q0 < n; q0 += NB) {
    const int nb = (q0 + NB <= n) ? NB : n - q0;
    const int cnt = nb * q0;
    inv_row_kernel<<<(cnt + 255) / 256, 256, 0, st>>>(A, X, T, n, q0, nb, status);
    inv_apply_kernel<<<(cnt + 255) / 256, 256, 0, st>>>(T, X, n, q0, nb, status);
    launches += 2;
  }
  linvh_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(X, n, LinvH, status);
  return launches + 1;
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

}  // namespace ace
