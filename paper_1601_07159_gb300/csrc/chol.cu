// FP64 Cholesky factorisation of -M and the inverse of its factor (Sec. 3:
// -M = L L^*, then Xi = W L^{-*} of Eq. Wtilde), blocked so that the FP64 work
// spreads over many SMs (FP64 throughput per SM is low on this part).
//
// Blocks of NB = 16 columns (the diagonal blocks run on one SM each, so they
// are kept small; 32 measured slightly slower). For panel p (rows/cols
// [p0, p0 + nb)):
//   diag    one CTA: A_pp -> L_pp (right-looking Cholesky in shared memory,
//           status word on a non-finite or non-positive pivot), D_p = L_pp^{-1}
//           (recursive-doubling inverse of a triangular matrix); L_pp is
//           stored in A, D_p in the diagonal block of X.
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

constexpr int NB = 16;   // panel width
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

// Factor and invert the diagonal block of panel p (nb <= NB); NB * NB threads.
// The block is padded to NB with the identity, so every loop runs NB uniform
// steps.
// Cholesky on unscaled columns: step j subtracts a_ij conj(a_kj) / d_j from
// the trailing lower triangle (d_j = a_jj at step j). The trailing triangle's
// elements are packed densely onto threads (a table ordered by decreasing
// column, so the elements of step j are the first (NB-1-j)(NB-j)/2), which
// keeps warps full: FP64 issue is the scarce resource on this part. The thread
// that updates a_{j+1,j+1} in step j also checks that pivot and forms its
// reciprocal, so a step needs one barrier and one FP64 reciprocal. The
// reciprocal is the FP32 one refined by two Newton-Raphson steps in FP64
// (r <- r + r (1 - d r); each step squares the relative error: 1e-7 -> 1e-14
// -> rounding). Afterwards L_jj = sqrt(d_j) and L_ij = a_ij / sqrt(d_j) in one
// parallel pass.
// Inverse by recursive doubling: for a lower-triangular [[A, 0], [B, C]],
// the inverse is [[A^-1, 0], [-C^-1 (B A^-1), C^-1]]; log2 NB levels (block
// edge 2, 4, ..., NB) of small products replace NB dependent column steps. The
// intermediate B A^-1 is kept, transposed, in the unused upper triangle of X.
__device__ __forceinline__ double recip_nr(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / d;   // outside FP32's comfortable range
  double r = (double)(1.0f / (float)d);
  r = fma(r, fma(-d, r, 1.0), r);
  r = fma(r, fma(-d, r, 1.0), r);
  return r;
}

constexpr int kTri = NB * (NB - 1) / 2;   // trailing-triangle elements (i >= k >= 1)

__global__ void __launch_bounds__(NB * NB)
diag_kernel(double2* __restrict__ A, double2* __restrict__ X, int n, int p0, int nb, int* status) {
  __shared__ double2 a[NB][NB + 1];
  __shared__ double2 x[NB][NB + 1];
  __shared__ double dl[NB], dil[NB], rj[NB];
  __shared__ unsigned char ti[kTri], tk[kTri];
  __shared__ int s_fail, s_piv;
  const int tid = threadIdx.x;
  const int ei = tid / NB, ek = tid % NB;
  if (status[0] != 0) return;
  {
    double2 v = make_double2(ei == ek ? 1.0 : 0.0, 0.0);
    if (ei < nb && ek <= ei) v = A[(long long)(p0 + ei) * n + p0 + ek];
    a[ei][ek] = v;
    x[ei][ek] = make_double2(0.0, 0.0);
  }
  // packed trailing-triangle table: entries (i, k), k = NB-1 down to 1, i = k .. NB-1
  if (tid < kTri) {
    int k = NB - 1, o = 0;
    while (tid >= o + (NB - k)) {
      o += NB - k;
      --k;
    }
    ti[tid] = (unsigned char)(k + (tid - o));
    tk[tid] = (unsigned char)k;
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  auto pivot = [&](int j) {     // one thread: check d_j, store its reciprocal
    const double d = a[j][j].x;
    if (!isfinite(d) || !(d > 0.0)) {
      s_fail = isfinite(d) ? -2 : -3;
      s_piv = j;
      rj[j] = 0.0;
    } else {
      rj[j] = recip_nr(d);
    }
  };
  if (tid == 0) pivot(0);
  __syncthreads();
  for (int j = 0; j < NB; ++j) {
    if (s_fail) {               // uniform: read after a barrier
      if (tid == 0) {
        status[0] = s_fail;
        status[1] = p0 + s_piv + 1;
      }
      return;
    }
    const int cnt = (NB - 1 - j) * (NB - j) / 2;
    if (tid < cnt) {
      const int i = ti[tid], k = tk[tid];
      const double r = rj[j];
      const double2 u = a[i][j];
      const double2 w = a[k][j];
      a[i][k] = zfmac(a[i][k], make_double2(-u.x * r, -u.y * r), w);
      if (i == j + 1 && k == j + 1) pivot(j + 1);
    }
    __syncthreads();
  }
  if (tid < NB) {
    const double l = sqrt(a[tid][tid].x);
    dl[tid] = l;
    dil[tid] = 1.0 / l;
  }
  __syncthreads();
  if (ek < ei) {
    a[ei][ek].x *= dil[ek];
    a[ei][ek].y *= dil[ek];
  } else if (ek == ei) {
    a[ei][ei] = make_double2(dl[ei], 0.0);
    x[ei][ei] = make_double2(dil[ei], 0.0);
  }
  __syncthreads();
  if (ei < nb && ek <= ei) A[(long long)(p0 + ei) * n + p0 + ek] = a[ei][ek];
  for (int h = 1; h < NB; h *= 2) {     // blocks of edge 2h at rows/cols b .. b + 2h
    const int cnt = (NB / (2 * h)) * h * h;
    // T = B A^{-1}: T_rc = sum_{m >= c} a[b+h+r][b+m] x[b+m][b+c], stored at x[b+c][b+h+r]
    for (int e = tid; e < cnt; e += blockDim.x) {
      const int blk = e / (h * h), r = (e / h) % h, c = e % h, b = blk * 2 * h;
      double2 t = make_double2(0.0, 0.0);
      for (int m = c; m < h; ++m) t = zfma(t, a[b + h + r][b + m], x[b + m][b + c]);
      x[b + c][b + h + r] = t;
    }
    __syncthreads();
    // X_B = -C^{-1} T: X[b+h+r][b+c] = -sum_{m <= r} x[b+h+r][b+h+m] T_mc
    for (int e = tid; e < cnt; e += blockDim.x) {
      const int blk = e / (h * h), r = (e / h) % h, c = e % h, b = blk * 2 * h;
      double2 t = make_double2(0.0, 0.0);
      for (int m = 0; m <= r; ++m) t = zfma(t, x[b + h + r][b + h + m], x[b + c][b + h + m]);
      x[b + h + r][b + c] = make_double2(-t.x, -t.y);
    }
    __syncthreads();
  }
  if (ei < nb && ek < nb) X[(long long)(p0 + ei) * n + p0 + ek] = ek <= ei ? x[ei][ek] : make_double2(0.0, 0.0);
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
// Block (32, KS): x indexes j, y strides over k; the KS partial sums are added
// in a fixed order, so the result does not depend on timing.
constexpr int KS = 8;
__global__ void __launch_bounds__(256)
inv_row_kernel(const double2* __restrict__ A, const double2* __restrict__ X, double2* __restrict__ T,
               int n, int q0, int nb, const int* status) {
  __shared__ double2 red[KS][32];
  if (status[0] != 0) return;
  const int r = blockIdx.y, j = blockIdx.x * 32 + threadIdx.x, ty = threadIdx.y;
  double2 s = make_double2(0.0, 0.0);
  if (j < q0)
    for (int k = j + ty; k < q0; k += KS) s = zfma(s, A[(long long)(q0 + r) * n + k], X[(long long)k * n + j]);
  red[ty][threadIdx.x] = s;
  __syncthreads();
  if (ty == 0 && j < q0) {
    for (int y = 1; y < KS; ++y) s = make_double2(s.x + red[y][threadIdx.x].x, s.y + red[y][threadIdx.x].y);
    T[(long long)r * q0 + j] = s;
  }
}

// X(q0 + r, j) = -sum_c D_q(r, c) T(c, j), r < nb, j < q0 (same block shape, y strides over c).
__global__ void __launch_bounds__(256)
inv_apply_kernel(const double2* __restrict__ T, double2* __restrict__ X, int n, int q0, int nb,
                 const int* status) {
  __shared__ double2 red[KS][32];
  if (status[0] != 0) return;
  const int r = blockIdx.y, j = blockIdx.x * 32 + threadIdx.x, ty = threadIdx.y;
  double2 s = make_double2(0.0, 0.0);
  if (j < q0)
    for (int c = ty; c <= r; c += KS) s = zfma(s, X[(long long)(q0 + r) * n + q0 + c], T[(long long)c * q0 + j]);
  red[ty][threadIdx.x] = s;
  __syncthreads();
  if (ty == 0 && j < q0) {
    for (int y = 1; y < KS; ++y) s = make_double2(s.x + red[y][threadIdx.x].x, s.y + red[y][threadIdx.x].y);
    X[(long long)(q0 + r) * n + j] = make_double2(-s.x, -s.y);
  }
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
    diag_kernel<<<1, NB * NB, 0, st>>>(A, X, n, p0, nb, status);
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
    const dim3 grid((q0 + 31) / 32, nb), block(32, KS);
    inv_row_kernel<<<grid, block, 0, st>>>(A, X, T, n, q0, nb, status);
    inv_apply_kernel<<<grid, block, 0, st>>>(T, X, n, q0, nb, status);
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

// X *= s over the first ng elements of each of `count` vectors of stride ld
// (real and imaginary parts alike): one packed run when ld == ng.
void launch_scale(bool f64, bool real, void* X, long long count, long long ng, long long ld, double s,
                  cudaStream_t st) {
  const long long per = real ? 1 : 2;   // reals per element
  const long long runs = ld == ng ? 1 : count, run = (ld == ng ? count * ng : ng) * per;
  const unsigned grid = (unsigned)((run + 255) / 256 < 152 * 16 ? (run + 255) / 256 : 152 * 16);
  for (long long v = 0; v < runs; ++v) {
    if (f64) scale_kernel_d<<<grid, 256, 0, st>>>(static_cast<double*>(X) + v * ld * per, run, s);
    else scale_kernel_f<<<grid, 256, 0, st>>>(static_cast<float*>(X) + v * ld * per, run, (float)s);
  }
}

}  // namespace ace
