// Register-resident mixed-radix DFTs (radices 2, 3, 4, 5) for one thread.
//
// A thread holds a whole line of N complex values in registers and transforms
// it with a fully unrolled decimation-in-time recursion: N = R * M, R sub-DFTs
// of length M over the decimated inputs a[r + R m], twiddles w_N^{r k}, then a
// radix-R butterfly across r. All indices are compile-time constants after
// unrolling, so the values stay in registers and the twiddles come from the
// kernel's constant parameter bank (a table of w_NTOP^k = exp(-2 pi i k/NTOP)
// for k < NTOP, computed on the host in FP64 from sin/cos). Exact quarter
// turns (w = 1, -i, -1, i) are applied as swaps, not multiplications.
//
// This is the Poisson solver's transform (Sec. 2: each solve is
// O(N_g log N_g) with FFTs); the 3-D transform is built from these line
// transforms in pair_kernels.cu.
//
// Radix order, fixed per translation unit by ACE_RADIX_ORDER: 0 (default)
// takes a radix 4 first, then 2, 3, 5; 1 takes the odd radix (3, then 5)
// first when the length has one, so 48 = 3 x 16 instead of 4 x 12 (other
// twiddle sets, other instruction schedules). The code of each order sits in
// its own inline namespace, so instances of both orders link into one library.
#pragma once
#include <cuda_runtime.h>

#ifndef ACE_RADIX_ORDER
#define ACE_RADIX_ORDER 0
#endif
#if ACE_RADIX_ORDER == 0
#define ACE_RADIX_NS radix0
#elif ACE_RADIX_ORDER == 1
#define ACE_RADIX_NS radix1
#else
#error "ACE_RADIX_ORDER must be 0 or 1"
#endif

namespace ace {
inline namespace ACE_RADIX_NS {

template <typename R> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename R> using cplx = typename cplx_t<R>::type;

template <typename T> __device__ __forceinline__ T cmk(decltype(T::x) x, decltype(T::x) y) {
  T r; r.x = x; r.y = y; return r;
}
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { return cmk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { return cmk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  return cmk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename T> __device__ __forceinline__ T cmulc(T a, T b) {
  return cmk<T>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename T> __device__ __forceinline__ T cscale(T a, decltype(T::x) s) { return cmk<T>(a.x * s, a.y * s); }
// acc + a b and acc + conj(a) b as four fused multiply-adds (accumulations)
template <typename T> __device__ __forceinline__ T cfma(T acc, T a, T b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
template <typename T> __device__ __forceinline__ T cfmac(T acc, T a, T b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
// multiply by -i (forward) or +i (inverse) -> "rotate by the forward quarter turn"
template <bool INV, typename T> __device__ __forceinline__ T rot_q(T a) {
  return INV ? cmk<T>(-a.y, a.x) : cmk<T>(a.y, -a.x);
}

template <typename R, int NTOP> struct TwTable { cplx<R> w[NTOP]; };

// w_N^e (forward sign), or its conjugate for the inverse transform, applied to x.
template <int N, int NTOP, bool INV, typename R>
__device__ __forceinline__ cplx<R> twiddle(cplx<R> x, int e, const TwTable<R, NTOP>& tw) {
  e %= N;
  if (e == 0) return x;
  if ((4 * e) % N == 0) {
    const int q = (4 * e) / N;             // quarter turns
    if (q == 1) return rot_q<INV>(x);
    if (q == 2) return cmk<cplx<R>>(-x.x, -x.y);
    return rot_q<!INV>(x);
  }
  const cplx<R> w = tw.w[e * (NTOP / N)];
  return INV ? cmk<cplx<R>>(x.x * w.x + x.y * w.y, x.y * w.x - x.x * w.y)   // x * conj(w)
             : cmul(x, w);
}

// The twiddle w_N^e (forward sign) or its conjugate as a value: exact for the
// quarter turns, from the table otherwise. With e a compile-time constant after
// unrolling this is a pair of constants.
template <int N, int NTOP, bool INV, typename R>
__device__ __forceinline__ cplx<R> twiddle_value(int e, const TwTable<R, NTOP>& tw) {
  e %= N;
  if (e == 0) return cmk<cplx<R>>(R(1), R(0));
  if ((4 * e) % N == 0) {
    const int q = (4 * e) / N;   // forward: -i, -1, +i
    if (q == 2) return cmk<cplx<R>>(R(-1), R(0));
    const R s = (q == 1) != INV ? R(-1) : R(1);
    return cmk<cplx<R>>(R(0), s);
  }
  const cplx<R> w = tw.w[e * (NTOP / N)];
  return INV ? cmk<cplx<R>>(w.x, -w.y) : w;
}

template <int N> __host__ __device__ constexpr int first_radix() {
  if constexpr (ACE_RADIX_ORDER == 1 && N % 3 == 0 && N != 3) return 3;
  if constexpr (ACE_RADIX_ORDER == 1 && N % 5 == 0 && N != 5) return 5;
  return (N % 4 == 0 && N != 4) ? 4 : (N % 2 == 0 ? 2 : (N % 3 == 0 ? 3 : (N % 5 == 0 ? 5 : N)));
}

template <int N, int NTOP, bool INV, typename R>
__device__ __forceinline__ void dft(cplx<R> (&a)[N], const TwTable<R, NTOP>& tw);

template <int NTOP, bool INV, typename R>
__device__ __forceinline__ void bfly2(cplx<R> (&a)[2]) {
  const cplx<R> t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}

template <int NTOP, bool INV, typename R>
__device__ __forceinline__ void bfly4(cplx<R> (&a)[4]) {
  const cplx<R> s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
  const cplx<R> s13 = cadd(a[1], a[3]), d13 = rot_q<INV>(csub(a[1], a[3]));
  a[0] = cadd(s02, s13);
  a[2] = csub(s02, s13);
  a[1] = cadd(d02, d13);
  a[3] = csub(d02, d13);
}

// radix 3: X1,2 = a0 + c (a1 + a2) -/+ i s (a1 - a2) with w_3 = c - i s (forward)
template <int NTOP, bool INV, typename R>
__device__ __forceinline__ void bfly3(cplx<R> (&a)[3], const TwTable<R, NTOP>& tw) {
  const cplx<R> w3 = tw.w[NTOP / 3];
  const R c = w3.x, s = -w3.y;
  const cplx<R> t = cadd(a[1], a[2]);
  const cplx<R> d = cscale(csub(a[1], a[2]), s);
  const cplx<R> u = cmk<cplx<R>>(a[0].x + c * t.x, a[0].y + c * t.y);
  a[0] = cadd(a[0], t);
  const cplx<R> rd = rot_q<INV>(d);
  a[1] = cadd(u, rd);
  a[2] = csub(u, rd);
}

// radix 5 with c1 = cos 2pi/5, c2 = cos 4pi/5, s1 = sin 2pi/5, s2 = sin 4pi/5
template <int NTOP, bool INV, typename R>
__device__ __forceinline__ void bfly5(cplx<R> (&a)[5], const TwTable<R, NTOP>& tw) {
  const cplx<R> w1 = tw.w[NTOP / 5], w2 = tw.w[2 * NTOP / 5];
  const R c1 = w1.x, s1 = -w1.y, c2 = w2.x, s2 = -w2.y;
  const cplx<R> t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
  const cplx<R> t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
  const cplx<R> b1 = cmk<cplx<R>>(a[0].x + c1 * t1.x + c2 * t2.x, a[0].y + c1 * t1.y + c2 * t2.y);
  const cplx<R> b2 = cmk<cplx<R>>(a[0].x + c2 * t1.x + c1 * t2.x, a[0].y + c2 * t1.y + c1 * t2.y);
  const cplx<R> e1 = rot_q<INV>(cmk<cplx<R>>(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
  const cplx<R> e2 = rot_q<INV>(cmk<cplx<R>>(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
  a[0] = cadd(a[0], cadd(t1, t2));
  a[1] = cadd(b1, e1);
  a[4] = csub(b1, e1);
  a[2] = cadd(b2, e2);
  a[3] = csub(b2, e2);
}

template <int N, int NTOP, bool INV, typename R>
__device__ __forceinline__ void dft(cplx<R> (&a)[N], const TwTable<R, NTOP>& tw) {
  static_assert(NTOP % N == 0, "sub-length must divide the table length");
  if constexpr (N == 1) {
    return;
  } else if constexpr (N == 2) {
    bfly2<NTOP, INV, R>(a);
  } else if constexpr (N == 3) {
    bfly3<NTOP, INV, R>(a, tw);
  } else if constexpr (N == 4) {
    bfly4<NTOP, INV, R>(a);
  } else if constexpr (N == 5) {
    bfly5<NTOP, INV, R>(a, tw);
  } else {
    constexpr int RX = first_radix<N>();
    static_assert(RX != N, "unsupported prime factor");
    constexpr int M = N / RX;
    cplx<R> sub[RX][M];
#pragma unroll
    for (int r = 0; r < RX; ++r)
#pragma unroll
      for (int m = 0; m < M; ++m) sub[r][m] = a[r + RX * m];
#pragma unroll
    for (int r = 0; r < RX; ++r) dft<M, NTOP, INV, R>(sub[r], tw);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      cplx<R> t[RX];
#pragma unroll
      for (int r = 0; r < RX; ++r) t[r] = twiddle<N, NTOP, INV, R>(sub[r][k], r * k, tw);
      dft<RX, NTOP, INV, R>(t, tw);
#pragma unroll
      for (int q = 0; q < RX; ++q) a[k + M * q] = t[q];
    }
  }
}

}  // namespace ACE_RADIX_NS
}  // namespace ace
