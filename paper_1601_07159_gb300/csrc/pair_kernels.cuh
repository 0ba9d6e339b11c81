// Pair FFT-Poisson solves: the hot loop of Eq. applyVX / Eq. W.
//
// For a batch of pairs (l, r) the 3-D solve v = F^-1[ K F[conj(x_l) y_r] ] is
// split into three passes over the batch's spectrum scratch S, each a set of
// register-resident line FFTs (fft_reg.cuh), plus one accumulate pass:
//
//   pass A  (per z-plane)   rho = conj(x_l) y_r; FFT along y (thread = column x,
//                           coalesced loads), transpose through shared memory,
//                           FFT along x (thread = row ky); store S[z][kx][ky]
//                           (coalesced along ky).
//   pass B  (per pencil)    FFT along z, multiply by K(G)/N_g, inverse FFT along
//                           z, in place (thread = (kx, ky) pencil, coalesced);
//                           optionally the Parseval energy sum K |rho_hat|^2.
//   pass C  (per z-plane)   inverse FFT along x (thread = ky), transpose through
//                           shared memory, inverse FFT along y (thread = x);
//                           store v(z, y, x) in place (coalesced along x).
//   pass D  (per point)     Out_r -= x_l v and, for symmetric tiles,
//                           Out_l -= y_r conj(v); registers hold the tile's
//                           orbitals and accumulators, one read-modify-write of
//                           each output per tile, fixed summation order (full
//                           off-diagonal tiles: two threads per point).
// In FP32 at the larger edges a line is held by two lanes instead of one
// thread (split_line_dft): passes A and C from n = 48, pass B from n = 64.
//
// Two ways to run a schedule of batches:
//  * four kernels per batch (pass_*_kernel), chained with programmatic
//    dependent launch, replayed from a CUDA graph (the default) or launched
//    eagerly (per-pass timing);
//  * one persistent launch (pair_engine_kernel): co-resident blocks take
//    tasks (one pass-A/C block of planes, one pass-B block of pencils, one
//    pass-D block of points) in schedule order from an atomic queue and wait,
//    with a bounded spin, on per-batch completion counters: pass p of batch k
//    needs all of pass p-1 of batch k, pass A of batch k needs the last pass of
//    batch k-1 (the scratch is reused). Tasks are taken in increasing order by
//    resident blocks, so every awaited task is already running: no deadlock.
//
// Tiles within a batch touch disjoint outputs (the schedule guarantees it) and
// batches run in order, so the accumulation needs no atomics and the result is
// bitwise reproducible. The engine sums a full off-diagonal tile's left
// outputs in one thread rather than two, so the two modes agree to rounding.
#pragma once
#include "ace_internal.h"
#include "fft_reg.cuh"

namespace ace {

template <typename R, int N> struct PairParams {
  const void* X;
  const void* Y;
  void* OutX;
  void* OutY;
  cplx<R>* S;
  const R* Kt;
  double* Epart;
  long long ld;
  R scale;
  int npairs;
  const TileDesc* tiles;   // device table of the batch's tiles
  int ntiles;
  TwTable<R, N> tw;
};

// Programmatic dependent launch (four-kernel mode): every pass is launched with
// programmatic stream serialisation, so its blocks can be scheduled while the
// previous pass drains; griddep_wait() blocks until the previous grid has
// completed and its writes are visible. Without the attribute both are no-ops.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename Kern, typename... Args>
inline void launch_pdl(bool pdl, Kern kern, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       const Args&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

// Loads and stores of data that other blocks of the same launch produce or
// consume (the pair scratch and the outputs, in the persistent engine) go
// through L2 (.cg): L1 is not coherent across SMs.
template <bool COH, typename T> __device__ __forceinline__ T ldx(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}
template <bool COH, typename T> __device__ __forceinline__ void stx(T* p, T v) {
  if constexpr (COH) __stcg(p, v);
  else *p = v;
}

// Slot p of the batch -> tile index and (l, r) orbital indices.
__device__ __forceinline__ int decode_pair(const TileDesc* __restrict__ tiles, int ntiles, int p, int& l, int& r) {
  int t = 0;
  while (t + 1 < ntiles && tiles[t + 1].slot0 <= p) ++t;
  const TileDesc d = tiles[t];
  int q = p - d.slot0;
  if (d.kind == 1) {
    int li = 0, len = d.nl;
    while (q >= len) { q -= len; ++li; --len; }
    l = d.l0 + li;
    r = d.r0 + li + q;
  } else {
    l = d.l0 + q / d.nr;
    r = d.r0 + q % d.nr;
  }
  return t;
}

template <typename R, bool REAL>
__device__ __forceinline__ cplx<R> load_vec(const void* base, long long idx) {
  if constexpr (REAL) {
    return cmk<cplx<R>>(static_cast<const R*>(base)[idx], R(0));
  } else {
    return static_cast<const cplx<R>*>(base)[idx];
  }
}

// The kernel table is folded (K depends on |G|^2 only): index k of an axis and
// n - k share an entry. kfold(k) = min(k, N - k); the table is [kz][kx][ky] over
// 0..N/2 each.
template <int N> __host__ __device__ __forceinline__ constexpr int kfold(int k) { return k <= N / 2 ? k : N - k; }
template <int N> constexpr int kKH = N / 2 + 1;
// offset of the (kx, ky) pencil f = kx N + ky in the folded table
template <int N> __device__ __forceinline__ int kt_pencil(int f) {
  const int kx = f / N, ky = f - kx * N;
  return kfold<N>(kx) * kKH<N> + kfold<N>(ky);
}

template <typename R, int N> __host__ __device__ constexpr int plane_items() {
  // items (pair, z-plane) per CTA of the plane kernels: ~256 threads, <= 96 KB
  constexpr int by_threads = (256 / N) > 0 ? (256 / N) : 1;
  constexpr int by_smem = (96 * 1024) / (N * (N + 1) * (int)sizeof(cplx<R>));
  constexpr int v = by_threads < by_smem ? by_threads : by_smem;
  return v > 0 ? v : 1;
}
constexpr int kEngineThreads = 256;
template <typename R, int N> __host__ __device__ constexpr int engine_items() {
  // items per plane task of the engine: all 256 threads, <= 200 KB of planes
  constexpr int by_threads = (kEngineThreads / N) > 0 ? (kEngineThreads / N) : 1;
  constexpr int by_smem = (200 * 1024) / (N * (N + 1) * (int)sizeof(cplx<R>));
  constexpr int v = by_threads < by_smem ? by_threads : by_smem;
  return v > 0 ? v : 1;
}

// ---------------------------------------------------------------- pass bodies
// Pass A on virtual block `vb` (IPB plane items, thread tid = ty * N + tx).
template <typename R, int N, bool REAL, bool COH, int IPB, bool PDL>
__device__ __forceinline__ void body_a(const PairParams<R, N>& P, const TileDesc* tiles, int ntiles, int npairs,
                                       cplx<R>* smem, long long vb, int tid) {
  const int tx = tid % N, ty = tid / N;
  cplx<R>* buf = smem + ty * N * (N + 1);
  const long long item = vb * IPB + ty;
  const bool active = ty < IPB && item < (long long)npairs * N;
  int p = 0, z = 0, l = 0, r = 0;
  if (active) {
    p = (int)(item / N);
    z = (int)(item % N);
    decode_pair(tiles, ntiles, p, l, r);
    cplx<R> a[N];
    const long long xo = (long long)l * P.ld + (long long)z * N * N + tx;
    const long long yo = (long long)r * P.ld + (long long)z * N * N + tx;
#pragma unroll
    for (int y = 0; y < N; ++y) {
      const cplx<R> xv = load_vec<R, REAL>(P.X, xo + y * N);
      const cplx<R> yv = load_vec<R, REAL>(P.Y, yo + y * N);
      a[y] = cmulc(xv, yv);                   // conj(x_l) * y_r
    }
    dft<N, N, false, R>(a, P.tw);             // along y
#pragma unroll
    for (int k = 0; k < N; ++k) buf[k * (N + 1) + tx] = a[k];
  }
  __syncthreads();
  if (active) {
    cplx<R> b[N];
#pragma unroll
    for (int x = 0; x < N; ++x) b[x] = buf[tx * (N + 1) + x];
    dft<N, N, false, R>(b, P.tw);             // along x, row ky = tx
    if constexpr (PDL) griddep_wait();        // the previous batch's pass D still reads S
    cplx<R>* out = P.S + ((long long)p * N + z) * N * N + tx;
#pragma unroll
    for (int kx = 0; kx < N; ++kx) stx<COH>(out + kx * N, b[kx]);
  }
}

// Pass B on virtual block `vb` of `nthr` pencils. mode 0: Poisson (forward z,
// K, inverse z); 1: energy only; 2: both. The energy partial of the block
// (mode != 0) is added to *eslot by thread 0 (one owner per slot).
template <typename R, int N, bool COH>
__device__ __forceinline__ void body_b(const PairParams<R, N>& P, const TileDesc* tiles, int ntiles, int npairs,
                                       int mode, long long vb, int tid, int nthr, double* red, double* eslot) {
  constexpr int N2 = N * N;
  const long long gid = vb * nthr + tid;
  const bool active = gid < (long long)npairs * N2;
  double e = 0.0;
  if (active) {
    const int p = (int)(gid / N2);
    const int f = (int)(gid % N2);
    cplx<R>* s = P.S + (long long)p * N * N2 + f;
    cplx<R> a[N];
#pragma unroll
    for (int zz = 0; zz < N; ++zz) a[zz] = ldx<COH>(s + (long long)zz * N2);
    dft<N, N, false, R>(a, P.tw);
    R acc = R(0);
    const R* kt = P.Kt + kt_pencil<N>(f);
#pragma unroll
    for (int kz = 0; kz < N; ++kz) {
      const R k = kt[kfold<N>(kz) * (kKH<N> * kKH<N>)];
      if (mode != 0) acc += k * (a[kz].x * a[kz].x + a[kz].y * a[kz].y);
      a[kz] = cscale(a[kz], k);
    }
    if (mode != 0) {
      int l, r;
      decode_pair(tiles, ntiles, p, l, r);
      e = (l == r ? 1.0 : 2.0) * (double)acc;
    }
    if (mode != 1) {
      dft<N, N, true, R>(a, P.tw);
#pragma unroll
      for (int zz = 0; zz < N; ++zz) stx<COH>(s + (long long)zz * N2, a[zz]);
    }
  }
  if (mode != 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((tid & 31) == 0) red[tid >> 5] = e;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < nthr / 32; ++w) s += red[w];
      *eslot += s;
    }
  }
}

// Pass C on virtual block `vb` (IPB plane items).
template <typename R, int N, bool COH, int IPB>
__device__ __forceinline__ void body_c(const PairParams<R, N>& P, int npairs, cplx<R>* smem, long long vb, int tid) {
  const int tx = tid % N, ty = tid / N;
  cplx<R>* buf = smem + ty * N * (N + 1);
  const long long item = vb * IPB + ty;
  const bool active = ty < IPB && item < (long long)npairs * N;
  cplx<R>* plane = nullptr;
  if (active) {
    const int p = (int)(item / N);
    const int z = (int)(item % N);
    plane = P.S + ((long long)p * N + z) * N * N;
    cplx<R> b[N];
#pragma unroll
    for (int kx = 0; kx < N; ++kx) b[kx] = ldx<COH>(plane + kx * N + tx);   // row ky = tx
    dft<N, N, true, R>(b, P.tw);                                            // inverse along x
#pragma unroll
    for (int x = 0; x < N; ++x) buf[tx * (N + 1) + x] = b[x];
  }
  __syncthreads();
  if (active) {
    cplx<R> a[N];
#pragma unroll
    for (int ky = 0; ky < N; ++ky) a[ky] = buf[ky * (N + 1) + tx];  // column x = tx
    dft<N, N, true, R>(a, P.tw);                                    // inverse along y
#pragma unroll
    for (int y = 0; y < N; ++y) stx<COH>(plane + y * N + tx, a[y]);
  }
}

template <typename R, bool REAL, bool COH>
__device__ __forceinline__ void rmw_out(void* base, long long idx, cplx<R> acc, R scale) {
  if constexpr (REAL) {
    R* o = static_cast<R*>(base) + idx;
    stx<COH>(o, ldx<COH>(o) - scale * acc.x);
  } else {
    cplx<R>* o = static_cast<cplx<R>*>(base) + idx;
    const cplx<R> c = ldx<COH>(o);
    stx<COH>(o, cmk<cplx<R>>(c.x - scale * acc.x, c.y - scale * acc.y));
  }
}

// Full tiles (kTileMax orbitals per side): no runtime guards, so all loads of
// the tile's pair potentials can be issued back to back. v is read once, so it
// is loaded with the streaming (evict-first) hint.
template <typename R, int N, bool REAL, bool COH>
__device__ __forceinline__ void d_full_diag(const PairParams<R, N>& P, const TileDesc& d,
                                            const cplx<R>* __restrict__ V, long long g) {
  constexpr long long NG = (long long)N * N * N;
  constexpr int B = kTileMax;
  cplx<R> x[B], acc[B];
#pragma unroll
  for (int o = 0; o < B; ++o) {
    acc[o] = cmk<cplx<R>>(R(0), R(0));
    x[o] = load_vec<R, REAL>(P.X, (long long)(d.l0 + o) * P.ld + g);
  }
#pragma unroll
  for (int li = 0; li < B; ++li) {
#pragma unroll
    for (int ri = li; ri < B; ++ri) {
      const int q = li * B - li * (li - 1) / 2 + (ri - li);
      const cplx<R> v = __ldcs(V + (long long)q * NG);
      acc[ri] = cadd(acc[ri], cmul(x[li], v));
      if (ri != li) acc[li] = cadd(acc[li], cmulc(v, x[ri]));
    }
  }
#pragma unroll
  for (int o = 0; o < B; ++o) rmw_out<R, REAL, COH>(P.OutY, (long long)(d.l0 + o) * P.ld + g, acc[o], P.scale);
}

template <typename R, int N, bool REAL, bool COH>
__device__ __forceinline__ void d_full_off(const PairParams<R, N>& P, const TileDesc& d,
                                           const cplx<R>* __restrict__ V, long long g) {
  constexpr long long NG = (long long)N * N * N;
  constexpr int B = kTileMax;
  cplx<R> xl[B], yr[B], al[B], ar[B];
#pragma unroll
  for (int o = 0; o < B; ++o) {
    al[o] = cmk<cplx<R>>(R(0), R(0));
    ar[o] = al[o];
    xl[o] = load_vec<R, REAL>(P.X, (long long)(d.l0 + o) * P.ld + g);
    yr[o] = load_vec<R, REAL>(P.Y, (long long)(d.r0 + o) * P.ld + g);
  }
#pragma unroll
  for (int li = 0; li < B; ++li) {
#pragma unroll
    for (int ri = 0; ri < B; ++ri) {
      const cplx<R> v = __ldcs(V + (long long)(li * B + ri) * NG);
      ar[ri] = cadd(ar[ri], cmul(xl[li], v));
      al[li] = cadd(al[li], cmulc(v, yr[ri]));
    }
  }
#pragma unroll
  for (int o = 0; o < B; ++o) {
    rmw_out<R, REAL, COH>(P.OutY, (long long)(d.r0 + o) * P.ld + g, ar[o], P.scale);
    rmw_out<R, REAL, COH>(P.OutX, (long long)(d.l0 + o) * P.ld + g, al[o], P.scale);
  }
}

// Off-diagonal full tile with two threads per grid point: thread half h takes
// the right orbitals r0 + 4h .. r0 + 4h + 3 (its 32 of the tile's 64 pair
// potentials), so each thread holds half the state of d_full_off and a block
// keeps twice the loads in flight. Each warp covers 32 consecutive points of
// one half (coalesced). The left outputs' two partial sums (over the two
// halves of r) meet through shared memory and are added in a fixed order;
// thread h then updates Out_l for l0 + 4h .. l0 + 4h + 3 and Out_r for its r.
constexpr int kDSplitPts = 128;   // points per 256-thread block
template <typename R, int N, bool REAL>
__device__ __forceinline__ void d_split_off(const PairParams<R, N>& P, const TileDesc& d, long long vbx, int tid,
                                            cplx<R>* xch) {
  constexpr long long NG = (long long)N * N * N;
  constexpr int B = kTileMax, H = kTileMax / 2;
  const int h = (tid >> 5) & 1;
  const int pt = ((tid >> 6) << 5) | (tid & 31);
  const long long g = vbx * kDSplitPts + pt;
  const bool act = g < NG;
  const cplx<R>* V = P.S + (long long)d.slot0 * NG + g;
  cplx<R> xl[B], yr[H], al[B], ar[H];
#pragma unroll
  for (int o = 0; o < B; ++o) {
    al[o] = cmk<cplx<R>>(R(0), R(0));
    xl[o] = act ? load_vec<R, REAL>(P.X, (long long)(d.l0 + o) * P.ld + g) : al[o];
  }
#pragma unroll
  for (int o = 0; o < H; ++o) {
    ar[o] = al[o];
    yr[o] = act ? load_vec<R, REAL>(P.Y, (long long)(d.r0 + h * H + o) * P.ld + g) : al[o];
  }
  if (act) {
#pragma unroll
    for (int li = 0; li < B; ++li) {
#pragma unroll
      for (int ri = 0; ri < H; ++ri) {
        const cplx<R> v = __ldcs(V + (long long)(li * B + h * H + ri) * NG);
        ar[ri] = cadd(ar[ri], cmul(xl[li], v));
        al[li] = cadd(al[li], cmulc(v, yr[ri]));
      }
    }
  }
#pragma unroll
  for (int o = 0; o < H; ++o) xch[o * 256 + tid] = h ? al[o] : al[H + o];   // the partner's half
  __syncthreads();
  if (!act) return;
  const int partner = tid ^ 32;                                           // same point, other half
#pragma unroll
  for (int o = 0; o < H; ++o) {
    const cplx<R> own = h ? al[H + o] : al[o];
    const cplx<R> other = xch[o * 256 + partner];
    const cplx<R> lo = h ? other : own, hi = h ? own : other;              // r-half 0 first, then 1
    rmw_out<R, REAL, false>(P.OutX, (long long)(d.l0 + h * H + o) * P.ld + g, cadd(lo, hi), P.scale);
    rmw_out<R, REAL, false>(P.OutY, (long long)(d.r0 + h * H + o) * P.ld + g, ar[o], P.scale);
  }
}

// Pass D for point block `vbx` (nthr points) of tile `d`.
template <typename R, int N, bool REAL, bool COH, bool FULL_OFF = true>
__device__ __forceinline__ void body_d(const PairParams<R, N>& P, const TileDesc& d, long long vbx, int tid,
                                       int nthr) {
  constexpr long long NG = (long long)N * N * N;
  const long long g = vbx * nthr + tid;
  if (g >= NG) return;
  const cplx<R>* V = P.S + (long long)d.slot0 * NG + g;
  if (d.kind == 1 && d.nl == kTileMax) {
    d_full_diag<R, N, REAL, COH>(P, d, V, g);
  } else if (FULL_OFF && d.kind == 0 && d.nl == kTileMax && d.nr == kTileMax) {
    d_full_off<R, N, REAL, COH>(P, d, V, g);
  } else if (d.kind == 1) {
    cplx<R> x[kTileMax], acc[kTileMax];
#pragma unroll
    for (int o = 0; o < kTileMax; ++o) {
      acc[o] = cmk<cplx<R>>(R(0), R(0));
      x[o] = o < d.nl ? load_vec<R, REAL>(P.X, (long long)(d.l0 + o) * P.ld + g) : acc[o];
    }
    int q = 0;
#pragma unroll
    for (int li = 0; li < kTileMax; ++li) {
#pragma unroll
      for (int ri = li; ri < kTileMax; ++ri) {
        if (li < d.nl && ri < d.nl) {
          const cplx<R> v = ldx<COH>(V + (long long)q * NG);
          ++q;
          acc[ri] = cadd(acc[ri], cmul(x[li], v));
          if (ri != li) acc[li] = cadd(acc[li], cmulc(v, x[ri]));   // x_r conj(v)
        }
      }
    }
#pragma unroll
    for (int o = 0; o < kTileMax; ++o)
      if (o < d.nl) rmw_out<R, REAL, COH>(P.OutY, (long long)(d.l0 + o) * P.ld + g, acc[o], P.scale);
  } else if (d.kind == 0) {
    cplx<R> xl[kTileMax], yr[kTileMax], al[kTileMax], ar[kTileMax];
#pragma unroll
    for (int o = 0; o < kTileMax; ++o) {
      al[o] = cmk<cplx<R>>(R(0), R(0));
      ar[o] = al[o];
      xl[o] = o < d.nl ? load_vec<R, REAL>(P.X, (long long)(d.l0 + o) * P.ld + g) : al[o];
      yr[o] = o < d.nr ? load_vec<R, REAL>(P.Y, (long long)(d.r0 + o) * P.ld + g) : al[o];
    }
#pragma unroll
    for (int li = 0; li < kTileMax; ++li) {
#pragma unroll
      for (int ri = 0; ri < kTileMax; ++ri) {
        if (li < d.nl && ri < d.nr) {
          const cplx<R> v = ldx<COH>(V + (long long)(li * d.nr + ri) * NG);
          ar[ri] = cadd(ar[ri], cmul(xl[li], v));
          al[li] = cadd(al[li], cmulc(v, yr[ri]));
        }
      }
    }
#pragma unroll
    for (int o = 0; o < kTileMax; ++o) {
      if (o < d.nr) rmw_out<R, REAL, COH>(P.OutY, (long long)(d.r0 + o) * P.ld + g, ar[o], P.scale);
      if (o < d.nl) rmw_out<R, REAL, COH>(P.OutX, (long long)(d.l0 + o) * P.ld + g, al[o], P.scale);
    }
  } else {
    cplx<R> ar[kTileMax];
#pragma unroll
    for (int o = 0; o < kTileMax; ++o) ar[o] = cmk<cplx<R>>(R(0), R(0));
    for (int li = 0; li < d.nl; ++li) {
      const cplx<R> xv = load_vec<R, REAL>(P.X, (long long)(d.l0 + li) * P.ld + g);
#pragma unroll
      for (int ri = 0; ri < kTileMax; ++ri) {
        if (ri < d.nr) {
          const cplx<R> v = ldx<COH>(V + (long long)(li * d.nr + ri) * NG);
          ar[ri] = cadd(ar[ri], cmul(xv, v));
        }
      }
    }
#pragma unroll
    for (int o = 0; o < kTileMax; ++o)
      if (o < d.nr) rmw_out<R, REAL, COH>(P.OutY, (long long)(d.r0 + o) * P.ld + g, ar[o], P.scale);
  }
}

// ---------------------------------------------------------------- four-kernel mode
template <typename R, int N, bool REAL>
__global__ void __launch_bounds__(N * plane_items<R, N>(), 2)
pass_a_kernel(const __grid_constant__ PairParams<R, N> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  griddep_launch();
  body_a<R, N, REAL, false, plane_items<R, N>(), true>(P, P.tiles, P.ntiles, P.npairs,
                                                       reinterpret_cast<cplx<R>*>(smem_raw), blockIdx.x, threadIdx.x);
}

// Pass B for the large edges (n >= 64), whose whole pencil per thread spills:
// two lanes per z-pencil (lanes 2q, 2q+1 of a warp; 128 pencils per block).
// Lane h holds the samples z = 2m + h and transforms them with a DFT of N/2:
//   forward  Y[k] = E[k] + w^k O[k], Y[k + N/2] = E[k] - w^k O[k]
//            (E, O the half-length transforms of the even / odd samples,
//            w = exp(-2 pi i / N)); lane h keeps k in [hN/4, (h+1)N/4) and gets
//            the partner's half of E or w^k O by one shuffle per value;
//   inverse  x[2m] = IDFT(Y[k] + Y[k + N/2]), x[2m+1] = IDFT((Y[k] - Y[k + N/2]) w^-k)
//            over k < N/2; each lane forms its quarter of both sequences and
//            swaps the other lane's by shuffle; lane 0 transforms the first,
//            lane 1 the second.
// Lane roles are selected arithmetically (no divergent branches). At n = 48 the
// shuffles cost more than the occupancy gains, so smaller edges keep one
// thread per pencil.
template <typename T> __device__ __forceinline__ T shfl_pair(T v) {
  T r;
  r.x = __shfl_xor_sync(0xffffffffu, v.x, 1);
  r.y = __shfl_xor_sync(0xffffffffu, v.y, 1);
  return r;
}
constexpr int kBSplitPencils = 128;   // pencils per 256-thread block of the split pass B

// FP64 pencils of 64+ points need the whole register file of a thread: one block per SM.
template <typename R, int N> constexpr int kBSplitBlocks = sizeof(R) == 8 ? 1 : 2;

template <typename R, int N>
__global__ void __launch_bounds__(256, kBSplitBlocks<R, N>)
pass_b_split_kernel(const __grid_constant__ PairParams<R, N> P, int mode) {
  using C = cplx<R>;
  constexpr int N2 = N * N, M = N / 2, H = N / 4;
  static_assert(N % 4 == 0, "the split pass B halves a pencil twice");
  __shared__ double red[8];
  griddep_launch();
  griddep_wait();
  const int tid = threadIdx.x, h = tid & 1;
  const long long gid = (long long)blockIdx.x * kBSplitPencils + (tid >> 1);
  const bool active = gid < (long long)P.npairs * N2;     // same for both lanes of a pencil
  const int p = active ? (int)(gid / N2) : 0;
  const int f = active ? (int)(gid % N2) : 0;
  C* s = P.S + (long long)p * N * N2 + f;
  const C zero = cmk<C>(R(0), R(0));
  C a[M];
#pragma unroll
  for (int m = 0; m < M; ++m) a[m] = active ? s[(long long)(2 * m + h) * N2] : zero;
  dft<M, N, false, R>(a, P.tw);                            // E (lane 0) or O (lane 1)
#pragma unroll
  for (int k = 0; k < M; ++k) {                            // lane 1: w^k O[k]
    const C t = twiddle<N, N, false, R>(a[k], k, P.tw);
    a[k] = h ? t : a[k];
  }
  C y[M];                                                  // y[j] = Y[hH + j], y[H + j] = Y[hH + j + M]
#pragma unroll
  for (int j = 0; j < H; ++j) {
    const C recv = shfl_pair(h ? a[j] : a[H + j]);
    const C ev = h ? recv : a[j];
    const C od = h ? a[H + j] : recv;
    y[j] = cadd(ev, od);
    y[H + j] = csub(ev, od);
  }
  R acc = R(0);
  const R* kt = P.Kt + kt_pencil<N>(f);
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const int kz = h * H + (j < H ? j : j - H + M);
    const R k = kt[kfold<N>(kz) * (kKH<N> * kKH<N>)];
    if (mode != 0) acc += k * (y[j].x * y[j].x + y[j].y * y[j].y);
    y[j] = cscale(y[j], k);
  }
  double e = 0.0;
  if (mode != 0 && active) {
    int l, r;
    decode_pair(P.tiles, P.ntiles, p, l, r);
    e = (l == r ? 1.0 : 2.0) * (double)acc;
  }
  if (mode != 1) {
#pragma unroll
    for (int j = 0; j < H; ++j) {                          // k = hH + j
      const C sum = cadd(y[j], y[H + j]);
      const C dif = twiddle<N, N, true, R>(csub(y[j], y[H + j]), h * H + j, P.tw);
      const C recv = shfl_pair(h ? sum : dif);
      a[j] = h ? recv : sum;                               // lane 0: the sums, lane 1: the differences
      a[H + j] = h ? dif : recv;
    }
    dft<M, N, true, R>(a, P.tw);                           // x[2m + h] = a[m]
    if (active) {
#pragma unroll
      for (int m = 0; m < M; ++m) s[(long long)(2 * m + h) * N2] = a[m];
    }
  }
  if (mode != 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((tid & 31) == 0) red[tid >> 5] = e;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int w = 0; w < 8; ++w) sum += red[w];
      P.Epart[blockIdx.x] += sum;                          // one block per slot
    }
  }
}

// A length-N transform of a line held by two lanes (lanes 2q, 2q+1): lane h
// holds the samples 2m + h in a[], and on return holds y[j] = Y[hN/4 + j] and
// y[N/4 + j] = Y[hN/4 + j + N/2] (the forward or inverse DFT, unnormalised):
// a DFT of N/2 per lane, the lane-1 twiddles w^{+-k}, one shuffle per value
// and the radix-2 combine (decimation in time).
template <int N, bool INV, typename R>
__device__ __forceinline__ void split_line_dft(cplx<R> (&a)[N / 2], cplx<R> (&y)[N / 2], int h,
                                               const TwTable<R, N>& tw) {
  using C = cplx<R>;
  constexpr int M = N / 2, H = N / 4;
  dft<M, N, INV, R>(a, tw);
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const C t = twiddle<N, N, INV, R>(a[k], k, tw);
    a[k] = h ? t : a[k];
  }
#pragma unroll
  for (int j = 0; j < H; ++j) {
    const C recv = shfl_pair(h ? a[j] : a[H + j]);
    const C ev = h ? recv : a[j];
    const C od = h ? a[H + j] : recv;
    y[j] = cadd(ev, od);
    y[H + j] = csub(ev, od);
  }
}
// FP32 edges whose plane passes use the two-lane line transforms (one plane
// per block), and the blocks per SM their launch bounds ask for: at 48^3 the
// half-length lines need 72-95 registers, so six 96-thread blocks (18-27 warps)
// fit an SM where the one-thread-per-line form runs 15 warps at 117-128.
// Below 48 the whole-line form is as fast (several planes per block). Pass A
// at 48^3 is held to 80 registers (eight blocks, 24 warps): 1.3 % faster steps.
// FP64 lines take the two-lane form from n = 64 (a whole FP64 line of 64 would
// not fit a thread's registers), with one or two blocks per SM.
constexpr int kSplitMinEdge = 48;
constexpr int kSplitMinEdgeF64 = 64;
template <typename R, int N> constexpr bool kSplitPlanes =
    N % 4 == 0 && (sizeof(R) == 4 ? N >= kSplitMinEdge : N >= kSplitMinEdgeF64);
template <typename R, int N> constexpr int kSplitBlocks = sizeof(R) == 8 ? (N >= 96 ? 1 : 2) : (N >= 96 ? 2 : 6);
template <typename R, int N> constexpr int kSplitBlocksA = sizeof(R) == 4 && N == 48 ? 8 : kSplitBlocks<R, N>;
template <typename R, int N> constexpr size_t kSplitSmem = (size_t)N * (N + 1) * sizeof(cplx<R>);

// frequency index held in y[j] by lane h
template <int N> __device__ __forceinline__ int split_index(int j, int h) {
  return h * (N / 4) + (j < N / 4 ? j : j - N / 4 + N / 2);
}

// Passes A and C with two lanes per line (FP32, n >= 48): one plane per block
// (2n threads), each pass's two line transforms by split_line_dft, the
// transpose through shared memory as in the one-thread-per-line form. Half the
// registers of a whole line per thread (which at 96^3 would need over 200), so
// more warps per SM hide the latency of the plane loads and stores.
template <typename R, int N, bool REAL>
__global__ void __launch_bounds__(2 * N, kSplitBlocksA<R, N>)
pass_a_split_kernel(const __grid_constant__ PairParams<R, N> P) {
  using C = cplx<R>;
  constexpr int M = N / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  griddep_launch();
  const int tid = threadIdx.x, q = tid >> 1, h = tid & 1;
  const long long item = blockIdx.x;                      // one (pair, z) plane per block
  const int p = (int)(item / N), z = (int)(item % N);
  int l, r;
  decode_pair(P.tiles, P.ntiles, p, l, r);
  C a[M], y[M];
  {   // column x = q: samples y = 2m + h
    const long long xo = (long long)l * P.ld + (long long)z * N * N + q;
    const long long yo = (long long)r * P.ld + (long long)z * N * N + q;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int yy = 2 * m + h;
      a[m] = cmulc(load_vec<R, REAL>(P.X, xo + yy * N), load_vec<R, REAL>(P.Y, yo + yy * N));
    }
    split_line_dft<N, false, R>(a, y, h, P.tw);          // along y
#pragma unroll
    for (int j = 0; j < M; ++j) buf[split_index<N>(j, h) * (N + 1) + q] = y[j];
  }
  __syncthreads();
  {   // row ky = q: samples x = 2m + h
#pragma unroll
    for (int m = 0; m < M; ++m) a[m] = buf[q * (N + 1) + 2 * m + h];
    split_line_dft<N, false, R>(a, y, h, P.tw);          // along x
    griddep_wait();                                        // the previous batch's pass D still reads S
    C* out = P.S + ((long long)p * N + z) * N * N + q;
#pragma unroll
    for (int j = 0; j < M; ++j) out[(long long)split_index<N>(j, h) * N] = y[j];
  }
}

template <typename R, int N>
__global__ void __launch_bounds__(2 * N, kSplitBlocks<R, N>)
pass_c_split_kernel(const __grid_constant__ PairParams<R, N> P) {
  using C = cplx<R>;
  constexpr int M = N / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  griddep_launch();
  griddep_wait();
  const int tid = threadIdx.x, q = tid >> 1, h = tid & 1;
  const long long item = blockIdx.x;
  const int p = (int)(item / N), z = (int)(item % N);
  C* plane = P.S + ((long long)p * N + z) * N * N;
  C a[M], y[M];
  {   // row ky = q of the spectrum: samples kx = 2m + h, inverse along x
#pragma unroll
    for (int m = 0; m < M; ++m) a[m] = plane[(long long)(2 * m + h) * N + q];
    split_line_dft<N, true, R>(a, y, h, P.tw);
#pragma unroll
    for (int j = 0; j < M; ++j) buf[q * (N + 1) + split_index<N>(j, h)] = y[j];   // row ky, column x
  }
  __syncthreads();
  {   // column x = q: samples ky = 2m + h, inverse along y
#pragma unroll
    for (int m = 0; m < M; ++m) a[m] = buf[(2 * m + h) * (N + 1) + q];
    split_line_dft<N, true, R>(a, y, h, P.tw);
#pragma unroll
    for (int j = 0; j < M; ++j) plane[(long long)split_index<N>(j, h) * N + q] = y[j];
  }
}

template <typename R, int N>
__global__ void __launch_bounds__(256, 2)
pass_b_kernel(const __grid_constant__ PairParams<R, N> P, int mode) {
  __shared__ double red[32];
  griddep_launch();
  griddep_wait();
  body_b<R, N, false>(P, P.tiles, P.ntiles, P.npairs, mode, blockIdx.x, threadIdx.x, blockDim.x, red,
                      mode != 0 ? P.Epart + blockIdx.x : nullptr);
}

template <typename R, int N>
__global__ void __launch_bounds__(N * plane_items<R, N>(), 2)
pass_c_kernel(const __grid_constant__ PairParams<R, N> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  griddep_launch();
  griddep_wait();
  body_c<R, N, false, plane_items<R, N>()>(P, P.npairs, reinterpret_cast<cplx<R>*>(smem_raw), blockIdx.x, threadIdx.x);
}

// Full off-diagonal tiles take two threads per grid point (d_split_off) at
// four blocks per SM (64 registers): more warps and loads in flight per SM,
// which measured faster than one thread per point at 2 or 3 blocks per SM
// (and than streaming the potentials through shared memory with bulk copies).
template <typename R, int N, bool REAL>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2)
pass_d_kernel(const __grid_constant__ PairParams<R, N> P) {
  __shared__ cplx<R> xch[(kTileMax / 2) * 256];
  griddep_launch();
  griddep_wait();
  const TileDesc d = P.tiles[blockIdx.y];
  if (d.kind == 0 && d.nl == kTileMax && d.nr == kTileMax) {
    d_split_off<R, N, REAL>(P, d, blockIdx.x, threadIdx.x, xch);
    return;
  }
  // other tiles: one thread per point, 256 points per block (the grid is
  // sized for 128-point blocks, so the upper half of the blocks has no work)
  if ((long long)blockIdx.x * 256 >= (long long)N * N * N) return;
  body_d<R, N, REAL, false, false>(P, d, blockIdx.x, threadIdx.x, blockDim.x);
}

// ---------------------------------------------------------------- persistent engine
template <typename R, int N> struct EngineParams {
  PairParams<R, N> P;           // npairs / ntiles unused: per batch from the table
  const EngineBatch* batches;   // per batch: tiles, pairs, first task, tasks per pass
  int nbatches;
  int npasses;                  // 4 (Poisson) or 2 (energy only: A, B)
  long long ntasks;
  unsigned long long* head;     // task queue head
  unsigned* done;               // done[4 k + p]: finished tasks of pass p of batch k
  int* status;                  // plan status word: timeout -> ACE_ERR_TIMEOUT
  int mode;                     // 0: Poisson + accumulate; 1: energy only; 2: both
  unsigned spin_limit;          // polls before a dependent wait gives up
  unsigned wait_bias;           // added to every awaited count (0; a test hook)
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// A wait gives up after E.spin_limit polls (by default 2^22 sleeps of >= 256
// ns, about a second or more); the block then records ACE_ERR_TIMEOUT and
// leaves, and so do the blocks that wait on it, so the launch always ends. A
// block only ever waits before it starts a task, with nothing of its own in
// flight, so leaving is always safe. E.wait_bias > 0 (a test hook) asks for
// more finished tasks than a pass has, so that every dependent wait runs out.

template <typename R, int N, bool REAL>
__global__ void __launch_bounds__(kEngineThreads, 2)
pair_engine_kernel(const __grid_constant__ EngineParams<R, N> E) {
  constexpr int IPB = engine_items<R, N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ long long s_loc;
  __shared__ int s_batch, s_pass, s_stop;
  const int tid = threadIdx.x;
  cplx<R>* smem = reinterpret_cast<cplx<R>*>(smem_raw);
  for (;;) {
    if (tid == 0) {
      const long long t = (long long)atomicAdd(E.head, 1ull);
      int stop = 0, k = 0, pass = 0;
      long long loc = 0;
      if (t >= E.ntasks) {
        stop = 1;
      } else {
        int lo = 0, hi = E.nbatches - 1;   // last batch whose first task <= t
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (E.batches[mid].task0 <= t) lo = mid;
          else hi = mid - 1;
        }
        k = lo;
        const EngineBatch b = E.batches[k];
        loc = t - b.task0;
        while (loc >= b.n[pass]) { loc -= b.n[pass]; ++pass; }
        const unsigned* want = nullptr;
        unsigned target = 0;
        if (pass > 0) {
          want = E.done + kCtrStride * (4 * k + pass - 1);
          target = (unsigned)b.n[pass - 1] + E.wait_bias;
        } else if (k > 0) {
          want = E.done + kCtrStride * (4 * (k - 1) + E.npasses - 1);
          target = (unsigned)E.batches[k - 1].n[E.npasses - 1] + E.wait_bias;
        }
        if (want) {
          unsigned it = 0;
          while (ld_acquire(want) < target) {
            __nanosleep(it < 64 ? 32 : 256);
            if (++it > E.spin_limit) {
              E.status[0] = -6;   // ACE_ERR_TIMEOUT
              E.status[1] = (int)(t & 0x7fffffff);
              stop = 1;
              break;
            }
          }
        }
      }
      s_stop = stop;
      s_batch = k;
      s_pass = pass;
      s_loc = loc;
    }
    __syncthreads();
    if (s_stop) return;
    const int k = s_batch, pass = s_pass;
    const long long loc = s_loc;
    const EngineBatch& b = E.batches[k];
    const TileDesc* tiles = E.P.tiles + b.toff;
    if (pass == 0) {
      body_a<R, N, REAL, true, IPB, false>(E.P, tiles, b.ntiles, b.npairs, smem, loc, tid);
    } else if (pass == 1) {
      body_b<R, N, true>(E.P, tiles, b.ntiles, b.npairs, E.mode, loc, tid, kEngineThreads, red,
                         E.mode != 0 ? E.P.Epart + loc : nullptr);
    } else if (pass == 2) {
      body_c<R, N, true, IPB>(E.P, b.npairs, smem, loc, tid);
    } else {
      const long long nvb = ((long long)N * N * N + kEngineThreads - 1) / kEngineThreads;
      const TileDesc d = tiles[loc / nvb];
      body_d<R, N, REAL, true>(E.P, d, loc % nvb, tid, kEngineThreads);
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(E.done + kCtrStride * (4 * k + pass), 1u);
    }
  }
}

// ---------------------------------------------------------------- host side
template <typename R, int N>
void fill_params(PairParams<R, N>& P, const PairLaunch& L, const Batch& b) {
  P.X = L.X;
  P.Y = L.Y;
  P.OutX = L.OutX;
  P.OutY = L.OutY;
  P.S = static_cast<cplx<R>*>(L.S);
  P.Kt = static_cast<const R*>(L.Kt);
  P.Epart = L.Epart;
  P.ld = L.ld;
  P.scale = (R)L.scale;
  P.npairs = b.npairs;
  P.tiles = L.dtiles;
  P.ntiles = b.ntiles;
  for (int k = 0; k < N; ++k) {
    P.tw.w[k].x = (R)L.tw[2 * k];
    P.tw.w[k].y = (R)L.tw[2 * k + 1];
  }
}

// Tasks per pass of a batch in the engine (A, B, C, D).
template <typename R, int N>
void engine_tasks(const Batch& b, int n[4]) {
  constexpr int IPB = engine_items<R, N>();
  n[0] = (int)(((long long)b.npairs * N + IPB - 1) / IPB);
  n[1] = (int)(((long long)b.npairs * N * N + kEngineThreads - 1) / kEngineThreads);
  n[2] = n[0];
  n[3] = (int)((((long long)N * N * N + kEngineThreads - 1) / kEngineThreads) * b.ntiles);
}

// The persistent engine holds whole lines per thread; FP64 lines of 64 or more
// points do not fit, so those edges have no engine (plans fall back to the four
// kernels per batch).
template <typename R, int N> constexpr bool kEngineBuilt = !(sizeof(R) == 8 && N >= kSplitMinEdgeF64);

template <typename R, int N>
void engine_prepare(EngineInfo& info) {
  if constexpr (!kEngineBuilt<R, N>) {
    info = EngineInfo{};
    return;
  } else {
  constexpr int IPB = engine_items<R, N>();
  constexpr size_t smem = (size_t)IPB * N * (N + 1) * sizeof(cplx<R>);
  info.smem = smem;
  info.threads = kEngineThreads;
  int dev = 0, sms = 0, per = 0, occ = 1 << 30;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto one = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kEngineThreads, smem);
    if (per < occ) occ = per;
  };
  one(pair_engine_kernel<R, N, false>);
  if constexpr (sizeof(R) == 8) one(pair_engine_kernel<R, N, true>);
  info.blocks = occ > 0 ? occ * sms : 0;
  }
}

template <typename R, int N>
bool launch_engine(const PairLaunch& L, const EngineLaunch& EL, cudaStream_t st) {
  if constexpr (!kEngineBuilt<R, N>) {
    return false;
  } else {
  EngineParams<R, N> E;
  Batch none{};
  fill_params<R, N>(E.P, L, none);
  E.P.tiles = EL.dtiles;
  E.batches = EL.batches;
  E.nbatches = EL.nbatches;
  E.npasses = L.mode == 1 ? 2 : 4;
  E.ntasks = EL.ntasks;
  E.head = EL.head;
  E.done = EL.done;
  E.status = EL.status;
  E.mode = L.mode;
  E.spin_limit = EL.spin_limit;
  E.wait_bias = EL.wait_bias;
  cudaLaunchConfig_t cfg{};
  long long blocks = EL.blocks;
  if (blocks > EL.ntasks) blocks = EL.ntasks;
  if (blocks < 1) return true;
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kEngineThreads);
  cfg.dynamicSmemBytes = EL.smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;   // all blocks co-resident (required by the waits)
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if constexpr (sizeof(R) == 8) {
    if (L.real_io) {
      cudaLaunchKernelEx(&cfg, pair_engine_kernel<R, N, true>, E);
      return true;
    }
  }
  if (L.real_io) return false;
  cudaLaunchKernelEx(&cfg, pair_engine_kernel<R, N, false>, E);
  return true;
  }
}

template <typename R, int N>
bool launch_edge(const PairLaunch& L, const Batch& b, cudaStream_t st) {
  constexpr int IPB = plane_items<R, N>();
  constexpr size_t smem = (size_t)IPB * N * (N + 1) * sizeof(cplx<R>);
  if (L.prepare_only) {
    // opt in to > 48 KB of dynamic shared memory and the largest carveout; done
    // once at plan creation on the plan's device, never during stream capture
    if constexpr (!kSplitPlanes<R, N>) {   // whole lines per thread
      if constexpr (sizeof(R) == 8) {
        cudaFuncSetAttribute(pass_a_kernel<R, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(pass_a_kernel<R, N, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      }
      cudaFuncSetAttribute(pass_a_kernel<R, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(pass_c_kernel<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(pass_a_kernel<R, N, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      cudaFuncSetAttribute(pass_c_kernel<R, N>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    } else {
      constexpr int s1 = (int)kSplitSmem<R, N>;
      if constexpr (sizeof(R) == 8) {
        cudaFuncSetAttribute(pass_a_split_kernel<R, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1);
        cudaFuncSetAttribute(pass_a_split_kernel<R, N, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      }
      cudaFuncSetAttribute(pass_a_split_kernel<R, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1);
      cudaFuncSetAttribute(pass_c_split_kernel<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1);
      cudaFuncSetAttribute(pass_a_split_kernel<R, N, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      cudaFuncSetAttribute(pass_c_split_kernel<R, N>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    return true;
  }
  PairParams<R, N> P;
  fill_params<R, N>(P, L, b);
  auto mark = [&](int k) { if (L.ev) cudaEventRecord(L.ev[k], st); };
  const long long items = (long long)b.npairs * N;
  const dim3 pblk(N * IPB);
  const unsigned pgrid = (unsigned)((items + IPB - 1) / IPB);
  const unsigned bgrid = (unsigned)(((long long)b.npairs * N * N + 255) / 256);
  const dim3 dgrid((unsigned)(((long long)N * N * N + kDSplitPts - 1) / kDSplitPts), (unsigned)b.ntiles);
  if constexpr (sizeof(R) != 8) {
    if (L.real_io) return false;
  }
  const int mask = L.pass_mask ? L.pass_mask : 15;
  mark(0);
  if (mask & 1) {
    if constexpr (kSplitPlanes<R, N>) {
      if (sizeof(R) == 8 && L.real_io)
        launch_pdl(!L.no_pdl, pass_a_split_kernel<R, N, sizeof(R) == 8>, dim3((unsigned)items), dim3(2 * N),
                   kSplitSmem<R, N>, st, P);
      else
        launch_pdl(!L.no_pdl, pass_a_split_kernel<R, N, false>, dim3((unsigned)items), dim3(2 * N), kSplitSmem<R, N>,
                   st, P);
    } else if constexpr (sizeof(R) == 8) {
      if (L.real_io) launch_pdl(!L.no_pdl, pass_a_kernel<R, N, true>, dim3(pgrid), pblk, smem, st, P);
      else launch_pdl(!L.no_pdl, pass_a_kernel<R, N, false>, dim3(pgrid), pblk, smem, st, P);
    } else {
      launch_pdl(!L.no_pdl, pass_a_kernel<R, N, false>, dim3(pgrid), pblk, smem, st, P);
    }
  }
  mark(1);
  if (mask & 2) {
    if constexpr (N >= 64) {
      const unsigned sgrid = (unsigned)(((long long)b.npairs * N * N + kBSplitPencils - 1) / kBSplitPencils);
      launch_pdl(!L.no_pdl, pass_b_split_kernel<R, N>, dim3(sgrid), dim3(256), 0, st, P, L.mode);
    } else {
      launch_pdl(!L.no_pdl, pass_b_kernel<R, N>, dim3(bgrid), dim3(256), 0, st, P, L.mode);
    }
  }
  mark(2);
  if (L.mode == 1) {
    mark(3);
    mark(4);
    return true;
  }
  if (mask & 4) {
    if constexpr (kSplitPlanes<R, N>)
      launch_pdl(!L.no_pdl, pass_c_split_kernel<R, N>, dim3((unsigned)items), dim3(2 * N), kSplitSmem<R, N>, st, P);
    else
      launch_pdl(!L.no_pdl, pass_c_kernel<R, N>, dim3(pgrid), pblk, smem, st, P);
  }
  mark(3);
  if (mask & 8) {
    if constexpr (sizeof(R) == 8) {
      if (L.real_io) launch_pdl(!L.no_pdl, pass_d_kernel<R, N, true>, dgrid, dim3(256), 0, st, P);
      else launch_pdl(!L.no_pdl, pass_d_kernel<R, N, false>, dgrid, dim3(256), 0, st, P);
    } else {
      launch_pdl(!L.no_pdl, pass_d_kernel<R, N, false>, dgrid, dim3(256), 0, st, P);
    }
  }
  mark(4);
  return true;
}

}  // namespace ace
