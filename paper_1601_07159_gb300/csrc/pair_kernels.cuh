// Pair FFT-Poisson solves: the hot loop of Eq. applyVX / Eq. W.
//
// For a batch of pairs (l, r) the 3-D solve v = F^-1[ K F[conj(x_l) y_r] ] is
// split into three passes over the batch's spectrum scratch S, each pass a
// set of register-resident line FFTs (fft_reg.cuh), plus one accumulate pass:
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
//                           each output per tile, fixed summation order.
//
// Tiles within a batch touch disjoint outputs (the schedule guarantees it), so
// pass D needs no atomics and the result is bitwise reproducible.
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

// Programmatic dependent launch: every pass is launched with programmatic
// stream serialisation, so its blocks can be scheduled while the previous pass
// drains; griddep_wait() blocks until the previous grid has completed and its
// writes are visible, and is called before the first access to data that grid
// produced (or will still read). Without the launch attribute both are no-ops.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename Kern, typename Arg>
inline void launch_pdl(Kern kern, dim3 grid, dim3 block, size_t smem, cudaStream_t st, const Arg& arg) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, arg);
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

template <typename R, int N> __host__ __device__ constexpr int plane_items() {
  // items (pair, z-plane) per CTA: ~256 threads, <= 96 KB of padded planes
  constexpr int by_threads = (256 / N) > 0 ? (256 / N) : 1;
  constexpr int by_smem = (96 * 1024) / (N * (N + 1) * (int)sizeof(cplx<R>));
  constexpr int v = by_threads < by_smem ? by_threads : by_smem;
  return v > 0 ? v : 1;
}

// ---------------------------------------------------------------- pass A
template <typename R, int N, bool REAL>
__global__ void __launch_bounds__(N * plane_items<R, N>(), 2)
pass_a_kernel(const __grid_constant__ PairParams<R, N> P) {
  constexpr int IPB = plane_items<R, N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* buf = reinterpret_cast<cplx<R>*>(smem_raw) + threadIdx.y * N * (N + 1);
  const int tx = threadIdx.x;
  const long long item = (long long)blockIdx.x * IPB + threadIdx.y;
  const bool active = item < (long long)P.npairs * N;
  griddep_launch();
  int p = 0, z = 0, l = 0, r = 0;
  if (active) {
    p = (int)(item / N);
    z = (int)(item % N);
    decode_pair(P.tiles, P.ntiles, p, l, r);
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
    griddep_wait();                           // the previous batch's pass D still reads S
    cplx<R>* out = P.S + ((long long)p * N + z) * N * N + tx;
#pragma unroll
    for (int kx = 0; kx < N; ++kx) out[kx * N] = b[kx];
  }
}

// ---------------------------------------------------------------- pass B
// MODE 0: Poisson (forward z, K, inverse z); 1: energy only; 2: both.
template <typename R, int N, int MODE>
__global__ void __launch_bounds__(256)
pass_b_kernel(const __grid_constant__ PairParams<R, N> P) {
  constexpr int N2 = N * N;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = gid < (long long)P.npairs * N2;
  double e = 0.0;
  griddep_launch();
  griddep_wait();
  if (active) {
    const int p = (int)(gid / N2);
    const int f = (int)(gid % N2);
    cplx<R>* s = P.S + (long long)p * N * N2 + f;
    cplx<R> a[N];
#pragma unroll
    for (int zz = 0; zz < N; ++zz) a[zz] = s[(long long)zz * N2];
    dft<N, N, false, R>(a, P.tw);
    if constexpr (MODE != 0) {
      int l, r;
      decode_pair(P.tiles, P.ntiles, p, l, r);
      R acc = R(0);
#pragma unroll
      for (int kz = 0; kz < N; ++kz) {
        const R k = P.Kt[kz * N2 + f];
        acc += k * (a[kz].x * a[kz].x + a[kz].y * a[kz].y);
      }
      e = (l == r ? 1.0 : 2.0) * (double)acc;
    }
    if constexpr (MODE != 1) {
#pragma unroll
      for (int kz = 0; kz < N; ++kz) a[kz] = cscale(a[kz], P.Kt[kz * N2 + f]);
      dft<N, N, true, R>(a, P.tw);
#pragma unroll
      for (int zz = 0; zz < N; ++zz) s[(long long)zz * N2] = a[zz];
    }
  }
  if constexpr (MODE != 0) {
    // deterministic block sum -> Epart[blockIdx.x] += sum (one owner per slot)
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      P.Epart[blockIdx.x] += s;
    }
  }
}

// ---------------------------------------------------------------- pass C
template <typename R, int N>
__global__ void __launch_bounds__(N * plane_items<R, N>(), 2)
pass_c_kernel(const __grid_constant__ PairParams<R, N> P) {
  constexpr int IPB = plane_items<R, N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* buf = reinterpret_cast<cplx<R>*>(smem_raw) + threadIdx.y * N * (N + 1);
  const int tx = threadIdx.x;
  const long long item = (long long)blockIdx.x * IPB + threadIdx.y;
  const bool active = item < (long long)P.npairs * N;
  cplx<R>* plane = nullptr;
  griddep_launch();
  griddep_wait();
  if (active) {
    const int p = (int)(item / N);
    const int z = (int)(item % N);
    plane = P.S + ((long long)p * N + z) * N * N;
    cplx<R> b[N];
#pragma unroll
    for (int kx = 0; kx < N; ++kx) b[kx] = plane[kx * N + tx];   // row ky = tx
    dft<N, N, true, R>(b, P.tw);                                   // inverse along x
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
    for (int y = 0; y < N; ++y) plane[y * N + tx] = a[y];
  }
}

// ---------------------------------------------------------------- pass D
template <typename R, bool REAL>
__device__ __forceinline__ void rmw_out(void* base, long long idx, cplx<R> acc, R scale) {
  if constexpr (REAL) {
    R* o = static_cast<R*>(base) + idx;
    *o = *o - scale * acc.x;
  } else {
    cplx<R>* o = static_cast<cplx<R>*>(base) + idx;
    const cplx<R> c = *o;
    *o = cmk<cplx<R>>(c.x - scale * acc.x, c.y - scale * acc.y);
  }
}

// Full tiles (kTileMax orbitals per side): no runtime guards, so all loads of
// the tile's pair potentials can be issued back to back. v is read once, so it
// is loaded with the streaming (evict-first) hint.
template <typename R, int N, bool REAL>
__device__ __forceinline__ void pass_d_full_diag(const PairParams<R, N>& P, const TileDesc& d,
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
  for (int o = 0; o < B; ++o) rmw_out<R, REAL>(P.OutY, (long long)(d.l0 + o) * P.ld + g, acc[o], P.scale);
}

template <typename R, int N, bool REAL>
__device__ __forceinline__ void pass_d_full_off(const PairParams<R, N>& P, const TileDesc& d,
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
    rmw_out<R, REAL>(P.OutY, (long long)(d.r0 + o) * P.ld + g, ar[o], P.scale);
    rmw_out<R, REAL>(P.OutX, (long long)(d.l0 + o) * P.ld + g, al[o], P.scale);
  }
}

template <typename R, int N, bool REAL>
__global__ void __launch_bounds__(256)
pass_d_kernel(const __grid_constant__ PairParams<R, N> P) {
  constexpr long long NG = (long long)N * N * N;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  griddep_launch();
  if (g >= NG) return;
  griddep_wait();
  const TileDesc d = P.tiles[blockIdx.y];
  const cplx<R>* V = P.S + (long long)d.slot0 * NG + g;
  if (d.kind == 1 && d.nl == kTileMax) {
    pass_d_full_diag<R, N, REAL>(P, d, V, g);
  } else if (d.kind == 0 && d.nl == kTileMax && d.nr == kTileMax) {
    pass_d_full_off<R, N, REAL>(P, d, V, g);
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
          const cplx<R> v = V[(long long)q * NG];
          ++q;
          acc[ri] = cadd(acc[ri], cmul(x[li], v));
          if (ri != li) acc[li] = cadd(acc[li], cmulc(v, x[ri]));   // x_r conj(v)
        }
      }
    }
#pragma unroll
    for (int o = 0; o < kTileMax; ++o)
      if (o < d.nl) rmw_out<R, REAL>(P.OutY, (long long)(d.l0 + o) * P.ld + g, acc[o], P.scale);
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
          const cplx<R> v = V[(long long)(li * d.nr + ri) * NG];
          ar[ri] = cadd(ar[ri], cmul(xl[li], v));
          al[li] = cadd(al[li], cmulc(v, yr[ri]));
        }
      }
    }
#pragma unroll
    for (int o = 0; o < kTileMax; ++o) {
      if (o < d.nr) rmw_out<R, REAL>(P.OutY, (long long)(d.r0 + o) * P.ld + g, ar[o], P.scale);
      if (o < d.nl) rmw_out<R, REAL>(P.OutX, (long long)(d.l0 + o) * P.ld + g, al[o], P.scale);
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
          const cplx<R> v = V[(long long)(li * d.nr + ri) * NG];
          ar[ri] = cadd(ar[ri], cmul(xv, v));
        }
      }
    }
#pragma unroll
    for (int o = 0; o < kTileMax; ++o)
      if (o < d.nr) rmw_out<R, REAL>(P.OutY, (long long)(d.r0 + o) * P.ld + g, ar[o], P.scale);
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

template <typename R, int N>
bool launch_edge(const PairLaunch& L, const Batch& b, cudaStream_t st) {
  constexpr int IPB = plane_items<R, N>();
  constexpr size_t smem = (size_t)IPB * N * (N + 1) * sizeof(cplx<R>);
  if (L.prepare_only) {
    // opt in to > 48 KB of dynamic shared memory and the largest carveout; done
    // once at plan creation on the plan's device, never during stream capture
    cudaFuncSetAttribute(pass_a_kernel<R, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(pass_a_kernel<R, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(pass_c_kernel<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(pass_a_kernel<R, N, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(pass_a_kernel<R, N, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(pass_c_kernel<R, N>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return true;
  }
  PairParams<R, N> P;
  fill_params<R, N>(P, L, b);
  auto mark = [&](int k) { if (L.ev) cudaEventRecord(L.ev[k], st); };
  const long long items = (long long)b.npairs * N;
  const dim3 pblk(N, IPB);
  const unsigned pgrid = (unsigned)((items + IPB - 1) / IPB);
  const unsigned bgrid = (unsigned)(((long long)b.npairs * N * N + 255) / 256);
  const dim3 dgrid((unsigned)(((long long)N * N * N + 255) / 256), (unsigned)b.ntiles);
  mark(0);
  if (L.real_io) launch_pdl(pass_a_kernel<R, N, true>, dim3(pgrid), pblk, smem, st, P);
  else launch_pdl(pass_a_kernel<R, N, false>, dim3(pgrid), pblk, smem, st, P);
  mark(1);
  if (L.mode == 0) launch_pdl(pass_b_kernel<R, N, 0>, dim3(bgrid), dim3(256), 0, st, P);
  else if (L.mode == 1) launch_pdl(pass_b_kernel<R, N, 1>, dim3(bgrid), dim3(256), 0, st, P);
  else launch_pdl(pass_b_kernel<R, N, 2>, dim3(bgrid), dim3(256), 0, st, P);
  mark(2);
  if (L.mode == 1) {
    mark(3);
    mark(4);
    return true;
  }
  launch_pdl(pass_c_kernel<R, N>, dim3(pgrid), pblk, smem, st, P);
  mark(3);
  if (L.real_io) launch_pdl(pass_d_kernel<R, N, true>, dgrid, dim3(256), 0, st, P);
  else launch_pdl(pass_d_kernel<R, N, false>, dgrid, dim3(256), 0, st, P);
  mark(4);
  return true;
}

}  // namespace ace
