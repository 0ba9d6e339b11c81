// Pair FFT-Poisson solves: the hot loop of Eq. applyVX / Eq. W.
//
// For a batch of pairs (l, r) the 3-D solve v = F^-1[ K F[conj(x_l) y_r] ] on an
// n_x x n_y x n_z grid is split into three passes over the batch's spectrum
// scratch S, each a set of register-resident line FFTs (fft_reg.cuh), plus one
// accumulate pass:
//
//   pass A  (per z-plane)   rho = conj(x_l) y_r; FFT along y (thread = column x,
//                           coalesced loads), transpose through shared memory,
//                           FFT along x (thread = row ky); store S[z][kx][ky]
//                           (coalesced along ky). Blocks run z-plane major, so
//                           the pairs of a tile that read the same orbital
//                           plane run together and find it in L2.
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
// The plane passes are compiled per (n_x, n_y), the pencil pass per n_z (the
// pencil's (kx, ky) position is a run-time index), the accumulate pass once per
// precision; a grid n_x x n_y x n_z runs when its plane and its pencil length
// are compiled in. On cubic grids passes B and D use instances with the grid
// compiled in (strides and offsets folded into the instructions). At the
// larger edges a line is held by two lanes instead of one thread
// (split_line_dft): the plane passes when the longer plane edge is >= 48
// (FP64: >= 64), FP64 pass B from n_z = 64; FP32 pencils of 64 and 96 are
// spread over four warps (pass_b_quad_kernel).
//
// Real vectors (R64) pack two pairs into one complex solve: a slot holds
// rho_lr + i rho_lr' (decode_slot_real), the kernel being real and even keeps
// V_lr and V_lr' in the real and imaginary parts, and pass D splits them.
//
// Two ways to run a schedule of batches:
//  * four kernels per batch (pass_*_kernel), chained with programmatic
//    dependent launch, replayed from a CUDA graph (the default) or launched
//    eagerly (per-pass timing);
//  * one persistent launch (pair_engine_kernel, cubic grids): co-resident
//    blocks take tasks (one pass-A/C block of planes, one pass-B block of
//    pencils, one pass-D block of points) in schedule order from an atomic
//    queue and wait, with a bounded spin, on per-batch completion counters:
//    pass p of batch k needs all of pass p-1 of batch k, pass A of batch k
//    needs the last pass of batch k-1 (the scratch is reused). Tasks are taken
//    in increasing order by resident blocks, so every awaited task is already
//    running: no deadlock.
//
// Tiles within a batch touch disjoint outputs (the schedule guarantees it) and
// batches run in order, so the accumulation needs no atomics and the result is
// bitwise reproducible. The engine sums a full off-diagonal tile's left
// outputs in one thread rather than two, so the two modes agree to rounding.
#pragma once
#include "ace_internal.h"
#include "fft_reg.cuh"


namespace ace {
inline namespace ACE_RADIX_NS {   // radix order of this translation unit (fft_reg.cuh)

// Twiddle tables of a plane: one per axis, shared when the plane is square.
template <typename R, int NX, int NY> struct PlaneTw {
  TwTable<R, NX> x;
  TwTable<R, NY> y;
  __device__ __forceinline__ const TwTable<R, NX>& tx() const { return x; }
  __device__ __forceinline__ const TwTable<R, NY>& ty() const { return y; }
  void fill(const double* twx, const double* twy) {
    for (int k = 0; k < NX; ++k) { x.w[k].x = (R)twx[2 * k]; x.w[k].y = (R)twx[2 * k + 1]; }
    for (int k = 0; k < NY; ++k) { y.w[k].x = (R)twy[2 * k]; y.w[k].y = (R)twy[2 * k + 1]; }
  }
};
template <typename R, int N> struct PlaneTw<R, N, N> {
  TwTable<R, N> x;
  __device__ __forceinline__ const TwTable<R, N>& tx() const { return x; }
  __device__ __forceinline__ const TwTable<R, N>& ty() const { return x; }
  void fill(const double* twx, const double*) {
    for (int k = 0; k < N; ++k) { x.w[k].x = (R)twx[2 * k]; x.w[k].y = (R)twx[2 * k + 1]; }
  }
};

// Passes A and C: the pair's vectors (pass A), the scratch, nz z-planes per pair.
template <typename R, int NX, int NY> struct PlaneParams {
  const void* X;
  const void* Y;
  cplx<R>* S;
  long long ld;
  int nz;
  int npairs;
  const TileDesc* tiles;   // device table of the batch's tiles
  int ntiles;
  PlaneTw<R, NX, NY> tw;
};

// Pass B: pencils of NZ points at the nxy = n_x n_y positions (kx, ky) of a plane.
template <typename R, int NZ> struct PencilParams {
  cplx<R>* S;
  const R* Kt;             // K(G) alpha / N_g, folded [kz][kx][ky] over 0..n/2 per axis
  double* Epart;
  int npairs;
  int nx, ny, nxy;
  int khy, kzs;            // folded table: row length n_y/2 + 1, kz stride (n_x/2 + 1)(n_y/2 + 1)
  const TileDesc* tiles;
  int ntiles;
  int packed;              // real vectors: two pairs per slot (energy weights by decode_slot_real)
  TwTable<R, NZ> tw;
};

// Pass D: the tile's vectors and outputs, the pair potentials in S.
template <typename R> struct PointParams {
  const void* X;
  const void* Y;
  void* OutX;
  void* OutY;
  const cplx<R>* S;
  long long ld;
  long long ng;
  R scale;
  const TileDesc* tiles;
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

// Slot s of a batch of real vectors -> tile index and the slot's pairs (l, r)
// (real part) and (l, r2) (imaginary part; r2 < 0: none). Diagonal tile row
// li: the slot (l, l) alone, then (l, l + 1 + 2m), (l, l + 2 + 2m); other
// tiles: row li holds (l, r0 + 2m), (l, r0 + 2m + 1).
__device__ __forceinline__ int decode_slot_real(const TileDesc* __restrict__ tiles, int ntiles, int s, int& l,
                                                int& r, int& r2) {
  int t = 0;
  while (t + 1 < ntiles && tiles[t + 1].slot0 <= s) ++t;
  const TileDesc d = tiles[t];
  int q = s - d.slot0;
  if (d.kind == 1) {
    int li = 0, len = 1 + d.nl / 2;
    while (q >= len) { q -= len; ++li; len = 1 + (d.nl - li) / 2; }
    l = d.l0 + li;
    r = q == 0 ? l : l + 2 * q - 1;
    r2 = (q != 0 && r + 1 < d.l0 + d.nl) ? r + 1 : -1;
  } else {
    const int w = (d.nr + 1) / 2;
    l = d.l0 + q / w;
    r = d.r0 + 2 * (q % w);
    r2 = r + 1 < d.r0 + d.nr ? r + 1 : -1;
  }
  return t;
}

// Energy weight of slot p: 1 for the diagonal pair (l, l), 2 otherwise (the
// pair and its mirror (r, l)).
__device__ __forceinline__ double slot_weight(const TileDesc* __restrict__ tiles, int ntiles, int p, bool real) {
  int l, r, r2;
  if (real) decode_slot_real(tiles, ntiles, p, l, r, r2);
  else decode_pair(tiles, ntiles, p, l, r);
  return l == r ? 1.0 : 2.0;
}

template <typename R, bool REAL>
__device__ __forceinline__ cplx<R> load_vec(const void* base, long long idx) {
  if constexpr (REAL) {
    return cmk<cplx<R>>(static_cast<const R*>(base)[idx], R(0));
  } else {
    return static_cast<const cplx<R>*>(base)[idx];
  }
}

// The kernel table is folded (K depends on |G|^2 only): index k of an axis of
// n points and n - k share an entry. kfold(k) = min(k, n - k).
template <int N> __host__ __device__ __forceinline__ constexpr int kfold(int k) { return k <= N / 2 ? k : N - k; }
__host__ __device__ __forceinline__ int kfold_rt(int k, int n) { return k <= n / 2 ? k : n - k; }
// Plane geometry seen by the pencil pass: compile-time for cubic grids
// (CUBE: n_x = n_y = n_z, so strides and table offsets fold into the
// instructions), read from the parameters otherwise.
template <typename R, int NZ, bool CUBE> struct PencilGeom {
  int nx, ny, nxy, khy, kzs;
  __device__ __forceinline__ explicit PencilGeom(const PencilParams<R, NZ>& P) {
    if constexpr (CUBE) {
      nx = NZ; ny = NZ; nxy = NZ * NZ; khy = NZ / 2 + 1; kzs = (NZ / 2 + 1) * (NZ / 2 + 1);
    } else {
      nx = P.nx; ny = P.ny; nxy = P.nxy; khy = P.khy; kzs = P.kzs;
    }
  }
  // offset of the (kx, ky) pencil f = kx n_y + ky in the folded table
  __device__ __forceinline__ int kt_pencil(int f) const {
    const int kx = f / ny, ky = f - kx * ny;
    return kfold_rt(kx, nx) * khy + kfold_rt(ky, ny);
  }
};

template <int NX, int NY> constexpr int kMaxLine = NX > NY ? NX : NY;

template <typename R, int NX, int NY> __host__ __device__ constexpr int plane_items() {
  // items (pair, z-plane) per CTA of the plane kernels: ~256 threads, <= 96 KB
  constexpr int ML = kMaxLine<NX, NY>;
  constexpr int by_threads = (256 / ML) > 0 ? (256 / ML) : 1;
  constexpr int by_smem = (96 * 1024) / (NY * (NX + 1) * (int)sizeof(cplx<R>));
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
// Pass A on virtual block `vb` (IPB plane items, thread tid = ty * max(NX, NY) + tx).
template <typename R, int NX, int NY, bool REAL, bool COH, int IPB, bool PDL>
__device__ __forceinline__ void body_a(const PlaneParams<R, NX, NY>& P, const TileDesc* tiles, int ntiles,
                                       int npairs, cplx<R>* smem, long long vb, int tid) {
  constexpr int ML = kMaxLine<NX, NY>;
  const int tx = tid % ML, ty = tid / ML;
  cplx<R>* buf = smem + ty * NY * (NX + 1);
  const long long item = vb * IPB + ty;
  const bool active = ty < IPB && item < (long long)npairs * P.nz;
  int p = 0, z = 0, l = 0, r = 0, r2 = -1;
  if (active) {   // z-plane major: the pairs of a tile that share an orbital plane run together
    z = (int)(item / npairs);
    p = (int)(item % npairs);
    if constexpr (REAL) decode_slot_real(tiles, ntiles, p, l, r, r2);
    else decode_pair(tiles, ntiles, p, l, r);
  }
  if (active && tx < NX) {
    cplx<R> a[NY];
    const long long xo = (long long)l * P.ld + (long long)z * NX * NY + tx;
    const long long yo = (long long)r * P.ld + (long long)z * NX * NY + tx;
    if constexpr (REAL) {                     // x_l (y_r + i y_r2)
      const R* Xr = static_cast<const R*>(P.X);
      const R* Yr = static_cast<const R*>(P.Y);
      const bool two = r2 >= 0;
      const long long y2o = (long long)(two ? r2 : r) * P.ld + (long long)z * NX * NY + tx;
#pragma unroll
      for (int y = 0; y < NY; ++y) {
        const R xv = Xr[xo + y * NX];
        a[y] = cmk<cplx<R>>(xv * Yr[yo + y * NX], two ? xv * Yr[y2o + y * NX] : R(0));
      }
    } else {
#pragma unroll
      for (int y = 0; y < NY; ++y) {
        const cplx<R> xv = load_vec<R, REAL>(P.X, xo + y * NX);
        const cplx<R> yv = load_vec<R, REAL>(P.Y, yo + y * NX);
        a[y] = cmulc(xv, yv);                 // conj(x_l) * y_r
      }
    }
    dft<NY, NY, false, R>(a, P.tw.ty());      // along y, column x = tx
#pragma unroll
    for (int k = 0; k < NY; ++k) buf[k * (NX + 1) + tx] = a[k];
  }
  __syncthreads();
  if (active && tx < NY) {
    cplx<R> b[NX];
#pragma unroll
    for (int x = 0; x < NX; ++x) b[x] = buf[tx * (NX + 1) + x];
    dft<NX, NX, false, R>(b, P.tw.tx());      // along x, row ky = tx
    if constexpr (PDL) griddep_wait();        // the previous batch's pass D still reads S
    cplx<R>* out = P.S + ((long long)p * P.nz + z) * NX * NY + tx;
#pragma unroll
    for (int kx = 0; kx < NX; ++kx) stx<COH>(out + kx * NY, b[kx]);
  }
}

// Pass B on virtual block `vb` of `nthr` pencils. mode 0: Poisson (forward z,
// K, inverse z); 1: energy only; 2: both. The energy partial of the block
// (mode != 0) is added to *eslot by thread 0 (one owner per slot).
template <typename R, int NZ, bool COH, bool CUBE>
__device__ __forceinline__ void body_b(const PencilParams<R, NZ>& P, const TileDesc* tiles, int ntiles, int npairs,
                                       int mode, long long vb, int tid, int nthr, double* red, double* eslot) {
  const PencilGeom<R, NZ, CUBE> G(P);
  const int nxy = G.nxy;
  const long long gid = vb * nthr + tid;
  const bool active = gid < (long long)npairs * nxy;
  double e = 0.0;
  if (active) {
    const int p = (int)(gid / nxy);
    const int f = (int)(gid % nxy);
    cplx<R>* s = P.S + (long long)p * NZ * nxy + f;
    cplx<R> a[NZ];
#pragma unroll
    for (int zz = 0; zz < NZ; ++zz) a[zz] = ldx<COH>(s + (long long)zz * nxy);
    dft<NZ, NZ, false, R>(a, P.tw);
    R acc = R(0);
    const R* kt = P.Kt + G.kt_pencil(f);
#pragma unroll
    for (int kz = 0; kz < NZ; ++kz) {
      const R k = kt[kfold<NZ>(kz) * G.kzs];
      if (mode != 0) acc += k * (a[kz].x * a[kz].x + a[kz].y * a[kz].y);
      a[kz] = cscale(a[kz], k);
    }
    if (mode != 0) e = slot_weight(tiles, ntiles, p, P.packed) * (double)acc;
    if (mode != 1) {
      dft<NZ, NZ, true, R>(a, P.tw);
#pragma unroll
      for (int zz = 0; zz < NZ; ++zz) stx<COH>(s + (long long)zz * nxy, a[zz]);
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
template <typename R, int NX, int NY, bool COH, int IPB>
__device__ __forceinline__ void body_c(const PlaneParams<R, NX, NY>& P, int npairs, cplx<R>* smem, long long vb,
                                       int tid) {
  constexpr int ML = kMaxLine<NX, NY>;
  const int tx = tid % ML, ty = tid / ML;
  cplx<R>* buf = smem + ty * NY * (NX + 1);
  const long long item = vb * IPB + ty;
  const bool active = ty < IPB && item < (long long)npairs * P.nz;
  cplx<R>* plane = nullptr;
  if (active) {
    const int p = (int)(item / P.nz);
    const int z = (int)(item % P.nz);
    plane = P.S + ((long long)p * P.nz + z) * NX * NY;
  }
  if (active && tx < NY) {
    cplx<R> b[NX];
#pragma unroll
    for (int kx = 0; kx < NX; ++kx) b[kx] = ldx<COH>(plane + kx * NY + tx);   // row ky = tx
    dft<NX, NX, true, R>(b, P.tw.tx());                                      // inverse along x
#pragma unroll
    for (int x = 0; x < NX; ++x) buf[tx * (NX + 1) + x] = b[x];
  }
  __syncthreads();
  if (active && tx < NX) {
    cplx<R> a[NY];
#pragma unroll
    for (int ky = 0; ky < NY; ++ky) a[ky] = buf[ky * (NX + 1) + tx];  // column x = tx
    dft<NY, NY, true, R>(a, P.tw.ty());                               // inverse along y
#pragma unroll
    for (int y = 0; y < NY; ++y) stx<COH>(plane + y * NX + tx, a[y]);
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
template <typename R, bool REAL, bool COH, long long NGC>
__device__ __forceinline__ void d_full_diag(const PointParams<R>& P, const TileDesc& d,
                                            const cplx<R>* __restrict__ V, long long g) {
  const long long NG = NGC ? NGC : P.ng;
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
      acc[ri] = cfma(acc[ri], x[li], v);
      if (ri != li) acc[li] = cfmac(acc[li], v, x[ri]);
    }
  }
#pragma unroll
  for (int o = 0; o < B; ++o) rmw_out<R, REAL, COH>(P.OutY, (long long)(d.l0 + o) * P.ld + g, acc[o], P.scale);
}

template <typename R, bool REAL, bool COH, long long NGC>
__device__ __forceinline__ void d_full_off(const PointParams<R>& P, const TileDesc& d,
                                           const cplx<R>* __restrict__ V, long long g) {
  const long long NG = NGC ? NGC : P.ng;
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
      ar[ri] = cfma(ar[ri], xl[li], v);
      al[li] = cfmac(al[li], v, yr[ri]);
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
template <typename R, bool REAL, long long NGC>
__device__ __forceinline__ void d_split_off(const PointParams<R>& P, const TileDesc& d, long long vbx, int tid,
                                            cplx<R>* xch) {
  const long long NG = NGC ? NGC : P.ng;
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
        ar[ri] = cfma(ar[ri], xl[li], v);
        al[li] = cfmac(al[li], v, yr[ri]);
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

// Pass D (complex vectors) for point block `vbx` (nthr points) of tile `d`;
// NGC = N_g at compile time (cubic grids) or 0 (read from the parameters).
template <typename R, bool REAL, bool COH, bool FULL_OFF, long long NGC>
__device__ __forceinline__ void body_d_cplx(const PointParams<R>& P, const TileDesc& d, long long vbx, int tid,
                                            int nthr) {
  const long long NG = NGC ? NGC : P.ng;
  const long long g = vbx * nthr + tid;
  if (g >= NG) return;
  const cplx<R>* V = P.S + (long long)d.slot0 * NG + g;
  if (d.kind == 1 && d.nl == kTileMax) {
    d_full_diag<R, REAL, COH, NGC>(P, d, V, g);
  } else if (FULL_OFF && d.kind == 0 && d.nl == kTileMax && d.nr == kTileMax) {
    d_full_off<R, REAL, COH, NGC>(P, d, V, g);
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
          acc[ri] = cfma(acc[ri], x[li], v);
          if (ri != li) acc[li] = cfmac(acc[li], v, x[ri]);   // x_r conj(v)
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
          ar[ri] = cfma(ar[ri], xl[li], v);
          al[li] = cfmac(al[li], v, yr[ri]);
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
          ar[ri] = cfma(ar[ri], xv, v);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < kTileMax; ++o)
      if (o < d.nr) rmw_out<R, REAL, COH>(P.OutY, (long long)(d.r0 + o) * P.ld + g, ar[o], P.scale);
  }
}

// ---- pass D for real vectors: a slot holds v = V_lr + i V_lr2 (decode_slot_real)
template <typename R, bool COH>
__device__ __forceinline__ void rmw_real(void* base, long long idx, R acc, R scale) {
  R* o = static_cast<R*>(base) + idx;
  stx<COH>(o, ldx<COH>(o) - scale * acc);
}
// full tiles read their potentials once, with the streaming hint
template <bool FULL, bool COH, typename T> __device__ __forceinline__ T ldv(const T* p) {
  if constexpr (FULL) return __ldcs(p);
  else return ldx<COH>(p);
}

// Diagonal tile: Out_l -= sum over its pairs; a pair (l, r != l) feeds both
// Out_r (x_l V_lr) and Out_l (x_r V_lr), the pair (l, l) Out_l once.
template <typename R, bool COH, bool FULL, long long NGC>
__device__ __forceinline__ void d_real_diag(const PointParams<R>& P, const TileDesc& d, const cplx<R>* V,
                                            long long g) {
  const long long NG = NGC ? NGC : P.ng;
  constexpr int B = kTileMax;
  const int n = FULL ? B : d.nl;
  const R* X = static_cast<const R*>(P.X);
  R x[B], acc[B];
#pragma unroll
  for (int o = 0; o < B; ++o) {
    acc[o] = R(0);
    x[o] = (FULL || o < n) ? X[(long long)(d.l0 + o) * P.ld + g] : R(0);
  }
  int q = 0;
#pragma unroll
  for (int li = 0; li < B; ++li) {
    if (FULL || li < n) {
      const cplx<R> v0 = ldv<FULL, COH>(V + (long long)q * NG);
      ++q;
      acc[li] += x[li] * v0.x;
#pragma unroll
      for (int ri = li + 1; ri < B; ri += 2) {
        if (FULL || ri < n) {
          const cplx<R> v = ldv<FULL, COH>(V + (long long)q * NG);
          ++q;
          acc[ri] += x[li] * v.x;
          acc[li] += v.x * x[ri];
          if (ri + 1 < B && (FULL || ri + 1 < n)) {
            acc[ri + 1] += x[li] * v.y;
            acc[li] += v.y * x[ri + 1];
          }
        }
      }
    }
  }
#pragma unroll
  for (int o = 0; o < B; ++o)
    if (FULL || o < n) rmw_real<R, COH>(P.OutY, (long long)(d.l0 + o) * P.ld + g, acc[o], P.scale);
}

// Off-diagonal tile of a symmetric schedule (one thread per point).
template <typename R, bool COH, bool FULL, long long NGC>
__device__ __forceinline__ void d_real_off(const PointParams<R>& P, const TileDesc& d, const cplx<R>* V,
                                           long long g) {
  const long long NG = NGC ? NGC : P.ng;
  constexpr int B = kTileMax, W2 = kTileMax / 2;
  const int nl = FULL ? B : d.nl, nr = FULL ? B : d.nr, w = FULL ? W2 : (d.nr + 1) / 2;
  const R* X = static_cast<const R*>(P.X);
  const R* Y = static_cast<const R*>(P.Y);
  R xl[B], yr[B], al[B], ar[B];
#pragma unroll
  for (int o = 0; o < B; ++o) {
    al[o] = R(0);
    ar[o] = R(0);
    xl[o] = (FULL || o < nl) ? X[(long long)(d.l0 + o) * P.ld + g] : R(0);
    yr[o] = (FULL || o < nr) ? Y[(long long)(d.r0 + o) * P.ld + g] : R(0);
  }
#pragma unroll
  for (int li = 0; li < B; ++li) {
#pragma unroll
    for (int m = 0; m < W2; ++m) {
      if ((FULL || li < nl) && (FULL || 2 * m < nr)) {
        const cplx<R> v = ldv<FULL, COH>(V + (long long)(li * w + m) * NG);
        ar[2 * m] += xl[li] * v.x;
        al[li] += v.x * yr[2 * m];
        if (FULL || 2 * m + 1 < nr) {
          ar[2 * m + 1] += xl[li] * v.y;
          al[li] += v.y * yr[2 * m + 1];
        }
      }
    }
  }
#pragma unroll
  for (int o = 0; o < B; ++o) {
    if (FULL || o < nr) rmw_real<R, COH>(P.OutY, (long long)(d.r0 + o) * P.ld + g, ar[o], P.scale);
    if (FULL || o < nl) rmw_real<R, COH>(P.OutX, (long long)(d.l0 + o) * P.ld + g, al[o], P.scale);
  }
}

// One-sided tile (V_X[Phi] Psi, Poisson solves): Out_r -= sum_l x_l V_lr.
template <typename R, bool COH, long long NGC>
__device__ __forceinline__ void d_real_rect(const PointParams<R>& P, const TileDesc& d, const cplx<R>* V,
                                            long long g) {
  const long long NG = NGC ? NGC : P.ng;
  constexpr int B = kTileMax, W2 = kTileMax / 2;
  const int w = (d.nr + 1) / 2;
  const R* X = static_cast<const R*>(P.X);
  R ar[B];
#pragma unroll
  for (int o = 0; o < B; ++o) ar[o] = R(0);
  for (int li = 0; li < d.nl; ++li) {
    const R xv = X[(long long)(d.l0 + li) * P.ld + g];
#pragma unroll
    for (int m = 0; m < W2; ++m) {
      if (2 * m < d.nr) {
        const cplx<R> v = ldx<COH>(V + (long long)(li * w + m) * NG);
        ar[2 * m] += xv * v.x;
        if (2 * m + 1 < d.nr) ar[2 * m + 1] += xv * v.y;
      }
    }
  }
#pragma unroll
  for (int o = 0; o < B; ++o)
    if (o < d.nr) rmw_real<R, COH>(P.OutY, (long long)(d.r0 + o) * P.ld + g, ar[o], P.scale);
}

// Full off-diagonal tile of real vectors with two threads per point, as
// d_split_off: half h takes the right orbitals r0 + 4h .. r0 + 4h + 3 (slots
// li * 4 + 2h, li * 4 + 2h + 1 of each row).
template <typename R, long long NGC>
__device__ __forceinline__ void d_split_off_real(const PointParams<R>& P, const TileDesc& d, long long vbx, int tid,
                                                 R* xch) {
  const long long NG = NGC ? NGC : P.ng;
  constexpr int B = kTileMax, H = kTileMax / 2, Q = H / 2;
  const int h = (tid >> 5) & 1;
  const int pt = ((tid >> 6) << 5) | (tid & 31);
  const long long g = vbx * kDSplitPts + pt;
  const bool act = g < NG;
  const cplx<R>* V = P.S + (long long)d.slot0 * NG + g;
  const R* X = static_cast<const R*>(P.X);
  const R* Y = static_cast<const R*>(P.Y);
  R xl[B], yr[H], al[B], ar[H];
#pragma unroll
  for (int o = 0; o < B; ++o) {
    al[o] = R(0);
    xl[o] = act ? X[(long long)(d.l0 + o) * P.ld + g] : R(0);
  }
#pragma unroll
  for (int o = 0; o < H; ++o) {
    ar[o] = R(0);
    yr[o] = act ? Y[(long long)(d.r0 + h * H + o) * P.ld + g] : R(0);
  }
  if (act) {
#pragma unroll
    for (int li = 0; li < B; ++li) {
#pragma unroll
      for (int m = 0; m < Q; ++m) {
        const cplx<R> v = __ldcs(V + (long long)(li * H + h * Q + m) * NG);
        ar[2 * m] += xl[li] * v.x;
        ar[2 * m + 1] += xl[li] * v.y;
        al[li] += v.x * yr[2 * m];
        al[li] += v.y * yr[2 * m + 1];
      }
    }
  }
#pragma unroll
  for (int o = 0; o < H; ++o) xch[o * 256 + tid] = h ? al[o] : al[H + o];   // the partner's half
  __syncthreads();
  if (!act) return;
  const int partner = tid ^ 32;
#pragma unroll
  for (int o = 0; o < H; ++o) {
    const R own = h ? al[H + o] : al[o];
    const R other = xch[o * 256 + partner];
    const R lo = h ? other : own, hi = h ? own : other;                    // r-half 0 first, then 1
    rmw_real<R, false>(P.OutX, (long long)(d.l0 + h * H + o) * P.ld + g, lo + hi, P.scale);
    rmw_real<R, false>(P.OutY, (long long)(d.r0 + h * H + o) * P.ld + g, ar[o], P.scale);
  }
}

// Pass D for point block `vbx` (nthr points) of tile `d`.
template <typename R, bool REAL, bool COH, bool FULL_OFF, long long NGC>
__device__ __forceinline__ void body_d(const PointParams<R>& P, const TileDesc& d, long long vbx, int tid,
                                       int nthr) {
  if constexpr (REAL) {
    const long long g = vbx * nthr + tid;
    if (g >= (NGC ? NGC : P.ng)) return;
    const cplx<R>* V = P.S + (long long)d.slot0 * (NGC ? NGC : P.ng) + g;
    if (d.kind == 1) {
      if (d.nl == kTileMax) d_real_diag<R, COH, true, NGC>(P, d, V, g);
      else d_real_diag<R, COH, false, NGC>(P, d, V, g);
    } else if (d.kind == 0) {
      if (FULL_OFF && d.nl == kTileMax && d.nr == kTileMax) d_real_off<R, COH, true, NGC>(P, d, V, g);
      else d_real_off<R, COH, false, NGC>(P, d, V, g);
    } else {
      d_real_rect<R, COH, NGC>(P, d, V, g);
    }
  } else {
    body_d_cplx<R, REAL, COH, FULL_OFF, NGC>(P, d, vbx, tid, nthr);
  }
}

// ---------------------------------------------------------------- four-kernel mode
template <typename R, int NX, int NY, bool REAL>
__global__ void __launch_bounds__(kMaxLine<NX, NY> * plane_items<R, NX, NY>(), 2)
pass_a_kernel(const __grid_constant__ PlaneParams<R, NX, NY> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  griddep_launch();
  body_a<R, NX, NY, REAL, false, plane_items<R, NX, NY>(), true>(
      P, P.tiles, P.ntiles, P.npairs, reinterpret_cast<cplx<R>*>(smem_raw), blockIdx.x, threadIdx.x);
}

template <typename T> __device__ __forceinline__ T shfl_pair(T v) {
  T r;
  r.x = __shfl_xor_sync(0xffffffffu, v.x, 1);
  r.y = __shfl_xor_sync(0xffffffffu, v.y, 1);
  return r;
}

// A length-N transform of a line held by two lanes (lanes 2q, 2q+1): lane h
// holds the samples 2m + h in a[], and on return holds y[j] = Y[hN/4 + j] and
// y[N/4 + j] = Y[hN/4 + j + N/2] (the forward or inverse DFT, unnormalised):
// a DFT of N/2 per lane, the lane-1 twiddles w^{+-k}, one shuffle per value
// and the radix-2 combine (decimation in time).
// The halves are exchanged before the twiddles, so each lane multiplies only
// the H odd-half values of its own outputs (by w^j on lane 0, w^{H+j} on lane
// 1: two compile-time constants, selected).
template <typename R> __device__ __forceinline__ cplx<R> csel(bool c, cplx<R> a, cplx<R> b) {
  return cmk<cplx<R>>(c ? a.x : b.x, c ? a.y : b.y);
}
// The radix-2 step alone, on a[] already holding the half-length transform:
// each output goes to sink(j, Y) as soon as it is formed (y index j as in
// split_line_dft), so a caller that stores it right away frees the registers
// of a[j], a[H + j] within the loop instead of holding a second array.
template <int N, bool INV, typename R, typename Sink>
__device__ __forceinline__ void split_combine(const cplx<R> (&a)[N / 2], int h, const TwTable<R, N>& tw,
                                              Sink sink) {
  using C = cplx<R>;
  constexpr int H = N / 4;
#pragma unroll
  for (int j = 0; j < H; ++j) {
    const C recv = shfl_pair(h ? a[j] : a[H + j]);       // lane 0 gets O[j], lane 1 gets E[H + j]
    const C ev = h ? recv : a[j];                        // E[hH + j]
    const C od = h ? a[H + j] : recv;                    // O[hH + j]
    const C w = csel<R>(h, twiddle_value<N, N, INV, R>(H + j, tw), twiddle_value<N, N, INV, R>(j, tw));
    const C t = cmul(od, w);
    sink(j, cadd(ev, t));
    sink(H + j, csub(ev, t));
  }
}
template <int N, bool INV, typename R>
__device__ __forceinline__ void split_line_dft(cplx<R> (&a)[N / 2], cplx<R> (&y)[N / 2], int h,
                                               const TwTable<R, N>& tw) {
  dft<N / 2, N, INV, R>(a, tw);                            // E (lane 0) or O (lane 1)
  split_combine<N, INV, R>(a, h, tw, [&](int j, cplx<R> v) { y[j] = v; });
}
// Pass B for the large FP64 pencils (n_z >= 64), whose whole pencil per thread
// spills (FP32 pencils of 64 and 96 take the four-warp form, pass_b_quad_kernel):
// two lanes per z-pencil (lanes 2q, 2q+1 of a warp; 128 pencils per block). Lane h holds the samples z = 2m + h and transforms them with a DFT of
// N/2:
//   forward  Y[k] = E[k] + w^k O[k], Y[k + N/2] = E[k] - w^k O[k]
//            (E, O the half-length transforms of the even / odd samples,
//            w = exp(-2 pi i / N)); lane h keeps k in [hN/4, (h+1)N/4) and gets
//            the partner's half of E or w^k O by one shuffle per value;
//   inverse  x[2m] = IDFT(Y[k] + Y[k + N/2]), x[2m+1] = IDFT((Y[k] - Y[k + N/2]) w^-k)
//            over k < N/2; each lane forms its quarter of both sequences and
//            swaps the other lane's by shuffle; lane 0 transforms the first,
//            lane 1 the second.
// Lane roles are selected arithmetically (no divergent branches). At n_z = 48
// the shuffles cost more than the occupancy gains, so shorter pencils keep one
// thread per pencil.
constexpr int kBSplitPencils = 128;   // pencils per 256-thread block of the split pass B
// FP64 pencils of 64+ points need the whole register file of a thread: one
// block per SM. (For FP32 pencils of 96 this form spilled a few hundred bytes
// at two blocks per SM, still faster than one block without spills: 25.7 vs
// 31.7 ms of pass B per 96^3 build of 128 orbitals; the four-warp form takes
// 19.3 ms.)
template <typename R, int N> constexpr int kBSplitBlocks = sizeof(R) == 8 ? 1 : 2;
template <int NZ> constexpr bool kSplitPencil = NZ >= 64 && NZ % 4 == 0;

template <typename R, int NZ, bool CUBE>
__global__ void __launch_bounds__(256, kBSplitBlocks<R, NZ>)
pass_b_split_kernel(const __grid_constant__ PencilParams<R, NZ> P, int mode) {
  using C = cplx<R>;
  constexpr int N = NZ, M = N / 2, H = N / 4;
  static_assert(N % 4 == 0, "the split pass B halves a pencil twice");
  __shared__ double red[8];
  griddep_launch();
  griddep_wait();
  const PencilGeom<R, NZ, CUBE> G(P);
  const int nxy = G.nxy;
  const int tid = threadIdx.x, h = tid & 1;
  const long long gid = (long long)blockIdx.x * kBSplitPencils + (tid >> 1);
  const bool active = gid < (long long)P.npairs * nxy;    // same for both lanes of a pencil
  const int p = active ? (int)(gid / nxy) : 0;
  const int f = active ? (int)(gid % nxy) : 0;
  C* s = P.S + (long long)p * N * nxy + f;
  const C zero = cmk<C>(R(0), R(0));
  C a[M];
#pragma unroll
  for (int m = 0; m < M; ++m) a[m] = active ? s[(long long)(2 * m + h) * nxy] : zero;
  C y[M];                                                  // y[j] = Y[hH + j], y[H + j] = Y[hH + j + M]
  split_line_dft<N, false, R>(a, y, h, P.tw);
  R acc = R(0);
  const R* kt = P.Kt + G.kt_pencil(f);
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const int kz = h * H + (j < H ? j : j - H + M);
    const R k = kt[kfold<N>(kz) * G.kzs];
    if (mode != 0) acc += k * (y[j].x * y[j].x + y[j].y * y[j].y);
    y[j] = cscale(y[j], k);
  }
  double e = 0.0;
  if (mode != 0 && active) e = slot_weight(P.tiles, P.ntiles, p, P.packed) * (double)acc;
  if (mode != 1) {
#pragma unroll
    for (int j = 0; j < H; ++j) {                          // k = hH + j
      const C sum = cadd(y[j], y[H + j]);
      const C w = csel<R>(h, twiddle_value<N, N, true, R>(H + j, P.tw), twiddle_value<N, N, true, R>(j, P.tw));
      const C dif = cmul(csub(y[j], y[H + j]), w);
      const C recv = shfl_pair(h ? sum : dif);
      a[j] = h ? recv : sum;                               // lane 0: the sums, lane 1: the differences
      a[H + j] = h ? dif : recv;
    }
    dft<M, N, true, R>(a, P.tw);                           // x[2m + h] = a[m]
    if (active) {
#pragma unroll
      for (int m = 0; m < M; ++m) s[(long long)(2 * m + h) * nxy] = a[m];
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

// Planes whose passes use the two-lane line transforms (one plane per block),
// and the blocks per SM their launch bounds ask for: at 48^3 the half-length
// lines need 72-95 registers, so six 96-thread blocks (18-27 warps) fit an SM
// where the one-thread-per-line form runs 15 warps at 117-128. Below 48 the
// whole-line form is as fast (several planes per block). Pass A at 48^3 is held
// to 80 registers (eight blocks, 24 warps): 1.3 % faster steps. FP64 lines take
// the two-lane form from 64 (a whole FP64 line of 64 would not fit a thread's
// registers), with one or two blocks per SM.
constexpr int kSplitMinEdge = 48;
constexpr int kSplitMinEdgeF64 = 64;
template <typename R, int NX, int NY> constexpr bool kSplitPlanes =
    NX % 4 == 0 && NY % 4 == 0 &&
    (sizeof(R) == 4 ? kMaxLine<NX, NY> >= kSplitMinEdge : kMaxLine<NX, NY> >= kSplitMinEdgeF64);
template <typename R, int NX, int NY> constexpr int kSplitBlocks =
    sizeof(R) == 8 ? (kMaxLine<NX, NY> >= 96 ? 1 : 2)
                   : (kMaxLine<NX, NY> >= 96 ? 2 : kMaxLine<NX, NY> >= 64 ? 4 : 6);
template <typename R, int NX, int NY> constexpr int kSplitBlocksA =
    sizeof(R) == 4 && NX == 48 && NY == 48 ? 8 : kSplitBlocks<R, NX, NY>;
template <typename R, int NX, int NY> constexpr size_t kSplitSmem = (size_t)NY * (NX + 1) * sizeof(cplx<R>);

// frequency index held in y[j] by lane h
template <int N> __device__ __forceinline__ int split_index(int j, int h) {
  return h * (N / 4) + (j < N / 4 ? j : j - N / 4 + N / 2);
}

// Passes A and C with two lanes per line: one plane per block (2 max(n_x, n_y)
// threads), each pass's two line transforms by split_line_dft, the transpose
// through shared memory as in the one-thread-per-line form. Half the registers
// of a whole line per thread (which at 96^3 would need over 200), so more
// warps per SM hide the latency of the plane loads and stores. On a
// non-square plane the lanes past the shorter edge compute on zeros and store
// nothing, so every lane of a warp takes part in the shuffles.
template <typename R, int NX, int NY, bool REAL>
__global__ void __launch_bounds__(2 * kMaxLine<NX, NY>, kSplitBlocksA<R, NX, NY>)
pass_a_split_kernel(const __grid_constant__ PlaneParams<R, NX, NY> P) {
  using C = cplx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  griddep_launch();
  const int tid = threadIdx.x, q = tid >> 1, h = tid & 1;
  const long long item = blockIdx.x;                      // one (pair, z) plane per block, z-major:
  const int z = (int)(item / P.npairs), p = (int)(item % P.npairs);   // pairs sharing a plane run together
  int l, r, r2 = -1;
  if constexpr (REAL) decode_slot_real(P.tiles, P.ntiles, p, l, r, r2);
  else decode_pair(P.tiles, P.ntiles, p, l, r);
  const C zero = cmk<C>(R(0), R(0));
  {   // column x = q: samples y = 2m + h
    constexpr int M = NY / 2;
    const bool act = q < NX;
    C a[M];
    const long long xo = (long long)l * P.ld + (long long)z * NX * NY + q;
    const long long yo = (long long)r * P.ld + (long long)z * NX * NY + q;
    if constexpr (REAL) {                                  // x_l (y_r + i y_r2)
      const R* Xr = static_cast<const R*>(P.X);
      const R* Yr = static_cast<const R*>(P.Y);
      const bool two = r2 >= 0;
      const long long y2o = (long long)(two ? r2 : r) * P.ld + (long long)z * NX * NY + q;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int yy = 2 * m + h;
        const R xv = act ? Xr[xo + yy * NX] : R(0);
        a[m] = act ? cmk<C>(xv * Yr[yo + yy * NX], two ? xv * Yr[y2o + yy * NX] : R(0)) : zero;
      }
    } else {
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int yy = 2 * m + h;
        a[m] = act ? cmulc(load_vec<R, REAL>(P.X, xo + yy * NX), load_vec<R, REAL>(P.Y, yo + yy * NX)) : zero;
      }
    }
    dft<M, NY, false, R>(a, P.tw.ty());                   // along y
    split_combine<NY, false, R>(a, h, P.tw.ty(), [&](int j, C v) {
      if (act) buf[split_index<NY>(j, h) * (NX + 1) + q] = v;
    });
  }
  __syncthreads();
  {   // row ky = q: samples x = 2m + h
    constexpr int M = NX / 2;
    const bool act = q < NY;
    C a[M];
#pragma unroll
    for (int m = 0; m < M; ++m) a[m] = act ? buf[q * (NX + 1) + 2 * m + h] : zero;
    dft<M, NX, false, R>(a, P.tw.tx());                   // along x
    griddep_wait();                                        // the previous batch's pass D still reads S
    C* out = P.S + ((long long)p * P.nz + z) * NX * NY + q;
    split_combine<NX, false, R>(a, h, P.tw.tx(), [&](int j, C v) {
      if (act) out[(long long)split_index<NX>(j, h) * NY] = v;
    });
  }
}

template <typename R, int NX, int NY>
__global__ void __launch_bounds__(2 * kMaxLine<NX, NY>, kSplitBlocks<R, NX, NY>)
pass_c_split_kernel(const __grid_constant__ PlaneParams<R, NX, NY> P) {
  using C = cplx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  griddep_launch();
  griddep_wait();
  const int tid = threadIdx.x, q = tid >> 1, h = tid & 1;
  const long long item = blockIdx.x;
  const int p = (int)(item / P.nz), z = (int)(item % P.nz);
  C* plane = P.S + ((long long)p * P.nz + z) * NX * NY;
  const C zero = cmk<C>(R(0), R(0));
  {   // row ky = q of the spectrum: samples kx = 2m + h, inverse along x
    constexpr int M = NX / 2;
    const bool act = q < NY;
    C a[M];
#pragma unroll
    for (int m = 0; m < M; ++m) a[m] = act ? plane[(long long)(2 * m + h) * NY + q] : zero;
    dft<M, NX, true, R>(a, P.tw.tx());
    split_combine<NX, true, R>(a, h, P.tw.tx(), [&](int j, C v) {
      if (act) buf[q * (NX + 1) + split_index<NX>(j, h)] = v;   // row ky, column x
    });
  }
  __syncthreads();
  {   // column x = q: samples ky = 2m + h, inverse along y
    constexpr int M = NY / 2;
    const bool act = q < NX;
    C a[M];
#pragma unroll
    for (int m = 0; m < M; ++m) a[m] = act ? buf[(2 * m + h) * (NX + 1) + q] : zero;
    dft<M, NY, true, R>(a, P.tw.ty());
    split_combine<NY, true, R>(a, h, P.tw.ty(), [&](int j, C v) {
      if (act) plane[(long long)split_index<NY>(j, h) * NX + q] = v;
    });
  }
}

// ---- four warps per 32 lines (pass B for FP32 pencils of 96)
// A length-N line transform (N = 4M, decimation in time by 4) is spread over
// four warps: the thread with phase h (warp-uniform) transforms the samples
// 4m + h (a DFT of M in registers) and multiplies by w_N^{hk}; after a block
// barrier the thread with phase h forms, for its M/4 frequencies k = hM/4 + j,
// the radix-4 combination Y[k + qM] = sum_h' (w_4)^{h'q} U_h'[k] (q = 0..3) of
// the four phases' values, read from shared memory. A thread holds a quarter of
// a line (M values) and needs no shuffles or lane-dependent selects (the phase
// is warp-uniform, so its twiddles are compile-time constants in one of four
// code paths). For the plane passes the same scheme measured slower than the
// two-lane form (six shared-memory accesses per point per pass: bound by the
// shared-memory pipe), so only pass B uses it.
template <int N, bool INV, typename R>
__device__ __forceinline__ void quad_sub_dft(cplx<R> (&a)[N / 4], int h, const TwTable<R, N>& tw) {
  constexpr int M = N / 4;
  dft<M, N, INV, R>(a, tw);
  if (h == 1) {
#pragma unroll
    for (int k = 1; k < M; ++k) a[k] = twiddle<N, N, INV, R>(a[k], k, tw);
  } else if (h == 2) {
#pragma unroll
    for (int k = 1; k < M; ++k) a[k] = twiddle<N, N, INV, R>(a[k], 2 * k, tw);
  } else if (h == 3) {
#pragma unroll
    for (int k = 1; k < M; ++k) a[k] = twiddle<N, N, INV, R>(a[k], 3 * k, tw);
  }
}

// The radix-4 step for one line whose value U_h'[k] sits at
// buf[base + (h'M + k) stride]: for j < M/4 and k = hM/4 + j,
// out[4j + q] = Y[k + qM].
template <int N, bool INV, typename R>
__device__ __forceinline__ void quad_combine(const cplx<R>* __restrict__ buf, int base, int stride, int h,
                                             cplx<R> (&out)[N / 4], const TwTable<R, N>& tw) {
  constexpr int M = N / 4, Q = M / 4;
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    cplx<R> u[4];
#pragma unroll
    for (int hh = 0; hh < 4; ++hh) u[hh] = buf[base + (hh * M + h * Q + j) * stride];
    dft<4, N, INV, R>(u, tw);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[4 * j + q] = u[q];
  }
}

// Pass B with four warps per 32 pencils (FP32 pencils of 64 and 96): warp h holds the
// samples z = 4m + h of its lane's pencil, transforms them (quad_sub_dft) and
// stores them to shared memory; after a barrier each thread forms the radix-4
// combination for its M/4 frequencies k = hM/4 + j, which gives it the 24
// spectrum values kz = k + qM (q = 0..3), multiplies them by K(G) (and sums
// the energy), and takes the inverse radix-4 step right away: for each of its k,
// Z_h'[k] = sum_q Y[k + qM] (w_4)^{-h'q} w_N^{-h'k}, h' = 0..3, written back to
// the same shared-memory places it read. After a second barrier warp h reads
// Z_h[k] for all k and an inverse DFT of M gives x[4m + h]. The 96-point pencil
// thus needs a quarter of it in registers per thread (no spills, where the
// two-lane form spills at two blocks per SM) and no shuffles.
constexpr int kQuadPencils = 32;   // pencils per 128-thread block of the four-warp pass B
// (At n_z = 48 the whole pencil per thread measured faster: 2.63 vs 2.84 ps per
// pair-point.)
template <typename R, int NZ> constexpr bool kQuadPencil = sizeof(R) == 4 && (NZ == 96 || NZ == 64);

// u[4j + h'] *= w_N^{-h'(HQ + j)} (inverse twiddles of warp phase H)
template <int N, int H, typename R>
__device__ __forceinline__ void quad_inv_twiddle(cplx<R> (&u)[N / 4], const TwTable<R, N>& tw) {
  constexpr int Q = N / 16;
#pragma unroll
  for (int j = 0; j < Q; ++j)
#pragma unroll
    for (int hp = 1; hp < 4; ++hp) u[4 * j + hp] = twiddle<N, N, true, R>(u[4 * j + hp], hp * (H * Q + j), tw);
}

template <typename R, int NZ, bool CUBE>
__global__ void __launch_bounds__(128, 5)
pass_b_quad_kernel(const __grid_constant__ PencilParams<R, NZ> P, int mode) {
  using C = cplx<R>;
  constexpr int N = NZ, M = N / 4, Q = M / 4, LP = kQuadPencils;
  static_assert(M % 4 == 0, "M / 4 frequencies per thread");
  __shared__ C buf[N * LP];                                // [phase h, k][pencil]
  __shared__ double red[4];
  griddep_launch();
  griddep_wait();
  const PencilGeom<R, NZ, CUBE> G(P);
  const int nxy = G.nxy;
  const int h = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long gid = (long long)blockIdx.x * LP + lane;
  const bool active = gid < (long long)P.npairs * nxy;
  const int p = active ? (int)(gid / nxy) : 0;
  const int f = active ? (int)(gid % nxy) : 0;
  C* s = P.S + (long long)p * N * nxy + f;
  const C zero = cmk<C>(R(0), R(0));
  C a[M];
#pragma unroll
  for (int m = 0; m < M; ++m) a[m] = active ? s[(long long)(4 * m + h) * nxy] : zero;
  quad_sub_dft<N, false, R>(a, h, P.tw);
#pragma unroll
  for (int k = 0; k < M; ++k) buf[(h * M + k) * LP + lane] = a[k];
  __syncthreads();
  quad_combine<N, false, R>(buf, lane, LP, h, a, P.tw);    // a[4j + q] = Y[hQ + j + qM]
  R acc = R(0);
  const R* kt = P.Kt + G.kt_pencil(f);
#pragma unroll
  for (int j = 0; j < Q; ++j) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int kz = h * Q + j + q * M;
      const R kv = kt[kfold<N>(kz) * G.kzs];
      C& v = a[4 * j + q];
      if (mode != 0) acc += kv * (v.x * v.x + v.y * v.y);
      v = cscale(v, kv);
    }
  }
  if (mode != 1) {
#pragma unroll
    for (int j = 0; j < Q; ++j) {                          // inverse radix-4 over q: outputs by phase h'
      C u[4] = {a[4 * j], a[4 * j + 1], a[4 * j + 2], a[4 * j + 3]};
      dft<4, N, true, R>(u, P.tw);
#pragma unroll
      for (int hp = 0; hp < 4; ++hp) a[4 * j + hp] = u[hp];
    }
    if (h == 0) quad_inv_twiddle<N, 0, R>(a, P.tw);
    else if (h == 1) quad_inv_twiddle<N, 1, R>(a, P.tw);
    else if (h == 2) quad_inv_twiddle<N, 2, R>(a, P.tw);
    else quad_inv_twiddle<N, 3, R>(a, P.tw);
#pragma unroll
    for (int j = 0; j < Q; ++j)                            // the places quad_combine read
#pragma unroll
      for (int hp = 0; hp < 4; ++hp) buf[(hp * M + h * Q + j) * LP + lane] = a[4 * j + hp];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < M; ++k) a[k] = buf[(h * M + k) * LP + lane];   // Z_h[k], k < M
    dft<M, N, true, R>(a, P.tw);                           // x[4m + h] = a[m]
    if (active) {
#pragma unroll
      for (int m = 0; m < M; ++m) s[(long long)(4 * m + h) * nxy] = a[m];
    }
  }
  if (mode != 0) {
    double e = active ? slot_weight(P.tiles, P.ntiles, p, P.packed) * (double)acc : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if (lane == 0) red[h] = e;
    __syncthreads();
    if (threadIdx.x == 0) P.Epart[blockIdx.x] += red[0] + red[1] + red[2] + red[3];   // one block per slot
  }
}

// FP64 pencils of 48 hold 96 doubles: one block per SM (two would cap a thread
// at 128 registers and spill about 3 KB).
template <typename R, int NZ, bool CUBE>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 1 : 2)
pass_b_kernel(const __grid_constant__ PencilParams<R, NZ> P, int mode) {
  __shared__ double red[32];
  griddep_launch();
  griddep_wait();
  body_b<R, NZ, false, CUBE>(P, P.tiles, P.ntiles, P.npairs, mode, blockIdx.x, threadIdx.x, blockDim.x, red,
                             mode != 0 ? P.Epart + blockIdx.x : nullptr);
}

template <typename R, int NX, int NY>
__global__ void __launch_bounds__(kMaxLine<NX, NY> * plane_items<R, NX, NY>(), 2)
pass_c_kernel(const __grid_constant__ PlaneParams<R, NX, NY> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  griddep_launch();
  griddep_wait();
  body_c<R, NX, NY, false, plane_items<R, NX, NY>()>(P, P.npairs, reinterpret_cast<cplx<R>*>(smem_raw), blockIdx.x,
                                                     threadIdx.x);
}

// Full off-diagonal tiles take two threads per grid point (d_split_off) at
// four blocks per SM (64 registers): more warps and loads in flight per SM,
// which measured faster than one thread per point at 2 or 3 blocks per SM
// (and than streaming the potentials through shared memory with bulk copies).
// The tiles other than full off-diagonal ones (diagonal, ragged, one-sided):
// one thread per point, 256 points per block (the grid is sized for 128-point
// blocks, so the upper half of the blocks has no work). Not inlined, so that
// its larger register state does not spill into the full-tile path.
template <typename R, bool REAL, long long NGC>
__device__ __noinline__ void pass_d_other(const PointParams<R>& P, const TileDesc& d) {
  if ((long long)blockIdx.x * 256 >= (NGC ? NGC : P.ng)) return;
  body_d<R, REAL, false, false, NGC>(P, d, blockIdx.x, threadIdx.x, blockDim.x);
}

template <typename R, bool REAL, long long NGC>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2)
pass_d_kernel(const __grid_constant__ PointParams<R> P) {
  __shared__ cplx<R> xch[(kTileMax / 2) * 256];
  griddep_launch();
  griddep_wait();
  const TileDesc d = P.tiles[blockIdx.y];
  if (d.kind == 0 && d.nl == kTileMax && d.nr == kTileMax) {
    if constexpr (REAL) d_split_off_real<R, NGC>(P, d, blockIdx.x, threadIdx.x, reinterpret_cast<R*>(xch));
    else d_split_off<R, REAL, NGC>(P, d, blockIdx.x, threadIdx.x, xch);
    return;
  }
  pass_d_other<R, REAL, NGC>(P, d);
}

// ---------------------------------------------------------------- persistent engine
template <typename R, int N> struct EngineParams {
  PlaneParams<R, N, N> pl;      // npairs / ntiles unused: per batch from the table
  PencilParams<R, N> pe;
  PointParams<R> pt;
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
    const TileDesc* tiles = E.pl.tiles + b.toff;
    if (pass == 0) {
      body_a<R, N, N, REAL, true, IPB, false>(E.pl, tiles, b.ntiles, b.npairs, smem, loc, tid);
    } else if (pass == 1) {
      body_b<R, N, true, true>(E.pe, tiles, b.ntiles, b.npairs, E.mode, loc, tid, kEngineThreads, red,
                               E.mode != 0 ? E.pe.Epart + loc : nullptr);
    } else if (pass == 2) {
      body_c<R, N, N, true, IPB>(E.pl, b.npairs, smem, loc, tid);
    } else {
      const long long nvb = ((long long)N * N * N + kEngineThreads - 1) / kEngineThreads;
      const TileDesc d = tiles[loc / nvb];
      body_d<R, REAL, true, true, (long long)N * N * N>(E.pt, d, loc % nvb, tid, kEngineThreads);
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(E.done + kCtrStride * (4 * k + pass), 1u);
    }
  }
}

// ---------------------------------------------------------------- host side
template <typename R, int NX, int NY>
void fill_plane(PlaneParams<R, NX, NY>& P, const PairLaunch& L, const Batch& b) {
  P.X = L.X;
  P.Y = L.Y;
  P.S = static_cast<cplx<R>*>(L.S);
  P.ld = L.ld;
  P.nz = L.nz;
  P.npairs = b.npairs;
  P.tiles = L.dtiles;
  P.ntiles = b.ntiles;
  P.tw.fill(L.twx, L.twy);
}

template <typename R, int NZ>
void fill_pencil(PencilParams<R, NZ>& P, const PairLaunch& L, const Batch& b) {
  P.S = static_cast<cplx<R>*>(L.S);
  P.Kt = static_cast<const R*>(L.Kt);
  P.Epart = L.Epart;
  P.npairs = b.npairs;
  P.nx = L.nx;
  P.ny = L.ny;
  P.nxy = L.nx * L.ny;
  P.khy = L.ny / 2 + 1;
  P.kzs = (L.nx / 2 + 1) * (L.ny / 2 + 1);
  P.tiles = L.dtiles;
  P.ntiles = b.ntiles;
  P.packed = L.real_io ? 1 : 0;
  for (int k = 0; k < NZ; ++k) {
    P.tw.w[k].x = (R)L.twz[2 * k];
    P.tw.w[k].y = (R)L.twz[2 * k + 1];
  }
}

template <typename R>
void fill_point(PointParams<R>& P, const PairLaunch& L) {
  P.X = L.X;
  P.Y = L.Y;
  P.OutX = L.OutX;
  P.OutY = L.OutY;
  P.S = static_cast<const cplx<R>*>(L.S);
  P.ld = L.ld;
  P.ng = (long long)L.nx * L.ny * L.nz;
  P.scale = (R)L.scale;
  P.tiles = L.dtiles;
}

// Pass A (pass == 0) or C (pass == 2) of one batch, or (prepare_only) the
// kernels' shared-memory attributes, set once at plan creation on the plan's
// device, never during stream capture.
template <typename R, int NX, int NY>
bool launch_plane(const PairLaunch& L, const Batch& b, int pass, cudaStream_t st) {
  constexpr int IPB = plane_items<R, NX, NY>();
  constexpr int ML = kMaxLine<NX, NY>;
  constexpr size_t smem = (size_t)IPB * NY * (NX + 1) * sizeof(cplx<R>);
  if constexpr (sizeof(R) != 8) {
    if (L.real_io) return false;
  }
  if (L.prepare_only) {
    if constexpr (!kSplitPlanes<R, NX, NY>) {   // whole lines per thread
      if constexpr (sizeof(R) == 8) {
        cudaFuncSetAttribute(pass_a_kernel<R, NX, NY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(pass_a_kernel<R, NX, NY, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      }
      cudaFuncSetAttribute(pass_a_kernel<R, NX, NY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(pass_c_kernel<R, NX, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(pass_a_kernel<R, NX, NY, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      cudaFuncSetAttribute(pass_c_kernel<R, NX, NY>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    } else {
      constexpr int s1 = (int)kSplitSmem<R, NX, NY>;
      if constexpr (sizeof(R) == 8) {
        cudaFuncSetAttribute(pass_a_split_kernel<R, NX, NY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1);
        cudaFuncSetAttribute(pass_a_split_kernel<R, NX, NY, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      }
      cudaFuncSetAttribute(pass_a_split_kernel<R, NX, NY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1);
      cudaFuncSetAttribute(pass_c_split_kernel<R, NX, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1);
      cudaFuncSetAttribute(pass_a_split_kernel<R, NX, NY, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      cudaFuncSetAttribute(pass_c_split_kernel<R, NX, NY>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    return true;
  }
  PlaneParams<R, NX, NY> P;
  fill_plane<R, NX, NY>(P, L, b);
  const long long items = (long long)b.npairs * L.nz;
  const bool pdl = !L.no_pdl;
  if constexpr (kSplitPlanes<R, NX, NY>) {
    const dim3 grid((unsigned)items), blk(2 * ML);
    if (pass == 0) {
      if (sizeof(R) == 8 && L.real_io)
        launch_pdl(pdl, pass_a_split_kernel<R, NX, NY, sizeof(R) == 8>, grid, blk, kSplitSmem<R, NX, NY>, st, P);
      else
        launch_pdl(pdl, pass_a_split_kernel<R, NX, NY, false>, grid, blk, kSplitSmem<R, NX, NY>, st, P);
    } else {
      launch_pdl(pdl, pass_c_split_kernel<R, NX, NY>, grid, blk, kSplitSmem<R, NX, NY>, st, P);
    }
  } else {
    const dim3 grid((unsigned)((items + IPB - 1) / IPB)), blk(ML * IPB);
    if (pass == 0) {
      if (sizeof(R) == 8 && L.real_io)
        launch_pdl(pdl, pass_a_kernel<R, NX, NY, sizeof(R) == 8>, grid, blk, smem, st, P);
      else
        launch_pdl(pdl, pass_a_kernel<R, NX, NY, false>, grid, blk, smem, st, P);
    } else {
      launch_pdl(pdl, pass_c_kernel<R, NX, NY>, grid, blk, smem, st, P);
    }
  }
  return true;
}

// Pass B of one batch (the compile-time geometry on cubic grids).
template <typename R, int NZ, bool CUBE>
void launch_pencil_as(const PencilParams<R, NZ>& P, const PairLaunch& L, long long pencils, cudaStream_t st) {
  if constexpr (kQuadPencil<R, NZ>) {
    const unsigned grid = (unsigned)((pencils + kQuadPencils - 1) / kQuadPencils);
    launch_pdl(!L.no_pdl, pass_b_quad_kernel<R, NZ, CUBE>, dim3(grid), dim3(128), 0, st, P, L.mode);
  } else if constexpr (kSplitPencil<NZ>) {
    const unsigned grid = (unsigned)((pencils + kBSplitPencils - 1) / kBSplitPencils);
    launch_pdl(!L.no_pdl, pass_b_split_kernel<R, NZ, CUBE>, dim3(grid), dim3(256), 0, st, P, L.mode);
  } else {
    const unsigned grid = (unsigned)((pencils + 255) / 256);
    launch_pdl(!L.no_pdl, pass_b_kernel<R, NZ, CUBE>, dim3(grid), dim3(256), 0, st, P, L.mode);
  }
}
template <typename R, int NZ>
bool launch_pencil(const PairLaunch& L, const Batch& b, cudaStream_t st) {
  if (L.prepare_only) return true;
  PencilParams<R, NZ> P;
  fill_pencil<R, NZ>(P, L, b);
  const long long pencils = (long long)b.npairs * L.nx * L.ny;
  if (L.nx == NZ && L.ny == NZ) launch_pencil_as<R, NZ, true>(P, L, pencils, st);
  else launch_pencil_as<R, NZ, false>(P, L, pencils, st);
  return true;
}

// Pass D of one batch: NGC = N_g of a cubic grid compiled in, or 0 (any grid).
template <typename R, long long NGC>
bool launch_point(const PairLaunch& L, const Batch& b, cudaStream_t st) {
  if (L.prepare_only) return true;
  PointParams<R> P;
  fill_point<R>(P, L);
  if (NGC && P.ng != NGC) return false;
  const dim3 grid((unsigned)((P.ng + kDSplitPts - 1) / kDSplitPts), (unsigned)b.ntiles);
  if constexpr (sizeof(R) == 8) {
    if (L.real_io) {
      launch_pdl(!L.no_pdl, pass_d_kernel<R, true, NGC>, grid, dim3(256), 0, st, P);
      return true;
    }
  } else {
    if (L.real_io) return false;
  }
  launch_pdl(!L.no_pdl, pass_d_kernel<R, false, NGC>, grid, dim3(256), 0, st, P);
  return true;
}

// The persistent engine holds whole lines per thread; FP64 lines of 64 or more
// points do not fit, so those edges have no engine (plans fall back to the four
// kernels per batch).
template <typename R, int N> constexpr bool kEngineBuilt = !(sizeof(R) == 8 && N >= kSplitMinEdgeF64);

// Tasks per pass of a batch in the engine (A, B, C, D).
template <typename R, int N>
void engine_tasks(const Batch& b, int n[4]) {
  constexpr int IPB = engine_items<R, N>();
  n[0] = (int)(((long long)b.npairs * N + IPB - 1) / IPB);
  n[1] = (int)(((long long)b.npairs * N * N + kEngineThreads - 1) / kEngineThreads);
  n[2] = n[0];
  n[3] = (int)((((long long)N * N * N + kEngineThreads - 1) / kEngineThreads) * b.ntiles);
}

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
    if (L.nx != N || L.ny != N || L.nz != N) return false;
    EngineParams<R, N> E;
    Batch none{};
    fill_plane<R, N, N>(E.pl, L, none);
    fill_pencil<R, N>(E.pe, L, none);
    fill_point<R>(E.pt, L);
    E.pl.tiles = EL.dtiles;
    E.pe.tiles = EL.dtiles;
    E.pt.tiles = EL.dtiles;
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

}  // namespace ACE_RADIX_NS
}  // namespace ace
