// Xi = W L^{-*} (Eq. Wtilde) to FP64 accuracy on the FP16 tensor cores, for
// FP32 vectors W: an error-free splitting of both operands into small-integer
// slices (the Ozaki scheme), exact integer products on tcgen05 (kind::f16),
// exact accumulation, and a single scaling to FP64 at the end.
//
// As in the tensor-core GEMMs of tc_gemm.cu the complex product is a real GEMM
// on interleaved data: rows are grid points g, K' = 2 nk real terms (Re, Im of
// W_k(g)), and a tile of BB complex output columns b is TN = 2 BB real columns
// (j < BB: (Re C_kb, -Im C_kb) -> Re Xi_b; BB + j: (Im C_kb, Re C_kb) -> Im Xi_b).
//
// Splitting (beta = 8 bits per slice):
//   row g of A is scaled by 2^-e_g, e_g the smallest exponent with |A_gk| < 2^e_g
//   for every k; column b of C by 2^-f_b likewise. The scaled value x in (-1, 1)
//   is peeled into signed digits d_1 = rint(2^8 x), d_s = rint(2^8 r_{s-1})
//   with r the remainders (|d_1| <= 256, |d_s| <= 128), so that
//   x = sum_s d_s 2^{-8 s} + O(2^{-8 S}); every step is exact in FP32 (A) or
//   FP64 (C) arithmetic, and every digit is an integer that FP16 holds exactly.
// Products:
//   Xi_gb = 2^{e_g + f_b} sum_{s,t} 2^{-8 (s+t)} P_st,  P_st = sum_k a^(s)_gk c^(t)_kb,
//   keeping the slice pairs with s + t <= T = 6 and 5 slices per operand. The
//   error before the final rounding is then below about 2^-41 max_k |A_gk|
//   sum_k |C_kb| (the truncated slices and the dropped pairs): FP64 accuracy
//   relative to the size of the terms of the sum, which an ill-conditioned
//   L (large entries of L^{-*}) makes much larger than Xi itself; with
//   T = 5 (2^-33) such cases lost FP32 accuracy. The products of one weight
//   w = s + t share a tensor-memory accumulator. Over a group of 128 real K
//   terms every partial sum is an integer below 2^24 in magnitude (at most 1.5
//   2^16 per term and weight), so the FP32 accumulation is exact whatever its
//   rounding; after each group the accumulators are read back (tcgen05.ld),
//   converted to int32 exactly and added into per-thread int64 sums shifted by
//   8 (T - w) bits (below 2^60: no overflow). The final value is
//   sum 2^(e_g + f_b - 8 T): the integer sum is rounded once to the output type
//   and scaled by the power of two (exact), in FP32 for FP32 outputs (no FP64
//   arithmetic, which is slow on this part).
//
// Per CTA (512 threads, one per SM): T - 1 accumulators of TN columns in TMEM;
// K runs in chunks of 32 real terms (16 orbitals) through three shared-memory
// stages, each holding T - 1 A slices (split on the fly from the FP32 loads) and
// the chunk's B slices (split once per call by oz_slice_b_kernel into the
// stage layout, brought in by one bulk copy per chunk on the TMA unit, which
// completes on the stage's second mbarrier). One thread issues the bulk copy
// and, once it has landed, the MMAs of the chunk (2 K-steps per slice pair),
// and commits them to the stage's first mbarrier;
// the threads drain the accumulators after the last chunk of each group.
// L^{-*} is upper triangular, so tile [b0, b0 + BB) runs k < b0 + BB only.
// Every mbarrier wait is bounded: on timeout the CTA records ACE_ERR_TIMEOUT,
// stops issuing, waits (bounded) for what it issued and frees its TMEM.
#include <cstdint>
#include <cuda_fp16.h>

#include "ace_internal.h"
#include "tcgen05.cuh"

namespace ace {

namespace {

constexpr int OZ_THREADS = 512;
constexpr int OZ_TM = 128;                     // rows per CTA (M of the MMA)
constexpr int OZ_KC = 32;                      // real K terms per chunk
constexpr int OZ_SBO = (OZ_KC / 8) * 128;      // bytes between 8-row groups of 16-bit elements = 512
constexpr int OZ_BETA = 8;                     // bits per slice
constexpr int OZ_GROUP = 4;                    // chunks per exact accumulation group (128 real K)
constexpr int OZ_NSTAGE = 3;
constexpr unsigned kOzWaitLimit = 1u << 24;

template <int T> struct Oz {
  static_assert(T == 5 || T == 6, "slice depth");
  static constexpr int SA = T - 1;             // A slices: 8 (T - 1) bits below the row maximum
  static constexpr int SB = T - 1;             // C slices
  static constexpr int NW = T - 1;             // accumulators, weights w = 2 .. T
  static constexpr int TN = T == 5 ? 128 : 96; // NW x TN <= 512 TMEM columns
  static constexpr int BB = TN / 2;
  static constexpr int NACC = TN / 4;          // columns per thread (4 column groups of warps)
  static constexpr int A_SLICE = OZ_TM * OZ_KC * 2;
  static constexpr int B_SLICE = TN * OZ_KC * 2;
  static constexpr int STAGE = SA * A_SLICE + SB * B_SLICE;
  static constexpr int SMEM = OZ_NSTAGE * STAGE + 1024 + 128;   // stages, alignment, 6 barriers + TMEM slot
  // instruction descriptor: D = F32, A = B = F16, both K-major, N = TN, M = 128
  static constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(OZ_TM >> 4) << 24);
};

// byte offset of (row r, real k) in a 16-bit operand tile of one chunk
__device__ __forceinline__ int oz_off(int r, int k) {
  return (r >> 3) * OZ_SBO + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ unsigned short f16_bits(float d) { return __half_as_ushort(__float2half_rn(d)); }

// rint(x) for |x| < 2^22 by two full-rate additions: adding 1.5 * 2^23 rounds x
// to an integer (round to nearest, ties to even, as rint) in the low mantissa
// bits, and subtracting it again is exact.
__device__ __forceinline__ float round_int(float x) {
  return __fadd_rn(__fadd_rn(x, 12582912.0f), -12582912.0f);
}

template <int T>
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(Oz<T>::IDESC), "r"(accumulate)
      : "memory");
}

// smallest e with |x| < 2^e (0 for x == 0)
__device__ __forceinline__ int exp_above(double m) {
  int e = 0;
  if (m > 0.0) frexp(m, &e);
  return e;
}

// e_g for every grid point: the row maximum of |Re W_k(g)|, |Im W_k(g)| over k.
__global__ void oz_row_exp_kernel(const float2* __restrict__ A, int nk, long long ld, long long ng,
                                  int* __restrict__ erow) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (long long)gridDim.x * blockDim.x) {
    float m = 0.f;
    for (int k = 0; k < nk; ++k) {
      const float2 v = A[(long long)k * ld + g];
      m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    erow[g] = exp_above((double)m);
  }
}

// One block per complex column b of C (FP64 [nk][nb], upper triangular): f_b,
// then the SB digits of the column's real entries, written into the stage
// layout of chunk c = k / 16, tile bt = b / BB: Bsl[((bt * nch + c) * SB + t)]
// holds a TN x 32 16-bit operand tile. Bsl must be zero beforehand (padding).
template <int T>
__global__ void __launch_bounds__(256)
oz_slice_b_kernel(const double* __restrict__ C, int nk, int nb, int nch, unsigned short* __restrict__ Bsl,
                  int* __restrict__ fcol) {
  using O = Oz<T>;
  __shared__ double red[256];
  const int b = blockIdx.x;
  const int kend = b + 1 < nk ? b + 1 : nk;          // C[k][b] = 0 for k > b
  double m = 0.0;
  for (int k = threadIdx.x; k < kend; k += blockDim.x) {
    const long long o = 2 * ((long long)k * nb + b);
    m = fmax(m, fmax(fabs(C[o]), fabs(C[o + 1])));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const int f = exp_above(red[0]);
  if (threadIdx.x == 0) fcol[b] = f;
  const int bt = b / O::BB, j = b % O::BB;
  for (int k = threadIdx.x; k < kend; k += blockDim.x) {
    const long long o = 2 * ((long long)k * nb + b);
    const double re = C[o], im = C[o + 1];
    const int c = k / 16, kk = 2 * (k % 16);          // real rows kk (Re A) and kk + 1 (Im A)
    unsigned short* tile = Bsl + (size_t)(bt * nch + c) * O::SB * (O::TN * OZ_KC);
    // (row j: Re C, -Im C), (row BB + j: Im C, Re C)
    const double v[4] = {re, -im, im, re};
    const int rr[4] = {j, j, O::BB + j, O::BB + j}, kr[4] = {kk, kk + 1, kk, kk + 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double x = ldexp(v[q], OZ_BETA - f);
#pragma unroll
      for (int t = 0; t < O::SB; ++t) {
        const double d = rint(x);
        x = (x - d) * (double)(1 << OZ_BETA);
        tile[(size_t)t * (O::TN * OZ_KC) + oz_off(rr[q], kr[q]) / 2] = f16_bits((float)d);
      }
    }
  }
}

// Grid: one CTA per SM (or fewer), each taking the (column tile, 128-row
// block) tiles blockIdx.x, blockIdx.x + gridDim.x, ... A: complex FP32 [nk][ld];
// Out: complex FP32 or FP64 [nb][ld].
template <int T, typename OUT>
__global__ void __launch_bounds__(OZ_THREADS, 1)
oz_outer_kernel(const float2* __restrict__ A, int nk, int nb, long long ld, long long ng,
                const int* __restrict__ erow, const unsigned short* __restrict__ Bsl, const int* __restrict__ fcol,
                int nch, OUT* __restrict__ Out, int* status) {
  using O = Oz<T>;
  constexpr int NACC = O::NACC;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + OZ_NSTAGE * O::STAGE);        // MMAs of the stage done
  uint64_t* full = bar + OZ_NSTAGE;                                                    // B slices of the stage landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + OZ_NSTAGE * O::STAGE + 64);
  __shared__ int s_fail;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < OZ_NSTAGE; ++i) {
      tc::mbar_init(&bar[i], 1);
      tc::mbar_init(&full[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (tid < 32) tc::tmem_alloc_warp(tmem_slot, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  // tiles (column tile bt, 128-row block) in bt-fastest order, strided over the
  // resident CTAs (persistent: setup, TMEM allocation and barriers once per CTA)
  const int nbt = (nb + O::BB - 1) / O::BB;
  const int ntiles = nbt * (int)((ng + OZ_TM - 1) / OZ_TM);   // < 2^31 for every supported grid
  int bt = 0, b0 = 0, kend = 0, nchunks = 0;
  int g0 = 0, g = 0;
  float sa = 1.f;
  // this thread's A elements: row r = 8 w + lane % 8, real K 4q .. 4q + 3 with q = lane / 8 and
  // q + 4, so that a warp's 8-byte slice stores cover 256 contiguous bytes (no bank conflicts)
  const int r = 8 * w + (lane & 7), q = lane >> 3;
  const uint32_t lane_col = ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(NACC * (w >> 2));
  long long acc[NACC];

  auto load_a = [&](int c, float4 (&v)[2]) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int k = c * 16 + 2 * (q + 4 * i);
      float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
      if (g < ng) {
        if (k < kend) { const float2 x = A[(long long)k * ld + g]; t.x = x.x; t.y = x.y; }
        if (k + 1 < kend) { const float2 x = A[(long long)(k + 1) * ld + g]; t.z = x.x; t.w = x.y; }
      }
      v[i] = t;
    }
  };
  // the SA slices of this thread's 8 values into stage `st`
  auto store_a = [&](unsigned char* st, const float4 (&v)[2]) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      float x[4] = {v[i].x * sa, v[i].y * sa, v[i].z * sa, v[i].w * sa};
      const int off = oz_off(r, 4 * (q + 4 * i));
#pragma unroll
      for (int s = 0; s < O::SA; ++s) {
        float d[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          d[e] = round_int(x[e]);
          x[e] = (x[e] - d[e]) * (float)(1 << OZ_BETA);
        }
        const __half2 h01 = __floats2half2_rn(d[0], d[1]), h23 = __floats2half2_rn(d[2], d[3]);   // exact
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t*>(&h01);
        u.y = *reinterpret_cast<const uint32_t*>(&h23);
        *reinterpret_cast<uint2*>(st + s * O::A_SLICE + off) = u;
      }
    }
  };
  constexpr unsigned B_BYTES = O::SB * O::B_SLICE;
  static_assert(B_BYTES % 16 == 0 && (O::SA * O::A_SLICE) % 16 == 0, "bulk copy alignment");
  auto copy_b = [&](unsigned char* st, int c, int s) {   // thread 0
    tc::mbar_arrive_expect_tx(&full[s], B_BYTES);
    tc::bulk_g2s(st + O::SA * O::A_SLICE, Bsl + (size_t)(bt * nch + c) * O::SB * (O::TN * OZ_KC), B_BYTES, &full[s]);
  };
  auto issue = [&](const unsigned char* st, bool group_first) {
    const uint32_t a0 = tc::smem_u32(st), bb0 = a0 + O::SA * O::A_SLICE;
    bool first[O::NW];
#pragma unroll
    for (int i = 0; i < O::NW; ++i) first[i] = group_first;
#pragma unroll
    for (int wt = 2; wt <= T; ++wt) {
#pragma unroll
      for (int s = 1; s <= O::SA; ++s) {
        const int t = wt - s;
        if (t < 1 || t > O::SB) continue;
#pragma unroll
        for (int ks = 0; ks < OZ_KC / 16; ++ks) {
          const uint32_t o = ks * 256;    // two core matrices of 16 B along K per K-step of 16
          mma_f16<T>(tmem + (uint32_t)((wt - 2) * O::TN), tc::kmajor_desc(a0 + (s - 1) * O::A_SLICE + o, OZ_SBO),
                     tc::kmajor_desc(bb0 + (t - 1) * O::B_SLICE + o, OZ_SBO), first[wt - 2] ? 0u : 1u);
          first[wt - 2] = false;
        }
      }
    }
  };
  auto drain = [&]() {
    tc::fence_after_sync();
#pragma unroll
    for (int wt = 2; wt <= T; ++wt) {
      const uint32_t ta = tmem + lane_col + (uint32_t)((wt - 2) * O::TN);
      const int sh = OZ_BETA * (T - wt);
      uint32_t v[32];
      if constexpr (NACC == 32) {
        tc::tmem_ld32(ta, v);
      } else {
        tc::tmem_ld16(ta, v);
        tc::tmem_ld8(ta + 16, v + 16);
      }
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < NACC; ++j) acc[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << sh;
    }
    tc::fence_before_sync();
  };

  // Thread 0 alone waits on the barriers: the MMA commits (bit s of `issued`:
  // a commit on stage s not yet seen) and the bulk copies (`inflight`).
  unsigned phase = 0, issued = 0;
  unsigned fphase = 0, inflight = 0;
  bool ok = true;
  auto landed = [&](int s) -> bool {   // bounded wait for the bulk copy into stage s
    if (!tc::mbar_wait(&full[s], (fphase >> s) & 1u, kOzWaitLimit)) return false;
    fphase ^= 1u << s;
    inflight &= ~(1u << s);
    return true;
  };
  auto settle = [&](int s) -> bool {   // bounded wait for the MMAs last committed on stage s
    if (!tc::mbar_wait(&bar[s], (phase >> s) & 1u, kOzWaitLimit)) return false;
    phase ^= 1u << s;
    issued &= ~(1u << s);
    return true;
  };
  float4 cur[2], nxt[2];
  int cc = 0;                          // chunks issued by this CTA (stage rotation)
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    bt = tile % nbt;
    b0 = bt * O::BB;
    g0 = (tile / nbt) * OZ_TM;
    kend = b0 + O::BB < nk ? b0 + O::BB : nk;
    nchunks = (kend + 15) / 16;
    g = g0 + r;
    sa = ldexpf(1.0f, OZ_BETA - (g < ng ? erow[g] : 0));   // exact power of two
#pragma unroll
    for (int j = 0; j < NACC; ++j) acc[j] = 0;
    if (nchunks > 0) load_a(0, cur);
    for (int c = 0; c < nchunks; ++c, ++cc) {
      // stage s is free: thread 0 saw its previous MMAs (chunk cc - 3) complete
      // before the barrier of chunk cc - 1, or at the last drain
      const int s = cc % OZ_NSTAGE;
      unsigned char* st = base + s * O::STAGE;
      if (c + 1 < nchunks) load_a(c + 1, nxt);
      if (tid == 0) {
        copy_b(st, c, s);
        inflight |= 1u << s;
      }
      store_a(st, cur);
      tc::fence_async_smem();
      if (tid == 0) {                  // the stage the next chunk writes: its MMAs (chunk cc - 2)
        const int sn = (s + 1) % OZ_NSTAGE;
        if (((issued >> sn) & 1u) && !settle(sn)) s_fail = 1;
      }
      __syncthreads();
      if (s_fail) { ok = false; break; }
      if (tid == 0) {
        if (landed(s)) {
          tc::fence_after_sync();
          issue(st, (c % OZ_GROUP) == 0);
          tc::mma_commit(&bar[s]);
          issued |= 1u << s;
        } else {
          s_fail = 1;                  // seen by every thread after the next barrier
        }
      }
      if ((c % OZ_GROUP) == OZ_GROUP - 1 || c == nchunks - 1) {
        // thread 0 sees every MMA so far complete, then all threads drain
        if (tid == 0 && !s_fail)
          for (int i = 0; i < OZ_NSTAGE; ++i)
            if (((issued >> i) & 1u) && !settle(i)) s_fail = 1;
        __syncthreads();
        if (s_fail) { ok = false; break; }
        drain();
      }
      cur[0] = nxt[0];
      cur[1] = nxt[1];
    }
    if (!ok) break;
    {   // the tile's outputs
      const int row = 32 * (w & 3) + lane;
      const long long gg = g0 + row;
      const int ergg = gg < ng ? erow[gg] : 0;
      const int ri = (w >> 2) >= 2 ? 1 : 0;                 // column groups 0-1 real, 2-3 imaginary
      const int jq = ((w >> 2) & 1) * NACC;
      if (gg < ng) {
#pragma unroll
        for (int j = 0; j < NACC; ++j) {
          const int b = b0 + jq + j;
          if (b < nb) {
            const int e = ergg + fcol[b] - OZ_BETA * T;
            if constexpr (sizeof(OUT) == 8)   // one rounding of the exact integer, then an exact power of two
              reinterpret_cast<float*>(Out)[2 * ((long long)b * ld + gg) + ri] = ldexpf(__ll2float_rn(acc[j]), e);
            else
              reinterpret_cast<double*>(Out)[2 * ((long long)b * ld + gg) + ri] = ldexp(__ll2double_rn(acc[j]), e);
          }
        }
      }
    }
  }   // tiles
  // commits and bulk copies still outstanding (bounded; also after a lost wait)
  if (tid == 0) {
    for (int i = 0; i < OZ_NSTAGE; ++i)
      if (((issued >> i) & 1u) && !settle(i)) s_fail = 1;
    for (int i = 0; i < OZ_NSTAGE; ++i)
      if (((inflight >> i) & 1u) && !landed(i)) s_fail = 1;
  }
  __syncthreads();
  if ((!ok || s_fail) && tid == 0) {
    status[0] = -6;   // ACE_ERR_TIMEOUT
    status[1] = -3;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid < 32) tc::tmem_dealloc_warp(tmem, 512);
}

template <int T> size_t oz_bsl_bytes(int nk, int nb) {
  using O = Oz<T>;
  const size_t ntiles = (size_t)(nb + O::BB - 1) / O::BB;
  const size_t nch = (size_t)(nk + 15) / 16;
  return ntiles * nch * O::SB * O::TN * OZ_KC * 2;
}

size_t align256_(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

constexpr int kOzT = 6;   // slice depth for both output precisions

bool xi_oz_prepare() {
  cudaFuncSetAttribute(oz_outer_kernel<kOzT, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Oz<kOzT>::SMEM);
  cudaFuncSetAttribute(oz_outer_kernel<kOzT, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Oz<kOzT>::SMEM);
  return cudaGetLastError() == cudaSuccess;
}

size_t xi_oz_scratch_bytes(long long ng, int nk, int nb, bool) {
  return align256_((size_t)ng * sizeof(int)) + align256_((size_t)nb * sizeof(int)) + align256_(oz_bsl_bytes<kOzT>(nk, nb));
}

int launch_xi_oz(const void* A, int nk, const double* C, int nb, long long ld, long long ng, void* Out,
                 bool out_f64, void* scratch, int* status, cudaStream_t st) {
  char* p = static_cast<char*>(scratch);
  int* erow = reinterpret_cast<int*>(p);
  p += align256_((size_t)ng * sizeof(int));
  int* fcol = reinterpret_cast<int*>(p);
  p += align256_((size_t)nb * sizeof(int));
  unsigned short* bsl = reinterpret_cast<unsigned short*>(p);
  const float2* a = static_cast<const float2*>(A);
  const int nch = (nk + 15) / 16;
  const unsigned rgrid = (unsigned)((ng + 255) / 256 < 152 * 8 ? (ng + 255) / 256 : 152 * 8);
  oz_row_exp_kernel<<<rgrid, 256, 0, st>>>(a, nk, ld, ng, erow);
  using O = Oz<kOzT>;
  cudaMemsetAsync(bsl, 0, oz_bsl_bytes<kOzT>(nk, nb), st);
  oz_slice_b_kernel<kOzT><<<nb, 256, 0, st>>>(C, nk, nb, nch, bsl, fcol);
  const long long ntiles = (long long)((nb + O::BB - 1) / O::BB) * ((ng + OZ_TM - 1) / OZ_TM);
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const dim3 grid((unsigned)(ntiles < sms ? ntiles : sms));   // one resident CTA per SM
  if (out_f64)
    oz_outer_kernel<kOzT, double2><<<grid, OZ_THREADS, O::SMEM, st>>>(a, nk, nb, ld, ng, erow, bsl, fcol, nch,
                                                                       static_cast<double2*>(Out), status);
  else
    oz_outer_kernel<kOzT, float2><<<grid, OZ_THREADS, O::SMEM, st>>>(a, nk, nb, ld, ng, erow, bsl, fcol, nch,
                                                                      static_cast<float2*>(Out), status);
  return 3;
}

}  // namespace ace
