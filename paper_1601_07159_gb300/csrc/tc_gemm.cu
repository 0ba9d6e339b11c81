// Tensor-core (tcgen05, kind::tf32) GEMMs of the ACE construction and apply for
// complex FP32 vectors (Sec. 3):
//   gram   part[s][a][b] = sum_{g in chunk s} conj(A_a(g)) B_b(g)      (M = dV Phi^* W, C = dV Xi^* psi)
//   outer  Out_b(g) = alpha sum_k A_k(g) C[k][b]                        (Xi = W L^{-*}, Y = -Xi C)
//
// Complex products as real GEMMs on interleaved (re, im) data, for a tile of
// BB = TN / 2 complex output columns b (MMA width N = TN real columns):
//   gram:  K' = 2 N_g real terms; output columns j < BB take B_b as stored
//          (re, im) -> Re conj(a) b; columns BB + j take (im, -re) -> Im conj(a) b.
//   outer: rows = grid points g, K' = 2 K (re, im of A_k(g)); output columns
//          j < BB use (Re C, -Im C) -> Re Out, BB + j use (Im C, Re C) -> Im Out.
// TN is 128, 192 or 256, chosen per call so that the b range is covered with
// the fewest MMA columns (ties to the wider tile): a wider tile reads each A
// row from shared memory once for more output columns, and the MMAs of the
// 3-term split at N = 128 already ask for the whole shared-memory bandwidth.
// FP32 accuracy from TF32 inputs: each operand is split x = hi + lo (hi = x with
// the low 13 mantissa bits cleared, lo = x - hi exactly) and three products
// hi.hi + hi.lo + lo.hi accumulate in FP32 in tensor memory (the lo.lo term is
// below FP32 rounding).
//
// Per CTA (512 threads, one per SM): two 128 x TN FP32 accumulators in TMEM.
// K runs in chunks of 32 real terms: the threads split a chunk from registers
// and store it (then fetch the next one into the same registers at TN = 192 /
// 256; at TN = 128 two more chunks are already in flight), in the canonical
// K-major no-swizzle layout (core matrices of 8 rows x 16 bytes; LBO = 128 B
// between core matrices along K, SBO = 1024 B between 8-row groups; eight
// consecutive threads fill one core matrix, so the 16-byte stores are free of
// bank conflicts), into one of NSTAGE shared-memory stages (three of 64 KB at
// TN = 128, two of 80 / 96 KB at TN = 192 / 256). One thread issues 4 K-steps
// x 3 products of tcgen05.mma (M = 128, N = TN, K = 8) and commits them to the
// stage's mbarrier; a stage is refilled only after its commit has been seen.
//
// BF16 split (the same kernels with BF = true, tcgen05 kind::f16 with BF16
// operands): x = hi + lo with hi = bf16(x), lo = bf16(x - hi) (round to
// nearest), the same three products; 16 significant bits per operand, so a
// product carries a relative error of about 2^-16 (the lo.lo term and the
// rounding of lo) instead of FP32 rounding. The operand tiles hold 2-byte
// elements (core matrices of 8 rows x 8 values; SBO = 512 B for the 32 real
// K terms of a chunk), and a K-step of the MMA takes 16 terms, so a chunk is
// two K-steps of 3 products instead of four.
//
// The tensor core's FP32 accumulation truncates, so a long chain of MMAs into
// one accumulator drifts toward zero (about 2^-24 per accumulation). The
// accumulator therefore restarts every kGroup chunks (12 MMAs each, drift
// ~3e-6 relative), alternating between the two TMEM buffers; a finished group
// is read back (tcgen05.ld, warp w owns lanes 32 (w % 4)..+31) and added in
// FP32 registers, round-to-nearest, while the next group's MMAs run.
// Every mbarrier wait is bounded: on timeout the CTA records ACE_ERR_TIMEOUT in
// the status word, stops issuing work, waits (bounded) for what it issued and
// releases its tensor memory.
#include <cstdint>

#include "ace_internal.h"
#include "tcgen05.cuh"
#include <cuda_bf16.h>

namespace ace {

namespace {

using tc::smem_u32;
using tc::mbar_init;
using tc::mma_commit;

constexpr int THREADS = 512;
constexpr int TM = 128;                    // rows per CTA (M of the MMA)
constexpr int KC = 32;                     // real K terms per stage
constexpr int kGroup = 4;                  // chunks per accumulator group
constexpr unsigned kWaitLimit = 1u << 24;

// operand element bytes, bytes between 8-row groups (1024 TF32, 512 BF16),
// one A operand tile (128 x 32: 16 KB TF32, 8 KB BF16)
template <bool BF> constexpr int kES = BF ? 2 : 4;
template <bool BF> constexpr int kSBO = (KC * kES<BF> / 16) * 128;
template <bool BF> constexpr int kOPA = TM * KC * kES<BF>;

template <int TN, bool BF> struct Tile {
  static_assert(TN == 128 || TN == 192 || TN == 256, "MMA width");
  static constexpr int BB = TN / 2;                          // complex output columns per tile
  static constexpr int NACC = TN / 4;                        // accumulator columns per thread
  static constexpr int OPA_BYTES = kOPA<BF>;
  static constexpr int OPB_BYTES = TN * KC * kES<BF>;        // one B operand tile
  static constexpr int STAGE_BYTES = 2 * OPA_BYTES + 2 * OPB_BYTES;   // A_hi, A_lo, B_hi, B_lo
  static constexpr int NSTAGE = TN == 128 ? 3 : 2;           // chunk c uses stage c % NSTAGE
  static constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024 + 64;
  static constexpr int TMEM_COLS = TN == 128 ? 256 : 512;    // two accumulators, a power of two
  // instruction descriptor: D = F32, A = B = TF32 (format 2) or BF16 (format 1),
  // both K-major, N = TN, M = 128
  static constexpr uint32_t FMT = BF ? 1u : 2u;
  static constexpr uint32_t IDESC = (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)(TN >> 3) << 17) |
                                    ((uint32_t)(TM >> 4) << 24);
};

// shared-memory matrix descriptor of an operand tile (K-major, no swizzle)
template <bool BF> __device__ __forceinline__ uint64_t mat_desc(uint32_t addr) {
  return tc::kmajor_desc(addr, kSBO<BF>);
}

// byte offset of element (row r, real k) in an operand tile: core matrices of
// 8 rows x 16 bytes (4 TF32 or 8 BF16 values along K)
template <bool BF> __device__ __forceinline__ int tile_off(int r, int k) {
  constexpr int V = 16 / kES<BF>;
  return (r >> 3) * kSBO<BF> + (k / V) * 128 + (r & 7) * 16 + (k % V) * kES<BF>;
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ unsigned bf16_pair(float a, float b) {
  return (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
         ((unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}
__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// four consecutive K values of one row into the hi and lo tiles
template <bool BF> __device__ __forceinline__ void split_store(unsigned char* hi, unsigned char* lo, int off, float4 v) {
  if constexpr (BF) {
    const float4 h = make_float4(bf16_round(v.x), bf16_round(v.y), bf16_round(v.z), bf16_round(v.w));
    *reinterpret_cast<uint2*>(hi + off) = make_uint2(bf16_pair(h.x, h.y), bf16_pair(h.z, h.w));
    *reinterpret_cast<uint2*>(lo + off) = make_uint2(bf16_pair(v.x - h.x, v.y - h.y), bf16_pair(v.z - h.z, v.w - h.w));
  } else {
    const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
  }
}

// bounded wait for the phase with parity `parity`; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  return tc::mbar_wait(bar, parity, kWaitLimit);
}

template <int TN, bool BF>
__device__ __forceinline__ void mma_split(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  if constexpr (BF) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(Tile<TN, BF>::IDESC), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(Tile<TN, BF>::IDESC), "r"(accumulate)
        : "memory");
  }
}

// 32 consecutive accumulator columns of this thread's lane, added into acc[o .. o + 31]
template <int NACC>
__device__ __forceinline__ void tmem_add32(uint32_t taddr, float (&acc)[NACC], int o) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[o + i] += __uint_as_float(r[i]);
}

// 16 columns, added into acc[o .. o + 15]
template <int NACC>
__device__ __forceinline__ void tmem_add16(uint32_t taddr, float (&acc)[NACC], int o) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[o + i] += __uint_as_float(r[i]);
}

// this thread's NACC accumulator columns (32-column pieces, then a 16-column one)
template <int NACC>
__device__ __forceinline__ void tmem_add(uint32_t taddr, float (&acc)[NACC]) {
#pragma unroll
  for (int o = 0; o + 32 <= NACC; o += 32) tmem_add32<NACC>(taddr + (uint32_t)o, acc, o);
  if constexpr (NACC % 32 == 16) tmem_add16<NACC>(taddr + (uint32_t)(NACC - 16), acc, NACC - 16);
}

struct TcState {
  uint64_t* bar;        // [NSTAGE] stage barriers
  uint32_t* tmem_slot;  // TMEM base address written by tcgen05.alloc
  unsigned char* stage; // NSTAGE stages
};

template <int TN, bool BF>
__device__ __forceinline__ TcState tc_setup(unsigned char* smem) {
  using T = Tile<TN, BF>;
  TcState s;
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem + 1023) & ~(uintptr_t)1023);
  s.stage = base;
  s.bar = reinterpret_cast<uint64_t*>(base + T::NSTAGE * T::STAGE_BYTES);
  s.tmem_slot = reinterpret_cast<uint32_t*>(base + T::NSTAGE * T::STAGE_BYTES + 32);
  if (threadIdx.x == 0) {
    for (int i = 0; i < T::NSTAGE; ++i) mbar_init(&s.bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {   // warp 0 allocates the two accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s.tmem_slot)),
                 "r"(T::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return s;
}

template <int TN, bool BF>
__device__ __forceinline__ void tc_teardown(uint32_t tmem) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Tile<TN, BF>::TMEM_COLS)
                 : "memory");
}

// One K chunk in a stage: 4 (TF32) or 2 (BF16) K-steps x 3 split products into
// accumulator `dtmem`, committed to `bar`.
template <int TN, bool BF>
__device__ __forceinline__ void issue_chunk(uint32_t dtmem, const unsigned char* st, uint64_t* bar, bool first) {
  using T = Tile<TN, BF>;
  const uint32_t ah = smem_u32(st), al = ah + T::OPA_BYTES, bh = ah + 2 * T::OPA_BYTES, bl = bh + T::OPB_BYTES;
#pragma unroll
  for (int ks = 0; ks < KC / (BF ? 16 : 8); ++ks) {
    const uint32_t o = ks * 256;   // two core matrices of 16 B along K per step
    mma_split<TN, BF>(dtmem, mat_desc<BF>(ah + o), mat_desc<BF>(bh + o), (first && ks == 0) ? 0u : 1u);
    mma_split<TN, BF>(dtmem, mat_desc<BF>(ah + o), mat_desc<BF>(bl + o), 1u);
    mma_split<TN, BF>(dtmem, mat_desc<BF>(al + o), mat_desc<BF>(bh + o), 1u);
  }
  mma_commit(bar);
}

// Main loop shared by both kernels: load(c, regs) fetches chunk c from global
// memory, store(stage, regs) splits it into the stage. At TN = 128 (three
// stages) chunks are fetched two ahead in two register sets. At TN = 192 / 256
// one register set serves: chunk c + 1 is fetched into it as soon as chunk c
// is stored, and arrives while the thread waits on the MMAs of chunk c - 1.
// (A second set held across the iteration pushed TN = 256 past the 128-register
// cap of 512 threads, and its spills exposed the loads' latency: 29 % slower.)
// On return thread (warp w, lane) holds acc[j] = D[row 32 (w % 4) + lane][col
// NACC (w / 4) + j]. Each thread waits (bounded) for the commit of the chunk
// that last used a stage before storing into it, and drains a finished
// accumulator group when that commit is the group's last; one block barrier
// per chunk hands the stage to the issuing thread. A lost wait sets s_fail,
// which every thread reads after that barrier, so all leave the loop together.
template <int TN, bool BF, typename Regs, typename Load, typename Store>
__device__ __forceinline__ bool tc_mainloop(const TcState& S, uint32_t tmem, int nchunks,
                                            float (&acc)[Tile<TN, BF>::NACC], Load load, Store store) {
  using T = Tile<TN, BF>;
  constexpr int NS = T::NSTAGE;
  const int tid = threadIdx.x, w = tid >> 5;
  const uint32_t lane_col = ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(T::NACC * (w >> 2));
  __shared__ int s_fail;
  // per-stage state in registers: bit s of `phase` / `issued` (commit on the
  // stage not yet seen), two bits per stage of `drain` (1 + accumulator buffer
  // to read once that commit is seen, 0 for none)
  unsigned phase = 0, issued = 0, drain = 0;
  bool ok = true;
#pragma unroll
  for (int j = 0; j < T::NACC; ++j) acc[j] = 0.f;
  if (tid == 0) s_fail = 0;
  __syncthreads();

  // this thread's bounded wait for the commit on stage s, then the pending drain
  auto settle = [&](int s) -> bool {
    if (!mbar_wait(&S.bar[s], (phase >> s) & 1u)) {
      s_fail = 1;
      return false;
    }
    phase ^= 1u << s;
    issued &= ~(1u << s);
    const unsigned d = (drain >> (2 * s)) & 3u;
    if (d) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      tmem_add<T::NACC>(tmem + lane_col + (uint32_t)(TN * (d - 1)), acc);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      drain &= ~(3u << (2 * s));
    }
    return true;
  };
  // chunk c from registers into its stage (with `reload`, chunk c + 1 then
  // fetched into the same registers), then the MMAs; false once a wait was lost
  auto step = [&](int c, int s, Regs& cur, bool reload) -> bool {
    unsigned char* st = S.stage + s * T::STAGE_BYTES;
    if ((issued >> s) & 1u) settle(s);   // the MMAs of chunk c - NSTAGE read this stage
    store(st, cur);
    if (reload && c + 1 < nchunks) load(c + 1, cur);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (s_fail) return false;
    const int group = c / kGroup;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      issue_chunk<TN, BF>(tmem + (uint32_t)(TN * (group & 1)), st, &S.bar[s], (c % kGroup) == 0);
    }
    issued |= 1u << s;
    if ((c % kGroup) == kGroup - 1 || c == nchunks - 1) drain |= (1u + (unsigned)(group & 1)) << (2 * s);
    return true;
  };

  int s = 0;
  if constexpr (NS == 3) {
    Regs r0, r1, r2;   // chunks c, c + 1, c + 2 (rotated by register moves)
    if (nchunks > 0) load(0, r0);
    if (nchunks > 1) load(1, r1);
    for (int c = 0; c < nchunks; ++c) {
      if (c + 2 < nchunks) load(c + 2, r2);
      if (!step(c, s, r0, false)) {
        ok = false;
        break;
      }
      r0 = r1;
      r1 = r2;
      s = s + 1 == NS ? 0 : s + 1;
    }
  } else {
    Regs r0;           // chunk c, then (once stored) chunk c + 1
    if (nchunks > 0) load(0, r0);
    for (int c = 0; c < nchunks; ++c) {
      if (!step(c, s, r0, true)) {
        ok = false;
        break;
      }
      s = s + 1 == NS ? 0 : s + 1;
    }
  }
  // remaining commits, in chunk order (bounded; also after a lost wait)
  for (int i = 0; i < NS; ++i) {
    if (((issued >> s) & 1u) && !settle(s)) ok = false;
    s = s + 1 == NS ? 0 : s + 1;
  }
  __syncthreads();
  return ok && !s_fail;
}

// ---------------------------------------------------------------- gram
// Grid: (ceil(na/128), ceil(nb/BB), splits). part is FP64 complex [splits][na][nb].
// Chunk element e (A: 0..1023, B: 0..8 BB - 1) -> row 8 (e / 64) + e % 8, complex
// pair (e / 8) % 8 (four real K terms).
template <int TN, bool BF>
__global__ void __launch_bounds__(THREADS, 1)
gram_tc_kernel(const float2* __restrict__ A, int na, const float2* __restrict__ B, int nb, long long ld,
               long long ng, double* __restrict__ part, long long chunk, int* status) {
  using T = Tile<TN, BF>;
  constexpr int BB = T::BB, NACC = T::NACC;
  constexpr int NBE = 8 * BB;                           // B float4 elements per chunk
  constexpr int NBT = (NBE + THREADS - 1) / THREADS;    // per thread
  extern __shared__ unsigned char smem_raw[];
  TcState S = tc_setup<TN, BF>(smem_raw);
  const uint32_t tmem = *S.tmem_slot;
  const int tid = threadIdx.x;
  const int a0 = blockIdx.x * TM, b0 = blockIdx.y * BB;
  const long long g_begin = (long long)blockIdx.z * chunk;
  const long long g_end = g_begin + chunk < ng ? g_begin + chunk : ng;
  const int nchunks = g_end > g_begin ? (int)((g_end - g_begin + KC / 2 - 1) / (KC / 2)) : 0;
  struct Regs { float4 a[2], b[NBT]; };
  auto rowq = [](int e, int& r, int& q) { r = ((e >> 6) << 3) | (e & 7); q = (e >> 3) & 7; };
  auto load = [&](int c, Regs& Rg) {
    const long long g0 = g_begin + (long long)c * (KC / 2);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      int r, q;
      rowq(tid + THREADS * i, r, q);
      const long long g = g0 + 2 * q;   // even; g_end is even, so g < g_end covers g + 1
      Rg.a[i] = (a0 + r < na && g < g_end)
                    ? *reinterpret_cast<const float4*>(A + (long long)(a0 + r) * ld + g)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < NBT; ++i) {
      const int e = tid + THREADS * i;
      int r, q;
      rowq(e, r, q);
      const long long g = g0 + 2 * q;
      Rg.b[i] = (e < NBE && b0 + r < nb && g < g_end)
                    ? *reinterpret_cast<const float4*>(B + (long long)(b0 + r) * ld + g)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto store = [&](unsigned char* st, const Regs& Rg) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      int r, q;
      rowq(tid + THREADS * i, r, q);
      split_store<BF>(st, st + T::OPA_BYTES, tile_off<BF>(r, 4 * q), Rg.a[i]);
    }
    unsigned char* bh = st + 2 * T::OPA_BYTES;
    unsigned char* bl = bh + T::OPB_BYTES;
#pragma unroll
    for (int i = 0; i < NBT; ++i) {
      const int e = tid + THREADS * i;
      if (e < NBE) {
        int r, q;
        rowq(e, r, q);
        const float4 vb = Rg.b[i];
        split_store<BF>(bh, bl, tile_off<BF>(r, 4 * q), vb);
        split_store<BF>(bh, bl, tile_off<BF>(r + BB, 4 * q), make_float4(vb.y, -vb.x, vb.w, -vb.z));
      }
    }
  };
  float acc[NACC];
  const bool ok = tc_mainloop<TN, BF, Regs>(S, tmem, nchunks, acc, load, store);
  if (!ok && tid == 0) {
    status[0] = -6;   // ACE_ERR_TIMEOUT
    status[1] = -1;
  }
  const int w = tid >> 5, lane = tid & 31;
  const int a = a0 + 32 * (w & 3) + lane;
  const int ri = (w >> 2) >> 1, bq = ((w >> 2) & 1) * NACC;   // column blocks 0-1 real, 2-3 imaginary
  if (ok && a < na) {
    double* out = part + ((long long)blockIdx.z * na + a) * nb * 2 + ri;
#pragma unroll
    for (int j = 0; j < NACC; ++j)
      if (b0 + bq + j < nb) out[2 * (b0 + bq + j)] = (double)acc[j];
  }
  tc_teardown<TN, BF>(tmem);
}

// ---------------------------------------------------------------- outer
// Grid: (ceil(nb/BB), ceil(ng/128)). C: complex [nk][nb] rounded to FP32 once
// per call (c_to_f32_kernel), so the CTAs of every row block read FP32.
// A element e (0..1023): grid point g0 + e % 128, K pair e / 128 (k = 2 (e / 128)).
// B element e (0..8 BB - 1): b = b0 + e % BB, K pair e / BB.
template <int TN, bool BF>
__global__ void __launch_bounds__(THREADS, 1)
outer_tc_kernel(const float2* __restrict__ A, int nk, const float2* __restrict__ C, int nb, long long ld,
                long long ng, double alpha, float* __restrict__ Out, int* status) {
  using T = Tile<TN, BF>;
  constexpr int BB = T::BB, NACC = T::NACC;
  constexpr int NBE = 8 * BB;
  constexpr int NBT = (NBE + THREADS - 1) / THREADS;
  extern __shared__ unsigned char smem_raw[];
  TcState S = tc_setup<TN, BF>(smem_raw);
  const uint32_t tmem = *S.tmem_slot;
  const int tid = threadIdx.x;
  const int b0 = blockIdx.x * BB;
  const long long g0 = (long long)blockIdx.y * TM;
  const int nchunks = (nk + KC / 2 - 1) / (KC / 2);
  struct Regs { float4 a[2], c[NBT]; };
  auto load = [&](int c, Regs& Rg) {
    const int k0 = c * (KC / 2);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int e = tid + THREADS * i, r = e & 127, k = k0 + 2 * (e >> 7);
      const long long g = g0 + r;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (g < ng) {
        if (k < nk) { const float2 t = A[(long long)k * ld + g]; v.x = t.x; v.y = t.y; }
        if (k + 1 < nk) { const float2 t = A[(long long)(k + 1) * ld + g]; v.z = t.x; v.w = t.y; }
      }
      Rg.a[i] = v;
    }
#pragma unroll
    for (int i = 0; i < NBT; ++i) {
      const int e = tid + THREADS * i, j = e % BB, k = k0 + 2 * (e / BB);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e < NBE && b0 + j < nb) {
        if (k < nk) {
          const float2 t = C[(long long)k * nb + b0 + j];
          v.x = t.x;
          v.y = t.y;
        }
        if (k + 1 < nk) {
          const float2 t = C[(long long)(k + 1) * nb + b0 + j];
          v.z = t.x;
          v.w = t.y;
        }
      }
      Rg.c[i] = v;   // (Re C_k, Im C_k, Re C_k+1, Im C_k+1)
    }
  };
  auto store = [&](unsigned char* st, const Regs& Rg) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int e = tid + THREADS * i, r = e & 127, kq = 4 * (e >> 7);
      split_store<BF>(st, st + T::OPA_BYTES, tile_off<BF>(r, kq), Rg.a[i]);
    }
    unsigned char* bh = st + 2 * T::OPA_BYTES;
    unsigned char* bl = bh + T::OPB_BYTES;
#pragma unroll
    for (int i = 0; i < NBT; ++i) {
      const int e = tid + THREADS * i, j = e % BB, kq = 4 * (e / BB);
      if (e < NBE) {
        const float4 v = Rg.c[i];
        split_store<BF>(bh, bl, tile_off<BF>(j, kq), make_float4(v.x, -v.y, v.z, -v.w));
        split_store<BF>(bh, bl, tile_off<BF>(j + BB, kq), make_float4(v.y, v.x, v.w, v.z));
      }
    }
  };
  float acc[NACC];
  const bool ok = tc_mainloop<TN, BF, Regs>(S, tmem, nchunks, acc, load, store);
  if (!ok && tid == 0) {
    status[0] = -6;   // ACE_ERR_TIMEOUT
    status[1] = -2;
  }
  const int w = tid >> 5, lane = tid & 31;
  const long long g = g0 + 32 * (w & 3) + lane;
  const int ri = (w >> 2) >> 1, bq = ((w >> 2) & 1) * NACC;
  if (ok && g < ng) {
#pragma unroll
    for (int j = 0; j < NACC; ++j)
      if (b0 + bq + j < nb) Out[2 * ((long long)(b0 + bq + j) * ld + g) + ri] = (float)alpha * acc[j];
  }
  tc_teardown<TN, BF>(tmem);
}

// Exact diagonal of the gram product: Mc[a][a] = (scale Re sum_g conj(A_a) B_a, 0),
// FP32 products summed in FP32 over short runs and in FP64 across them.
// Grid: (na, splits), splits <= kDiagSplits; part: FP64 [na][kDiagSplits].
constexpr int kDiagSplits = 32;
__global__ void __launch_bounds__(256)
diag_dot_kernel(const float2* __restrict__ A, const float2* __restrict__ B, long long ld, long long ng,
                double* __restrict__ part) {
  __shared__ double red[8];
  const int a = blockIdx.x;
  const long long per = (ng + gridDim.y - 1) / gridDim.y;
  const long long g0 = blockIdx.y * per, g1 = g0 + per < ng ? g0 + per : ng;
  double s = 0.0;
  float run = 0.f;
  int cnt = 0;
  for (long long g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const float2 x = A[(long long)a * ld + g], y = B[(long long)a * ld + g];
    run = fmaf(x.x, y.x, fmaf(x.y, y.y, run));
    if (++cnt == 16) { s += (double)run; run = 0.f; cnt = 0; }
  }
  s += (double)run;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    part[(long long)a * kDiagSplits + blockIdx.y] = t;
  }
}

__global__ void diag_fix_kernel(const double* __restrict__ part, int na, int splits, double scale,
                                double* __restrict__ Mc) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= na) return;
  double t = 0.0;
  for (int k = 0; k < splits; ++k) t += part[(long long)a * kDiagSplits + k];
  Mc[2 * ((long long)a * na + a)] = scale * t;
  Mc[2 * ((long long)a * na + a) + 1] = 0.0;
}

// complex FP64 -> FP32 (the outer products' right operand, converted once)
__global__ void c_to_f32_kernel(const double2* __restrict__ C, long long count, float2* __restrict__ Cf) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) Cf[i] = make_float2((float)C[i].x, (float)C[i].y);
}

// MMA width for nb output columns: the fewest MMA columns over the b tiles,
// ties to the wider tile.
int tc_width(int nb) {
  int best = 256;
  long long cost = -1;
  for (const int tn : {256, 192, 128}) {
    const long long c = (long long)((nb + tn / 2 - 1) / (tn / 2)) * tn;
    if (cost < 0 || c < cost) {
      cost = c;
      best = tn;
    }
  }
  return best;
}

template <int TN, bool BF> void set_smem() {
  cudaFuncSetAttribute((const void*)gram_tc_kernel<TN, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       Tile<TN, BF>::SMEM_BYTES);
  cudaFuncSetAttribute((const void*)outer_tc_kernel<TN, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       Tile<TN, BF>::SMEM_BYTES);
}

template <int TN, bool BF>
void gram_tn(dim3 grid, cudaStream_t st, const float2* a, int na, const float2* b, int nb, long long ld,
             long long ng, double* part, long long chunk, int* status) {
  gram_tc_kernel<TN, BF><<<grid, THREADS, Tile<TN, BF>::SMEM_BYTES, st>>>(a, na, b, nb, ld, ng, part, chunk, status);
}

template <int TN, bool BF>
void outer_tn(dim3 grid, cudaStream_t st, const float2* a, int nk, const float2* C, int nb, long long ld,
              long long ng, double alpha, float* o, int* status) {
  outer_tc_kernel<TN, BF><<<grid, THREADS, Tile<TN, BF>::SMEM_BYTES, st>>>(a, nk, C, nb, ld, ng, alpha, o, status);
}

}  // namespace

bool tc_gemm_prepare() {
  set_smem<128, false>();
  set_smem<192, false>();
  set_smem<256, false>();
  set_smem<128, true>();
  set_smem<192, true>();
  set_smem<256, true>();
  return cudaGetLastError() == cudaSuccess;
}

// Split-K count for `tiles` output tiles on 152 SMs (one CTA per SM): the one
// that minimises waves / splits (the time of a CTA's K range times the number
// of waves). 1 tile -> 152 splits (one wave); 64 tiles -> 7 (448 CTAs, 98 % of
// three waves, where 2 splits left 24 SMs idle); 96 tiles -> 11 (1 split used
// 96 of 152 SMs). Ties within 2 % go to fewer splits (fewer partial sums).
int gram_tc_splits(long long ng, int na, int nb) {
  constexpr long long kSMs = 152, kMaxSplits = 1024;
  const int bb = tc_width(nb) / 2;
  const long long tiles = (long long)((na + TM - 1) / TM) * ((nb + bb - 1) / bb);
  long long max_s = (ng + KC / 2 - 1) / (KC / 2);
  if (max_s > kMaxSplits) max_s = kMaxSplits;
  long long best = 1;
  double best_cost = 1e300;
  for (long long s = 1; s <= max_s; ++s) {
    const double cost = (double)((tiles * s + kSMs - 1) / kSMs) / (double)s;
    if (cost < best_cost * 0.98) {
      best_cost = cost;
      best = s;
    }
  }
  return (int)best;
}

void launch_gram_tc(const void* A, int na, const void* B, int nb, long long ld, long long ng, double* part,
                    int splits, int* status, cudaStream_t st, bool bf16) {
  long long chunk = (ng + splits - 1) / splits;
  chunk = (chunk + KC / 2 - 1) / (KC / 2) * (KC / 2);
  const int tn = tc_width(nb), bb = tn / 2;
  const dim3 grid((na + TM - 1) / TM, (nb + bb - 1) / bb, splits);
  const float2* a = static_cast<const float2*>(A);
  const float2* b = static_cast<const float2*>(B);
  if (bf16) {
    if (tn == 256) gram_tn<256, true>(grid, st, a, na, b, nb, ld, ng, part, chunk, status);
    else if (tn == 192) gram_tn<192, true>(grid, st, a, na, b, nb, ld, ng, part, chunk, status);
    else gram_tn<128, true>(grid, st, a, na, b, nb, ld, ng, part, chunk, status);
  } else {
    if (tn == 256) gram_tn<256, false>(grid, st, a, na, b, nb, ld, ng, part, chunk, status);
    else if (tn == 192) gram_tn<192, false>(grid, st, a, na, b, nb, ld, ng, part, chunk, status);
    else gram_tn<128, false>(grid, st, a, na, b, nb, ld, ng, part, chunk, status);
  }
}

void launch_outer_tc(const void* A, int nk, const double* C64, int nb, long long ld, long long ng, double alpha,
                     void* Out, void* c32, int* status, cudaStream_t st, bool bf16) {
  const int tn = tc_width(nb), bb = tn / 2;
  const dim3 grid((nb + bb - 1) / bb, (unsigned)((ng + TM - 1) / TM));
  const float2* a = static_cast<const float2*>(A);
  float* o = static_cast<float*>(Out);
  const long long nc = (long long)nk * nb;
  float2* C = static_cast<float2*>(c32);
  c_to_f32_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(reinterpret_cast<const double2*>(C64), nc, C);
  if (bf16) {
    if (tn == 256) outer_tn<256, true>(grid, st, a, nk, C, nb, ld, ng, alpha, o, status);
    else if (tn == 192) outer_tn<192, true>(grid, st, a, nk, C, nb, ld, ng, alpha, o, status);
    else outer_tn<128, true>(grid, st, a, nk, C, nb, ld, ng, alpha, o, status);
  } else {
    if (tn == 256) outer_tn<256, false>(grid, st, a, nk, C, nb, ld, ng, alpha, o, status);
    else if (tn == 192) outer_tn<192, false>(grid, st, a, nk, C, nb, ld, ng, alpha, o, status);
    else outer_tn<128, false>(grid, st, a, nk, C, nb, ld, ng, alpha, o, status);
  }
}

size_t diag_dot_part_doubles(int na) { return (size_t)na * kDiagSplits; }

void launch_diag_exact(const void* A, const void* B, int na, long long ld, long long ng, double scale,
                       double* part, double* Mc, cudaStream_t st) {
  // about two waves of 256-thread blocks (eight per SM), at most kDiagSplits per orbital
  int splits = 2 * 152 * 8 / (na > 0 ? na : 1);
  splits = splits < 4 ? 4 : (splits > kDiagSplits ? kDiagSplits : splits);
  diag_dot_kernel<<<dim3(na, splits), 256, 0, st>>>(static_cast<const float2*>(A),
                                                    static_cast<const float2*>(B), ld, ng, part);
  diag_fix_kernel<<<(na + 127) / 128, 128, 0, st>>>(part, na, splits, scale, Mc);
}

}  // namespace ace
