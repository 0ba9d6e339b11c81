// Tensor-core (tcgen05, kind::tf32) GEMMs of the ACE construction and apply for
// complex FP32 vectors (Sec. 3):
//   gram   part[s][a][b] = sum_{g in chunk s} conj(A_a(g)) B_b(g)      (M = dV Phi^* W, C = dV Xi^* psi)
//   outer  Out_b(g) = alpha sum_k A_k(g) C[k][b]                        (Xi = W L^{-*}, Y = -Xi C)
//
// Complex products as real GEMMs on interleaved (re, im) data:
//   gram:  K' = 2 N_g real terms; output columns j < 64 take B_b as stored
//          (re, im) -> Re conj(a) b; columns 64 + j take (im, -re) -> Im conj(a) b.
//   outer: rows = grid points g, K' = 2 K (re, im of A_k(g)); output columns
//          j < 64 use (Re C, -Im C) -> Re Out, 64 + j use (Im C, Re C) -> Im Out.
// FP32 accuracy from TF32 inputs: each operand is split x = hi + lo (hi = x with
// the low 13 mantissa bits cleared, lo = x - hi exactly) and three products
// hi.hi + hi.lo + lo.hi accumulate in FP32 in tensor memory (the lo.lo term is
// below FP32 rounding).
//
// Per CTA: a 128 x 128 FP32 accumulator in TMEM (128 columns); 256 threads load
// a K chunk of 32 real terms, split it and store hi / lo in the canonical
// K-major no-swizzle layout (core matrices of 8 rows x 16 bytes; LBO = 128 B
// between core matrices along K, SBO = 1024 B between 8-row groups) in one of
// two shared-memory stages; one thread issues 4 K-steps x 3 products of
// tcgen05.mma (M = 128, N = 128, K = 8) and commits them to the stage's
// mbarrier, which the threads wait on before refilling that stage. Warps 0-3
// read the accumulator back with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31).
// Every mbarrier wait is bounded: on timeout the CTA records an error in the
// status word, stops issuing work, waits (bounded) for what it issued and
// releases its tensor memory.
#include <cstdint>

#include "ace_internal.h"

namespace ace {

namespace {

constexpr int TM = 128;            // rows per CTA (M of the MMA)
constexpr int TN = 128;            // accumulator columns (N of the MMA)
constexpr int KC = 32;             // real K terms per stage
constexpr int SBO = (KC / 4) * 128;        // bytes between 8-row groups = 1024
constexpr int OP_BYTES = TM * KC * 4;      // one operand tile (128 x 32 FP32) = 16 KB
constexpr int STAGE_BYTES = 4 * OP_BYTES;  // A_hi, A_lo, B_hi, B_lo = 64 KB
constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 1024;
constexpr unsigned kWaitLimit = 1u << 24;

// instruction descriptor: D = F32, A = B = TF32, both K-major, N = 128, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t mat_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(SBO >> 4) << 32) | (1ull << 46);
}

// byte offset of element (row r, real k) in an operand tile
__device__ __forceinline__ int tile_off(int r, int k) {
  return (r >> 3) * SBO + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ void split_store(unsigned char* hi, unsigned char* lo, int off, float4 v) {
  const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
  *reinterpret_cast<float4*>(hi + off) = h;
  *reinterpret_cast<float4*>(lo + off) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
}
__device__ __forceinline__ void split_store2(unsigned char* hi, unsigned char* lo, int off, float a, float b) {
  const float ha = tf32_hi(a), hb = tf32_hi(b);
  *reinterpret_cast<float2*>(hi + off) = make_float2(ha, hb);
  *reinterpret_cast<float2*>(lo + off) = make_float2(a - ha, b - hb);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// bounded wait for the phase with parity `parity`; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const uint32_t a = smem_u32(bar);
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
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
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared prologue / epilogue of both kernels.
struct TcState {
  uint64_t* bar;        // [2] stage barriers
  uint32_t* tmem_slot;  // TMEM base address written by tcgen05.alloc
  unsigned char* stage; // 2 stages of 64 KB
};

__device__ __forceinline__ TcState tc_setup(unsigned char* smem) {
  TcState s;
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem + 1023) & ~(uintptr_t)1023);
  s.stage = base;
  s.bar = reinterpret_cast<uint64_t*>(base + 2 * STAGE_BYTES);
  s.tmem_slot = reinterpret_cast<uint32_t*>(base + 2 * STAGE_BYTES + 16);
  if (threadIdx.x == 0) {
    mbar_init(&s.bar[0], 1);
    mbar_init(&s.bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {   // warp 0 allocates the 128-column accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s.tmem_slot)),
                 "r"(TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return s;
}

__device__ __forceinline__ void tc_teardown(const TcState& s, uint32_t tmem) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
}

// Block-uniform wait for the outstanding commit of stage s: thread 0 polls
// (bounded) and the block takes its answer; on success the stage's phase flips.
__device__ __forceinline__ bool stage_wait(const TcState& S, int s, unsigned (&phase)[2], int (&issued)[2]) {
  const bool mine = threadIdx.x == 0 ? mbar_wait(&S.bar[s], phase[s]) : true;
  const bool all = __syncthreads_and(mine ? 1 : 0) != 0;
  if (all) {
    phase[s] ^= 1;
    issued[s] = 0;
  }
  return all;
}

// One K chunk in a stage: 4 K-steps x 3 split products, committed to `bar`.
__device__ __forceinline__ void issue_chunk(uint32_t tmem, const unsigned char* st, uint64_t* bar, bool first) {
  const uint32_t ah = smem_u32(st), al = ah + OP_BYTES, bh = ah + 2 * OP_BYTES, bl = ah + 3 * OP_BYTES;
#pragma unroll
  for (int ks = 0; ks < KC / 8; ++ks) {
    const uint32_t o = ks * 256;   // two core matrices of 16 B along K per step
    mma_tf32(tmem, mat_desc(ah + o), mat_desc(bh + o), (first && ks == 0) ? 0u : 1u);
    mma_tf32(tmem, mat_desc(ah + o), mat_desc(bl + o), 1u);
    mma_tf32(tmem, mat_desc(al + o), mat_desc(bh + o), 1u);
  }
  mma_commit(bar);
}

// Main loop shared by both kernels. fill(stage, c) stores K chunk c. The TMEM
// accumulator restarts every kGroup chunks and is drained into FP32 registers:
// the tensor core's FP32 accumulation truncates, so a long chain of MMAs into
// one accumulator drifts toward zero (about 2^-24 per accumulation); groups
// of kGroup chunks (12 MMAs each) bound that drift to ~3e-6 relative, and the
// register sums across groups round to nearest. Thread (warp w, lane) ends
// with acc[j] = D[row 32 (w % 4) + lane][col 64 (w / 4) + j].
constexpr int kGroup = 4;

template <typename Regs, typename Load, typename Store>
__device__ __forceinline__ bool tc_mainloop(const TcState& S, uint32_t tmem, int nchunks, float (&acc)[64],
                                            Load load, Store store) {
  const int tid = threadIdx.x, w = tid >> 5;
  const uint32_t taddr = tmem + ((uint32_t)(32 * (w & 3)) << 16) + 64 * (w >> 2);
  unsigned phase[2] = {0, 0};
  int issued[2] = {0, 0};   // commits on a stage not yet waited for (0 or 1)
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 64; ++j) acc[j] = 0.f;
  Regs cur, nxt;   // chunk c in registers; chunk c + 1 loads while c is stored and issued
  if (nchunks > 0) load(0, cur);
  for (int c = 0; c < nchunks && ok; ++c) {
    const int s = c & 1;
    unsigned char* st = S.stage + s * STAGE_BYTES;
    if (c + 1 < nchunks) load(c + 1, nxt);
    if (issued[s]) {   // the MMAs of chunk c-2 read this stage
      ok = stage_wait(S, s, phase, issued);
      if (!ok) break;
    }
    store(st, cur);
    cur = nxt;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      issue_chunk(tmem, st, &S.bar[s], (c % kGroup) == 0);
    }
    issued[s] = 1;
    if ((c % kGroup) == kGroup - 1 || c == nchunks - 1) {
      ok = stage_wait(S, s, phase, issued);   // this commit covers every MMA issued so far
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float v[32];
      tmem_ld32(taddr, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] += v[j];
      tmem_ld32(taddr + 32, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[32 + j] += v[j];
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();   // all reads done before the next group's first MMA overwrites
    }
  }
  // commits still in flight (only after a timeout): bounded wait before TMEM is freed
  for (int s = 0; s < 2; ++s)
    if (issued[s]) ok = stage_wait(S, s, phase, issued) && ok;
  return ok;
}

// ---------------------------------------------------------------- gram
// Grid: (ceil(na/128), ceil(nb/64), splits). part is FP64 complex [splits][na][nb].
__global__ void __launch_bounds__(256, 1)
gram_tc_kernel(const float2* __restrict__ A, int na, const float2* __restrict__ B, int nb, long long ld,
               long long ng, double* __restrict__ part, long long chunk, int* status) {
  extern __shared__ unsigned char smem_raw[];
  TcState S = tc_setup(smem_raw);
  const uint32_t tmem = *S.tmem_slot;
  const int tid = threadIdx.x;
  const int a0 = blockIdx.x * TM, b0 = blockIdx.y * 64;
  const long long g_begin = (long long)blockIdx.z * chunk;
  const long long g_end = g_begin + chunk < ng ? g_begin + chunk : ng;
  const int nchunks = g_end > g_begin ? (int)((g_end - g_begin + KC / 2 - 1) / (KC / 2)) : 0;
  // A: 128 rows x 16 complex; B: 64 rows x 16 complex -> 128 operand rows.
  // Element e = tid + 256 i (i < 4): row e / 8, complex pair e % 8 (4 real K terms).
  struct Regs { float4 a[4], b[2]; };
  auto load = [&](int c, Regs& R) {
    const long long g0 = g_begin + (long long)c * (KC / 2);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + 256 * i, r = e >> 3, q = e & 7;
      const long long g = g0 + 2 * q;
      float4 va = make_float4(0.f, 0.f, 0.f, 0.f);
      if (a0 + r < na) {
        const float2* pa = A + (long long)(a0 + r) * ld + g;
        if (g < g_end) { const float2 t = pa[0]; va.x = t.x; va.y = t.y; }
        if (g + 1 < g_end) { const float2 t = pa[1]; va.z = t.x; va.w = t.y; }
      }
      R.a[i] = va;
      if (i < 2) {   // rows r < 64 also carry B
        float4 vb = make_float4(0.f, 0.f, 0.f, 0.f);
        if (b0 + r < nb) {
          const float2* pb = B + (long long)(b0 + r) * ld + g;
          if (g < g_end) { const float2 t = pb[0]; vb.x = t.x; vb.y = t.y; }
          if (g + 1 < g_end) { const float2 t = pb[1]; vb.z = t.x; vb.w = t.y; }
        }
        R.b[i] = vb;
      }
    }
  };
  auto store = [&](unsigned char* st, const Regs& R) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + 256 * i, r = e >> 3, q = e & 7;
      split_store(st, st + OP_BYTES, tile_off(r, 4 * q), R.a[i]);
      if (i < 2) {
        const float4 vb = R.b[i];
        split_store(st + 2 * OP_BYTES, st + 3 * OP_BYTES, tile_off(r, 4 * q), vb);
        split_store(st + 2 * OP_BYTES, st + 3 * OP_BYTES, tile_off(r + 64, 4 * q),
                    make_float4(vb.y, -vb.x, vb.w, -vb.z));
      }
    }
  };
  float acc[64];
  const bool ok = tc_mainloop<Regs>(S, tmem, nchunks, acc, load, store);
  if (!ok && tid == 0) {
    status[0] = -6;   // ACE_ERR_TIMEOUT
    status[1] = -1;
  }
  const int w = tid >> 5, lane = tid & 31;
  const int a = a0 + 32 * (w & 3) + lane, part_ri = w >> 2;   // 0: real columns, 1: imaginary
  if (ok && a < na) {
    double* out = part + ((long long)blockIdx.z * na + a) * nb * 2 + part_ri;
#pragma unroll
    for (int j = 0; j < 64; ++j)
      if (b0 + j < nb) out[2 * (b0 + j)] = (double)acc[j];
  }
  tc_teardown(S, tmem);
}

// ---------------------------------------------------------------- outer
// Grid: (ceil(nb/64), ceil(ng/128)). C: FP64 complex [nk][nb].
__global__ void __launch_bounds__(256, 1)
outer_tc_kernel(const float2* __restrict__ A, int nk, const double* __restrict__ C, int nb, long long ld,
                long long ng, double alpha, float* __restrict__ Out, int* status) {
  extern __shared__ unsigned char smem_raw[];
  TcState S = tc_setup(smem_raw);
  const uint32_t tmem = *S.tmem_slot;
  const int tid = threadIdx.x;
  const int b0 = blockIdx.x * 64;
  const long long g0 = (long long)blockIdx.y * TM;
  const int nchunks = (nk + KC / 2 - 1) / (KC / 2);
  // A rows = grid points: element (g, k) of A_k(g), e = tid + 256 i (i < 8):
  // k = e / 128, g = g0 + e % 128 (loads run along g, coalesced).
  // B rows: j < 64 -> (Re C, -Im C), 64 + j -> (Im C, Re C), for b = b0 + j;
  // e = tid + 256 i (i < 4): j = e / 16, k = e % 16.
  struct Regs { float2 a[8], c[4]; };
  auto load = [&](int c, Regs& R) {
    const int k0 = c * (KC / 2);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int e = tid + 256 * i, kk = e >> 7, r = e & 127;
      const long long g = g0 + r;
      float2 v = make_float2(0.f, 0.f);
      if (k0 + kk < nk && g < ng) v = A[(long long)(k0 + kk) * ld + g];
      R.a[i] = v;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + 256 * i, j = e >> 4, kk = e & 15;
      float2 v = make_float2(0.f, 0.f);
      if (k0 + kk < nk && b0 + j < nb) {
        const long long o = 2 * ((long long)(k0 + kk) * nb + b0 + j);
        v = make_float2((float)C[o], (float)C[o + 1]);
      }
      R.c[i] = v;
    }
  };
  auto store = [&](unsigned char* st, const Regs& R) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int e = tid + 256 * i, kk = e >> 7, r = e & 127;
      split_store2(st, st + OP_BYTES, tile_off(r, 2 * kk), R.a[i].x, R.a[i].y);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + 256 * i, j = e >> 4, kk = e & 15;
      const float cr = R.c[i].x, ci = R.c[i].y;
      split_store2(st + 2 * OP_BYTES, st + 3 * OP_BYTES, tile_off(j, 2 * kk), cr, -ci);
      split_store2(st + 2 * OP_BYTES, st + 3 * OP_BYTES, tile_off(j + 64, 2 * kk), ci, cr);
    }
  };
  float acc[64];
  const bool ok = tc_mainloop<Regs>(S, tmem, nchunks, acc, load, store);
  if (!ok && tid == 0) {
    status[0] = -6;   // ACE_ERR_TIMEOUT
    status[1] = -2;
  }
  const int w = tid >> 5, lane = tid & 31;
  const long long g = g0 + 32 * (w & 3) + lane;
  const int part_ri = w >> 2;
  if (ok && g < ng) {
#pragma unroll
    for (int j = 0; j < 64; ++j)
      if (b0 + j < nb) Out[2 * ((long long)(b0 + j) * ld + g) + part_ri] = (float)alpha * acc[j];
  }
  tc_teardown(S, tmem);
}

// Exact diagonal of the gram product: Mc[a][a] = (scale Re sum_g conj(A_a) B_a, 0),
// FP32 products summed in FP32 over short runs and in FP64 across them.
// Grid: (na, kDiagSplits); part: FP64 [na][kDiagSplits].
constexpr int kDiagSplits = 32;
__global__ void __launch_bounds__(256)
diag_dot_kernel(const float2* __restrict__ A, const float2* __restrict__ B, long long ld, long long ng,
                double* __restrict__ part) {
  __shared__ double red[8];
  const int a = blockIdx.x;
  const long long per = (ng + kDiagSplits - 1) / kDiagSplits;
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

__global__ void diag_fix_kernel(const double* __restrict__ part, int na, double scale, double* __restrict__ Mc) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= na) return;
  double t = 0.0;
  for (int k = 0; k < kDiagSplits; ++k) t += part[(long long)a * kDiagSplits + k];
  Mc[2 * ((long long)a * na + a)] = scale * t;
  Mc[2 * ((long long)a * na + a) + 1] = 0.0;
}

}  // namespace

bool tc_gemm_prepare() {
  cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  cudaFuncSetAttribute(outer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  return cudaGetLastError() == cudaSuccess;
}

int gram_tc_splits(long long ng, int na, int nb) {
  const long long tiles = (long long)((na + TM - 1) / TM) * ((nb + 63) / 64);
  long long s = 152 / tiles;   // one wave of one CTA per SM (132 KB of shared memory each)
  const long long max_s = (ng + KC / 2 - 1) / (KC / 2);
  if (s > max_s) s = max_s;
  if (s < 1) s = 1;
  return (int)s;
}

void launch_gram_tc(const void* A, int na, const void* B, int nb, long long ld, long long ng, double* part,
                    int splits, int* status, cudaStream_t st) {
  long long chunk = (ng + splits - 1) / splits;
  chunk = (chunk + KC / 2 - 1) / (KC / 2) * (KC / 2);
  const dim3 grid((na + TM - 1) / TM, (nb + 63) / 64, splits);
  gram_tc_kernel<<<grid, 256, SMEM_BYTES, st>>>(static_cast<const float2*>(A), na, static_cast<const float2*>(B), nb,
                                                ld, ng, part, chunk, status);
}

void launch_outer_tc(const void* A, int nk, const double* C, int nb, long long ld, long long ng, double alpha,
                     void* Out, int* status, cudaStream_t st) {
  const dim3 grid((nb + 63) / 64, (unsigned)((ng + TM - 1) / TM));
  outer_tc_kernel<<<grid, 256, SMEM_BYTES, st>>>(static_cast<const float2*>(A), nk, C, nb, ld, ng, alpha,
                                                 static_cast<float*>(Out), status);
}

size_t diag_dot_part_doubles(int na) { return (size_t)na * kDiagSplits; }

void launch_diag_exact(const void* A, const void* B, int na, long long ld, long long ng, double scale,
                       double* part, double* Mc, cudaStream_t st) {
  diag_dot_kernel<<<dim3(na, kDiagSplits), 256, 0, st>>>(static_cast<const float2*>(A),
                                                         static_cast<const float2*>(B), ld, ng, part);
  diag_fix_kernel<<<(na + 127) / 128, 128, 0, st>>>(part, na, scale, Mc);
}

}  // namespace ace
