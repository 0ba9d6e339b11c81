// Internal declarations shared by the host API and the kernel translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace ace {

constexpr int kMaxTiles = 64;   // pair tiles per batch (one kernel launch covers a batch)
constexpr int kTileMax = 8;     // orbitals per tile side (register accumulators in pass D)

// One tile of pair solves.
//  kind 0: off-diagonal symmetric tile, pairs (l, r) for l in [l0, l0+nl), r in [r0, r0+nr);
//          each pair feeds W_r (through conj(phi_l) phi_r) and W_l (through the conjugate).
//  kind 1: diagonal symmetric tile (l0 == r0, nl == nr), pairs l <= r.
//  kind 2: rectangular one-sided tile, pairs (l, r) feed Out_r only (V_X[Phi] Psi).
// Pair q of a tile lives in slot slot0 + q of the batch's spectrum scratch;
// the order is row-major over (l, r) (upper triangle for kind 1).
struct TileDesc {
  int l0, nl, r0, nr, kind, slot0;
};
struct Batch {
  int ntiles;
  int npairs;
  TileDesc t[kMaxTiles];
};

__host__ __device__ inline int tile_pairs(const TileDesc& d) {
  return d.kind == 1 ? d.nl * (d.nl + 1) / 2 : d.nl * d.nr;
}
// Scratch slots of a tile. Complex vectors: one per pair. Real vectors: two
// pairs (l, r), (l, r + 1) per slot, as the real and imaginary parts of one
// complex solve (the kernel is real and even, so the two stay apart); on a
// diagonal tile each row's pair (l, l) has a slot of its own, so that every
// slot's pairs carry the same energy weight. Diagonal tile of n orbitals:
// n + floor(n^2 / 4) slots; other tiles n_l ceil(n_r / 2).
__host__ __device__ inline int tile_slots(const TileDesc& d, bool real) {
  if (!real) return tile_pairs(d);
  return d.kind == 1 ? d.nl + d.nl * d.nl / 4 : d.nl * ((d.nr + 1) / 2);
}

// Launchers (pair_f32.cu / pair_f64.cu). Return false if edge n is not compiled.
struct PairLaunch {
  int nx, ny, nz;        // grid points along x, y, z
  long long ld;          // elements from one vector to the next (>= n_x n_y n_z)
  const void* X;         // l-side vectors (phi)
  const void* Y;         // r-side vectors (phi or psi)
  void* OutX;            // accumulators for the l side (symmetric tiles)
  void* OutY;            // accumulators for the r side
  void* S;               // spectrum scratch, max_pairs * N_g complex
  const void* Kt;        // kernel table K(G) alpha / N_g, folded [kz][kx][ky] over 0..n/2 per axis
  double* Epart;         // per-block energy partials (nullable)
  double scale;          // Out -= scale * sum
  const double* twx;     // host FP64 twiddles exp(-2 pi i k/n) per axis, 2n doubles each
  const double* twy;
  const double* twz;
  bool real_io;          // R64 vectors
  int mode;              // 0: W / Y accumulate; 1: energy only; 2: energy + accumulate
  cudaEvent_t* ev;       // nullable: 5 events recorded around passes A, B, C, D
  bool prepare_only;     // set kernel attributes for edge n, launch nothing
  const TileDesc* dtiles;  // device copy of the batch's tile descriptors
  bool no_pdl;           // launch the passes without programmatic dependent launch
  int pass_mask;         // passes to launch: bit 0 A, 1 B, 2 C, 3 D (0 = all)
  int radix;             // line-transform radix order: 0 radix 4 first, 1 odd radix first (FP32)
};
// Persistent engine counters: a queue head and one completion counter per
// (batch, pass), each on its own 128-byte line so that polling blocks do not
// contend with the atomics of the producers.
constexpr int kCtrStride = 32;   // unsigned ints between counters
inline size_t engine_ctr_bytes(long long nbatches) { return 128 + (size_t)512 * (size_t)nbatches; }

// Persistent engine: per-batch task table and launch description.
struct EngineBatch {
  int toff, ntiles, npairs, pad;
  long long task0;   // first global task of the batch
  int n[4];          // tasks of passes A, B, C, D (C, D zero in energy-only tables)
};
struct EngineInfo {
  size_t smem = 0;
  int threads = 0;
  int blocks = 0;    // co-resident blocks on the device (0: the engine does not fit)
};
// A persistent-engine wait gives up after this many polls (each sleeps >= 256
// ns: about a second or more) unless a plan sets another limit.
constexpr unsigned kEngineSpinDefault = 1u << 22;
struct EngineLaunch {
  unsigned spin_limit = kEngineSpinDefault;   // polls before a dependent wait gives up
  unsigned wait_bias = 0;                     // added to every awaited count (test hook)
  const TileDesc* dtiles;
  const EngineBatch* batches;
  int nbatches;
  long long ntasks;
  unsigned long long* head;
  unsigned* done;
  int* status;
  long long blocks;
  size_t smem;
};
bool engine_prepare_f32(int n, EngineInfo& info);
bool engine_prepare_f64(int n, EngineInfo& info);
bool engine_tasks_f32(int n, const Batch& b, int nt[4]);
bool engine_tasks_f64(int n, const Batch& b, int nt[4]);
bool launch_engine_f32(const PairLaunch& L, const EngineLaunch& E, cudaStream_t st);
bool launch_engine_f64(const PairLaunch& L, const EngineLaunch& E, cudaStream_t st);

bool launch_pair_batch_f32(const PairLaunch& L, const Batch& b, cudaStream_t st);
bool launch_pair_batch_f64(const PairLaunch& L, const Batch& b, cudaStream_t st);
// The grid's plane (n_x, n_y) and pencil length n_z are compiled in.
bool pair_grid_supported(bool f64, int nx, int ny, int nz);
// Energy partials one pair batch of npairs writes (one per pass-B block).
int energy_blocks(int nx, int ny, int nz, int npairs);

// Dense kernels (dense.cu).
void launch_gram(bool f64, bool real_in, const void* A, int na, const void* B, int nb, long long ld,
                 long long ng, double* part, int splits, cudaStream_t st);
int gram_splits(long long ng, int na, int nb);
int launch_gram_reduce(const double* part, int splits, int na, int nb, double scale, bool hermitize,
                       bool real_out, double* out, double* out_trace_half, cudaStream_t st);
void launch_outer(bool f64, bool real_io, const void* A, int nk, const double* C, int nb,
                  long long ld, long long ng, double alpha, void* Out, cudaStream_t st);
// M_out (n x n) and Ex_out = 1/2 Re of the first n_trace diagonal entries (all if < 0).
int launch_m_outputs(const double* Mc, int n, bool real, double* M_out, double* Ex_out, cudaStream_t st,
                     int n_trace = -1);
// Tensor-core GEMMs for complex FP32 with the 3-term split (tc_gemm.cu):
// tcgen05 kind::tf32, or kind::f16 with BF16 operands when bf16 is set.
bool tc_gemm_prepare();
int gram_tc_splits(long long ng, int na, int nb);
void launch_gram_tc(const void* A, int na, const void* B, int nb, long long ld, long long ng, double* part,
                    int splits, int* status, cudaStream_t st, bool bf16 = false);
// launch_outer_tc: C is complex FP64 [nk][nb]; c32 is scratch for its FP32
// copy (nk * nb * 8 bytes), made once per call.
void launch_outer_tc(const void* A, int nk, const double* C, int nb, long long ld, long long ng, double alpha,
                     void* Out, void* c32, int* status, cudaStream_t st, bool bf16 = false);
// Xi = W L^{-*} with FP64 arithmetic from complex FP32 W (dense.cu): C upper
// triangular FP64 [nk][nb]; Out complex FP32 or FP64 [nb][ld].
void launch_outer_f64acc(const void* A, int nk, const double* C, int nb, long long ld, long long ng, void* Out,
                         bool out_f64, cudaStream_t st);
// The same product to FP64 accuracy on the FP16 tensor cores (xi_oz.cu), with
// `scratch` of xi_oz_scratch_bytes(); returns the kernel count.
bool xi_oz_prepare();
size_t xi_oz_scratch_bytes(long long ng, int nk, int nb, bool out_f64);
int launch_xi_oz(const void* A, int nk, const double* C, int nb, long long ld, long long ng, void* Out,
                 bool out_f64, void* scratch, int* status, cudaStream_t st);
// Diagonal of dV A^* B recomputed with FP64 accumulation into Mc (after the
// tensor-core gram): keeps 1/2 tr M = E_x at FP32 accuracy. part: scratch.
size_t diag_dot_part_doubles(int na);
void launch_diag_exact(const void* A, const void* B, int na, long long ld, long long ng, double scale,
                       double* part, double* Mc, cudaStream_t st);
// Blocked FP64 Cholesky of -M and L^{-*}; returns the number of kernels launched.
int launch_cholesky_inv(const double* M, int n, double* work, double* LinvH, int* status,
                        cudaStream_t st);
size_t cholesky_work_doubles(int n);
void prepare_cholesky(int n);
// X *= s over the first ng elements of each of `count` vectors (stride ld).
void launch_scale(bool f64, bool real, void* X, long long count, long long ng, long long ld, double s,
                  cudaStream_t st);
void launch_energy_reduce(const double* part, int count, double factor, double* out, cudaStream_t st);
void launch_zero(void* p, size_t bytes, cudaStream_t st);
// count values (reals) uniform in [-1, 1) from a hash of (seed, index).
void launch_fill_random(void* x, long long count, bool f64, unsigned long long seed, cudaStream_t st);

}  // namespace ace
