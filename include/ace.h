/*
 * ace.h -- C ABI of the GB300 (sm_103a) adaptively compressed exchange path.
 *
 * Method: L. Lin, "Adaptively Compressed Exchange Operator" (arXiv:1601.07159).
 *   Eq. applyVX / applyVX2 : (V_X[phi] psi)(r) = -sum_j phi_j(r) int phi_j(r') psi(r') K(r-r') dr'
 *   Eq. W                  : W_i = V_X[phi] phi_i
 *   Eq. ACEconstruct2      : M_kl = <phi_k, W_l>,  -M = L L^*   (Sec. 3, Cholesky step)
 *   Eq. Wtilde             : Xi = W L^{-*}
 *   Eq. ACE                : V_ACE psi = -Xi (Xi^* psi)
 *   Eq. EX / EX_ACE        : E_x = -1/2 sum_ij (rho_ij | K | rho_ij) = 1/2 Re tr M
 *   Eq. EXSR               : screened kernel erfc(omega r)/r
 *
 * Discretisation (all entry points): a periodic orthorhombic cell L[0] x L[1] x
 * L[2] sampled on n[0] x n[1] x n[2] points; dV = Omega / N_g. Inner products are
 * <f, g> = dV sum_r conj(f(r)) g(r). The Poisson-type solve is
 *   v(r) = sum_G K(G) rho_hat(G) e^{iG.r},  rho_hat(G) = N_g^-1 sum_r rho(r) e^{-iG.r},
 * with K(G) = alpha * 4 pi/|G|^2 (ACE_KERNEL_BARE, K(0) = 0 by default) or
 * alpha * (4 pi/|G|^2)(1 - exp(-|G|^2 / 4 omega^2)) (ACE_KERNEL_ERFC, K(0) =
 * alpha * pi / omega^2 by default). ACE_KERNEL_KINETIC, K(G) = alpha |G|^2 / 2,
 * is not an exchange kernel: with it, ace_poisson applies the kinetic-energy
 * operator -1/2 Laplacian (spectrally) to its vectors, the T of Eq. HF, so a
 * model Hamiltonian can be applied with this library's FFT passes alone.
 * Complex orbitals use the Hermitian form
 * V_X(r, r') = -sum_j phi_j(r) conj(phi_j(r')) K(r - r').
 *
 * Conventions shared by every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller. Layout is
 *    orbital-major, x fastest: element (b, z, y, x) of an array of `count`
 *    vectors is at offset b * ld + (z * n[1] + y) * n[0] + x elements (ld =
 *    the plan's leading dimension, N_g by default). Storage type is
 *    the plan's dtype: ACE_DTYPE_R64 (double, real Gamma-point orbitals),
 *    ACE_DTYPE_C128 (interleaved double complex) or ACE_DTYPE_C64 (interleaved
 *    float complex). Pointers must be 16-byte aligned.
 *  - Work runs asynchronously on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream) on the current device, which must be the plan's device.
 *    The return code reports host-side validation and launch errors only;
 *    device-side failures (non-positive Cholesky pivot, non-finite pivot) are
 *    recorded in the plan's status word, read by ace_status_sync.
 *  - The library does not allocate on these calls: scratch memory is the
 *    caller's `ws` of at least ace_workspace_size() bytes (256-byte aligned).
 *  - A plan may be used by one stream at a time. Errors never throw across the
 *    ABI; ace_last_error() returns the calling thread's last message.
 */
#ifndef ACE_H
#define ACE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ACE_OK = 0,
  ACE_ERR_ARG = -1,          /* invalid argument (null pointer, size, alignment) */
  ACE_ERR_NOT_POSDEF = -2,   /* -M not positive definite (device status) */
  ACE_ERR_NONFINITE = -3,    /* NaN / Inf met in the Cholesky pivot (device status) */
  ACE_ERR_WORKSPACE = -4,    /* ws_bytes smaller than ace_workspace_size() */
  ACE_ERR_CUDA = -5,         /* a CUDA runtime call or launch failed */
  ACE_ERR_TIMEOUT = -6,      /* a bounded device wait ran out (device status) */
  ACE_ERR_UNSUPPORTED = -7   /* grid edge / dtype combination not built */
} ace_status;

typedef enum { ACE_DTYPE_R64 = 0, ACE_DTYPE_C128 = 1, ACE_DTYPE_C64 = 2 } ace_dtype;
typedef enum { ACE_KERNEL_BARE = 0, ACE_KERNEL_ERFC = 1, ACE_KERNEL_KINETIC = 2 } ace_kernel;
typedef enum {
  ACE_OP_EXCHANGE_APPLY = 0, ACE_OP_BUILD = 1, ACE_OP_APPLY = 2, ACE_OP_ENERGY_GRAD = 3,
  ACE_OP_BUILD_OVERSAMPLED = 4,  /* n_b = N_phi */
  ACE_OP_POISSON = 5,            /* n_b = number of densities */
  ACE_OP_ENERGY_GRAD_STORE = 6   /* ace_exchange_energy_grad with recompute = 0 */
} ace_op;

/* Arithmetic of the dense steps (M = Phi^* W, Xi = W L^{-*}, the apply) for
 * ACE_DTYPE_C64 plans; FP64 plans (R64, C128) compute everything in FP64 on
 * CUDA cores and accept ACE_PREC_DEFAULT only. The Cholesky factor and
 * L^{-1} are FP64 in every mode.
 *  ACE_PREC_SPLIT_TF32: tcgen05 TF32 tensor cores for all three products, each
 *    FP32 operand split into two TF32 terms, three products (FP32 accuracy).
 *  ACE_PREC_XI_FP64 (the C64 default, ACE_PREC_DEFAULT): as SPLIT_TF32, except
 *    Xi = W L^{-*}, which is computed to FP64 accuracy from the FP32 W and the
 *    FP64 L^{-*} on the FP16 tensor cores (error-free 8-bit integer slices of
 *    both operands, exact integer products, exact accumulation) and rounded
 *    once to FP32: before that rounding the error of Xi_b(g) is below about
 *    2^-41 max_k |W_k(g)| sum_k |(L^{-*})_kb|.
 *  ACE_PREC_XI_FP64_SIMT: the same Xi with plain FP64 arithmetic on CUDA cores.
 *  ACE_PREC_FP32: all three products in FP32 on CUDA cores.
 *  ACE_PREC_SPLIT_BF16: M = dV Phi^* W and the apply's two products on tcgen05
 *    BF16 tensor cores, each FP32 operand split into two BF16 terms (hi = the
 *    operand rounded to BF16, lo = the remainder rounded to BF16), three
 *    products accumulated in FP32: about 16 significant bits per operand, so
 *    these products carry relative errors near 2^-16 per term (the diagonal of
 *    M, and so E_x, is still summed from FP32 products); Xi as ACE_PREC_XI_FP64. */
typedef enum {
  ACE_PREC_DEFAULT = 0,
  ACE_PREC_SPLIT_TF32 = 1,
  ACE_PREC_FP32 = 2,
  ACE_PREC_XI_FP64 = 3,
  ACE_PREC_XI_FP64_SIMT = 4,
  ACE_PREC_SPLIT_BF16 = 5
} ace_prec;

typedef struct {
  int n[3];          /* grid points along x, y, z (N_g = n[0] n[1] n[2]); see ace_supported_grid */
  double L[3];       /* cell edges Lx, Ly, Lz (bohr), > 0 */
  int n_occ;         /* N: number of exchange orbitals phi, 1..1024 */
  int dtype;         /* ace_dtype. R64/C128: FP64 throughout. C64: FP32 pair/FFT path,
                        dense steps per `prec`, FP64 Cholesky and triangular inverse. */
  int prec;          /* ace_prec (0 = default) */
  int kernel;        /* ace_kernel */
  double omega;      /* screening parameter (bohr^-1) for ACE_KERNEL_ERFC, > 0 */
  double g0_value;   /* K(G=0) before alpha; NaN selects the default (0 bare and kinetic,
                        pi/omega^2 erfc) */
  double alpha;      /* overall kernel scale (1 = Hartree-Fock; 0.25 for PBE0/HSE fractions) */
  long long ld;      /* elements from one vector to the next in every vector array the
                        plan's calls take (Phi, Psi, W, Xi, Y, gradients, densities):
                        0 = N_g (packed), else >= N_g and even; elements between N_g
                        and ld are neither read nor written */
  int max_pairs;     /* complex solves (scratch slots of N_g points) in flight per batch
                        (0 = library default); sets the size of the pair-spectrum
                        scratch in the workspace. A slot holds one pair for complex
                        vectors, two for ACE_DTYPE_R64 (real and imaginary parts) */
  int tile;          /* orbitals per pair tile, 1..8 (0 = default 8) */
  int lanes;         /* concurrent batch streams inside one call with
                        ACE_FLAG_NO_OVERLAP, 1..8 (0 = default 2; at least 2
                        otherwise); the pair scratch is lanes * max_pairs slots */
  int flags;         /* ACE_FLAG_* */
} ace_desc;

/* Launch each pair batch eagerly instead of replaying a captured CUDA graph
 * (graphs are keyed by the call's pointers; see ace_build). */
#define ACE_FLAG_NO_GRAPH 1
/* Run the pair solves as one persistent cooperative launch per call (blocks
 * take pass tasks from an ordered queue and wait, with a bounded spin, on
 * per-batch completion counters) instead of the default four kernels per
 * batch (passes A-D chained by programmatic dependent launch). A wait that runs
 * out (about a second) leaves ACE_ERR_TIMEOUT in the status word. Cubic grids
 * only (FP64: edges up to 48); elsewhere the flag is ignored. */
#define ACE_FLAG_ENGINE 2
/* Launch the four pass kernels without programmatic dependent launch (a
 * tuning and diagnosis switch). With ACE_FLAG_NO_GRAPH and without
 * ACE_FLAG_ENGINE, ace_profile_end reports per-pass times. */
#define ACE_FLAG_NO_PDL 4
/* ACE_DTYPE_C64: the same as prec = ACE_PREC_FP32 (M, Xi and the apply in FP32
 * on CUDA cores). */
#define ACE_FLAG_SIMT_GEMM 8
/* By default, graph mode issues pass A of every pair batch on one stream and
 * passes B-D on a second, so that pass A of batch k+1 (which waits for pass C of
 * batch k) overlaps pass D of batch k; the scratch holds two batches (lanes is
 * raised to at least 2). This flag turns that off: the batches of a round are
 * then spread over `lanes` streams instead. Results are bitwise the same. */
#define ACE_FLAG_NO_OVERLAP 16
/* Radix order of the line transforms (ACE_DTYPE_C64 plans): by default a
 * transform of length n takes a radix 4 first, then 2, 3, 5; with this flag it
 * takes the odd radix (3, then 5) first, for the lengths where the orders
 * differ (those with a factor 3 or 5 beside a power of two: 12, 20, 24, 36,
 * 40, 48, 96). Results agree to FP32 rounding. A schedule choice of
 * ace_autotune; ignored by FP64 plans and by ACE_FLAG_ENGINE. */
#define ACE_FLAG_RADIX_ODD_FIRST 32

typedef struct ace_plan ace_plan;

/* Nonzero when grid edge n is compiled in for the dtype (register-resident FFT
 * lengths; radices 2, 3, 4, 5). */
int ace_supported_edge(int n, int dtype);

/* Nonzero when the n[0] x n[1] x n[2] grid is compiled in for the dtype: its
 * plane n[0] x n[1] (every square plane of a compiled edge, plus the listed
 * non-square planes 12x16, 16x12, 16x24, 24x16, 40x48, 48x40) and its pencil
 * length n[2] (any compiled edge). Compiled edges: 8, 12, 16, 20, 24, 32, 36,
 * 40, 48, 64, 96 for every dtype. */
int ace_supported_grid(const int n[3], int dtype);

/* Validate *desc and build a plan on the current device: Coulomb kernel table,
 * FFT twiddles (FP64 host sin/cos), the pair-tile schedule and small FP64 N x N
 * buffers. Returns ACE_ERR_ARG / ACE_ERR_UNSUPPORTED / ACE_ERR_CUDA on failure
 * and leaves *out NULL. Allocates; not for the hot path. */
ace_status ace_plan_create(const ace_desc* desc, ace_plan** out);

/* Free a plan and its device buffers (synchronises the device). NULL is a no-op. */
ace_status ace_plan_destroy(ace_plan* plan);

/* Bytes of scratch `ws` the entry point `op` needs for n_b target vectors
 * (N_phi for ACE_OP_BUILD_OVERSAMPLED; ignored for ACE_OP_BUILD /
 * ACE_OP_ENERGY_GRAD). 0 on invalid input. */
size_t ace_workspace_size(const ace_plan* plan, int op, int n_b);

/* Y = V_X[Phi] Psi (Eq. applyVX2): N x n_b pair solves, no pair symmetry.
 * Phi: N vectors, Psi: n_b vectors, Y: n_b vectors (overwritten). Y must not
 * alias Phi or Psi. */
ace_status ace_exchange_apply(ace_plan* plan, const void* Phi, const void* Psi, int n_b,
                              void* Y, void* ws, size_t ws_bytes, void* stream);

/* Graphs: ace_exchange_apply, ace_build and ace_exchange_energy_grad record the
 * kernels of their pair-solve section into a CUDA graph on first use with a
 * given set of pointers (and n_b), keep up to 8 such graphs per plan, and
 * replay them on later calls with the same pointers; a call with new pointers
 * captures a new graph (a few milliseconds, on a plan-owned stream). The
 * graph is launched on `stream`, so ordering with the caller's work is kept.
 *
 * ACE construction (Alg. 2, steps 2-3): W = V_X[Phi] Phi with N(N+1)/2 unique
 * pair solves (v_ij = conj(v_ji) halves the work), M = dV Phi^* W made
 * Hermitian, -M = L L^* (FP64), Xi = W L^{-*}.
 * Phi: N vectors (orthonormal in <.,.> for Eq. ACEcond to hold, not checked).
 * W_out: N vectors or NULL. Xi_out: N vectors (required).
 * M_out: NULL or device double[N*N] (R64) / double[2*N*N] (complex, interleaved),
 *        row-major M[k][l].
 * Ex_out: NULL or device double[1] = 1/2 Re tr M (Eq. EX_ACE with psi = phi).
 * A non-positive pivot stops the factorisation and is reported through
 * ace_status_sync (ACE_ERR_NOT_POSDEF, info = 1-based pivot); Xi is then undefined. */
ace_status ace_build(ace_plan* plan, const void* Phi, void* W_out, void* Xi_out,
                     double* M_out, double* Ex_out, void* ws, size_t ws_bytes, void* stream);

/* ACE construction with oversampling (Sec. 3, oversampling ratio
 * r = N_phi / N_e > 1): V_X is the exchange operator of the plan's N_e = n_occ
 * occupied orbitals Phi[0..N_e), and W_i = V_X Phi_i for all N_phi orbitals
 * (the N_e(N_e+1)/2 unique occupied pairs, then N_e (N_phi - N_e) one-sided
 * pairs); M = dV Phi^* W (N_phi x N_phi, Hermitian part), -M = L L^* in FP64,
 * Xi = W L^{-*} (N_phi vectors), so that V_ACE = -Xi Xi^* dV agrees with V_X on
 * span{Phi_0..Phi_{N_phi-1}}. Ex_out = 1/2 Re tr of the occupied block of M.
 * Phi: N_phi vectors, the occupied ones first. W_out: N_phi vectors or NULL;
 * Xi_out: N_phi vectors; M_out: NULL or N_phi x N_phi as in ace_build.
 * n_occ <= N_phi <= 1024; N_phi = n_occ gives ace_build's results.
 * ws: ace_workspace_size(plan, ACE_OP_BUILD_OVERSAMPLED, N_phi) bytes. */
ace_status ace_build_oversampled(ace_plan* plan, const void* Phi, int n_phi, void* W_out, void* Xi_out,
                                 double* M_out, double* Ex_out, void* ws, size_t ws_bytes, void* stream);

/* Periodic Poisson solves through the pair passes: V_b(r) = sum_G K(G)
 * rho_hat_b(G) e^{iG.r} (rho_hat = N_g^-1 sum_r rho e^{-iG.r}) with the plan's
 * kernel table (alpha K, K(0) = g0). With the bare kernel and rho the electron
 * density sum_i |psi_i|^2 this is the Hartree potential V_H[rho] of Eq. HF
 * (K(0) = 0: neutralising background). rho, V: n_b vectors of the plan's
 * layout and dtype (real densities in R64 plans), V must not alias rho.
 * ws: ace_workspace_size(plan, ACE_OP_POISSON, n_b) bytes. */
ace_status ace_poisson(ace_plan* plan, const void* rho, int n_b, void* V, void* ws, size_t ws_bytes,
                       void* stream);

/* Batched ACE construction: ace_build for n_sys independent systems (each with
 * its own plan: grid edge, N, dtype and kernel may all differ) issued as ONE
 * captured CUDA graph. The systems are spread over `chains` concurrent
 * streams (0 = 3), longest first, each to the chain with the least estimated
 * work (N(N+1)/2 N_g); inside a chain they run in turn, each with its own
 * two-stream pair schedule. The graph is cached process-wide under all the
 * pointers (plans, Phi[i], Xi[i], Ex, ws) and replayed on later calls.
 * plans: n_sys distinct plans on the current device. Phi[i], Xi[i]: N_i
 * vectors of plan i's layout (device, 16-byte aligned). Ex: NULL or device
 * double[n_sys], Ex[i] = 1/2 Re tr M_i. W is kept in the workspace only.
 * ws: ace_workspace_size_batched(plans, n_sys) bytes, 256-byte aligned.
 * Device-side failures land in each plan's status word (ace_status_sync). */
size_t ace_workspace_size_batched(ace_plan* const* plans, int n_sys);
ace_status ace_build_batched(ace_plan* const* plans, const void* const* Phi, void* const* Xi,
                             double* Ex, int n_sys, int chains, void* ws, size_t ws_bytes,
                             void* stream);

/* Autotuner (schedule choice only; results are the same for every choice up
 * to FP32 rounding order): times ace_build of the descriptor's problem on the
 * current device for each candidate schedule -- tile edge 8, 6 or 4 orbitals,
 * pair-batch scratch of about 36, 72 or 144 MiB, the two-stream overlapped
 * pair schedule or two lanes without overlap, and (C64 plans) the radix order
 * of the line transforms (ACE_FLAG_RADIX_ODD_FIRST) -- on seeded pseudo-random
 * orbitals, `reps` timed builds each (0 = 3) after one untimed build, and
 * writes the fastest into *best (a copy of *d with tile, max_pairs, lanes and
 * flags set) and its milliseconds per build into *ms_out (nullable), and
 * registers it for later plans of the same problem (ace_tuning_register).
 * Allocates its own device buffers (about 2 N N_g vectors plus the largest
 * workspace) and synchronises; call it outside timed or captured regions. */
ace_status ace_autotune(const ace_desc* d, int reps, ace_desc* best, double* ms_out);

/* Tuned schedules, process-wide: ace_autotune registers its result, and
 * ace_tuning_register adds one found earlier (for instance from a saved
 * tuning table); ace_plan_create then takes the registered max_pairs, tile,
 * lanes, ACE_FLAG_NO_OVERLAP and ACE_FLAG_RADIX_ODD_FIRST for a descriptor
 * with the same grid, n_occ,
 * dtype, prec and kernel whose max_pairs, tile and lanes are all 0.
 * ace_tuning_clear forgets every registered schedule. ace_plan_desc writes the
 * plan's effective descriptor (the schedule it runs, the resolved ld). */
ace_status ace_tuning_register(const ace_desc* tuned);
ace_status ace_tuning_clear(void);
ace_status ace_plan_desc(const ace_plan* plan, ace_desc* out);

/* Y = V_ACE Psi = -Xi (dV Xi^* Psi) (Eq. ACE). Xi: N vectors from ace_build,
 * Psi and Y: n_b vectors; Y must not alias Xi or Psi. No Poisson solves. */
ace_status ace_apply(ace_plan* plan, const void* Xi, const void* Psi, int n_b, void* Y,
                     void* ws, size_t ws_bytes, void* stream);

/* E_x[Phi] (Eq. EX, via Parseval: -1/2 sum_ij Omega sum_G K |rho_hat_ij|^2, FP64
 * accumulation) into device Ex_out[0], and the gradient grad_out = grad_scale
 * * 2 dV W (dE/dRe(phi) + i dE/dIm(phi)) when grad_out is non-NULL.
 *
 * recompute != 0: the pair potentials v_ij are formed and consumed batch by
 * batch and never kept: a call without grad_out runs the forward transforms
 * and the energy sum only; a call with grad_out solves every pair once and
 * accumulates the gradient in the same sweep. ws: ACE_OP_ENERGY_GRAD bytes.
 *
 * recompute == 0: the workspace keeps every unique pair potential (N(N+1)/2
 * N_g complex values, ace_workspace_size(plan, ACE_OP_ENERGY_GRAD_STORE, 0)
 * bytes) between two calls. A call without grad_out computes E_x and stores
 * the potentials; a later call with grad_out forms the gradient from the
 * stored potentials alone (the accumulate pass) and, if Ex_out is non-NULL,
 * writes E_x again from the stored energy sums. Between the two calls the
 * caller keeps ws and Phi unchanged and makes no other call with that ws; a
 * gradient call without a preceding energy call on the same ws gives undefined
 * values. The store trades N(N+1)/2 N_g complex values of memory for the
 * second sweep of pair solves; the library never picks it by itself. */
ace_status ace_exchange_energy_grad(ace_plan* plan, const void* Phi, double* Ex_out,
                                    void* grad_out, double grad_scale, int recompute, void* ws,
                                    size_t ws_bytes, void* stream);

/* Synchronise `stream` and read the plan's device status word: returns ACE_OK,
 * ACE_ERR_NOT_POSDEF, ACE_ERR_NONFINITE or ACE_ERR_TIMEOUT; *info (if
 * non-NULL) gets the 1-based Cholesky pivot that failed (the task index or a
 * negative kernel tag for a timeout), 0 otherwise. Clears the status. */
ace_status ace_status_sync(ace_plan* plan, void* stream, int* info);

/* Instrumentation (no counterpart in the paper; for benchmarks and profiles).
 * ace_profile_begin: create `max_events` CUDA events (allocates; call outside
 * timed or captured regions) and from now on record one event before each pair
 * pass launch and one after the batch, so pass durations can be summed; resets
 * the kernel-launch counter. Recording stops silently when the events run out.
 * ace_profile_end: synchronise the device, then write ms_out[0..4] = total
 * milliseconds of pass A (pair product + xy FFT), pass B (z FFT, kernel, inverse
 * z FFT), pass C (inverse xy FFT), pass D (accumulate) and their sum over the
 * recorded batches, and counts_out[0..2] = recorded batches, kernel launches by
 * this plan since ace_profile_begin, batches not recorded; frees the events.
 * Either output may be NULL. */
ace_status ace_profile_begin(ace_plan* plan, int max_events);
ace_status ace_profile_end(ace_plan* plan, double* ms_out, long long* counts_out);

/* Size of the device array behind ace_apply_static (bytes, per GPU). */
#define ACE_STATIC_SCRATCH_BYTES (16u << 20)

/* ace_apply_static: the same operation as ace_apply, Y = -Xi (dV Xi^* Psi),
 * for callers that cannot allocate device memory or pass a workspace (for
 * instance a plugin whose host application owns all device memory, or a
 * fixed-latency loop where an allocation could block). The paper has no
 * counterpart; this is a deployment variant of the apply.
 * Its scratch is a file-scope device array of ACE_STATIC_SCRATCH_BYTES that
 * every GPU loading the library keeps until the process exits; it holds
 * 2 * n_occ * n_b complex FP64 values at least, so n_occ * n_b must be at
 * most ACE_STATIC_SCRATCH_BYTES / 32 (524288), else ACE_ERR_ARG and nothing
 * runs. The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make it before any stream
 * capture. All calls on a device share the array: calls that may overlap on
 * the GPU (other streams, other plans) race and must be serialised by the
 * caller. Nothing needs clearing between calls. The GEMMs run on CUDA cores:
 * for FP64 plans the result equals ace_apply's up to the order of the split-K
 * sums; for ACE_DTYPE_C64 plans, whose ace_apply uses the TF32 3-term-split
 * tensor cores, the two agree to the FP32 apply tolerance (about 1e-6
 * relative), not bit for bit. Calls no allocator. */
ace_status ace_apply_static(ace_plan* plan, const void* Xi, const void* Psi, int n_b, void* Y,
                            void* stream);

/* Test and diagnosis hooks (no counterpart in the paper; they exist so that
 * failure handling can be exercised without faulting a GPU).
 *
 * ace_debug_engine_wait: for plans with ACE_FLAG_ENGINE, every wait of the
 * persistent engine on another block's work polls at most `polls` times (0
 * restores the default of 2^22 polls, about a second or more); with
 * `unreachable` nonzero each wait asks for one finished task more than the pass
 * it depends on has, so every dependent wait runs out. A wait that runs out
 * records ACE_ERR_TIMEOUT (info = the task index) in the plan's status word,
 * and the launch ends: blocks stop taking tasks and return, nothing of theirs
 * in flight. Outputs of that call are then undefined. Drops the plan's cached
 * graphs. Returns ACE_ERR_ARG for a NULL plan.
 *
 * ace_debug_fail_alloc: from now on, the k-th device allocation the library
 * makes (plan set-up, one-sided schedule uploads, ace_autotune's buffers)
 * fails as if the device were out of memory, so the calling entry point
 * returns ACE_ERR_CUDA after releasing what it had allocated; k <= 0 turns the
 * hook off. Returns the number of library allocations counted since the
 * previous call. Process-wide; not for concurrent use. */
ace_status ace_debug_engine_wait(ace_plan* plan, unsigned polls, int unreachable);

/* ace_debug_xi_product (ACE_DTYPE_C64 plans): Xi = W L^{-*} (Eq. Wtilde) with
 * the L^{-*} of the plan's last build, written in FP64 (interleaved double
 * complex, N vectors of stride ld) so that the FP64 accuracy of the product
 * itself can be checked: method 1 = the FP16-tensor-core slice product of
 * ACE_PREC_XI_FP64 (deeper slicing for FP64 output), 2 = plain FP64 on CUDA
 * cores. W: N complex FP32 vectors. Method 1 allocates its scratch and
 * synchronises `stream`. */
ace_status ace_debug_xi_product(ace_plan* plan, const void* W, void* Xi_out, int method, void* stream);
long long ace_debug_fail_alloc(long long k);

/* Message for the calling thread's last failed call ("" if none). */
const char* ace_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ACE_H */
