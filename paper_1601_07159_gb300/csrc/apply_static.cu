// ace_apply_static: the ACE apply (Y = -Xi (dV Xi^* Psi)) without a caller
// workspace, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand over a scratch buffer: a plugin
// whose host application owns every device allocation through its own pool,
// or a fixed-latency loop where an allocation may block. This entry point
// keeps the split-K partial sums and the small coefficient matrix C of the
// apply in one file-scope device array instead of the caller's workspace.
//
// The array is loaded with the library and stays resident on every GPU that
// loads it until the process exits. Host code cannot use its name as a device
// address, so the first call on each device (with that device current) looks
// the address up with cudaGetSymbolAddress; make that first call before any
// stream capture. Every call on a device shares the one array: calls that
// overlap on the GPU (different streams, or different plans) race on it and
// must be serialised by the caller. Nothing in it needs clearing between
// calls: each call writes every partial sum and every entry of C it reads.
#include <mutex>
#include <string>

#include "../../include/ace.h"
#include "ace_internal.h"

namespace {

__device__ __align__(256) unsigned char g_apply_scratch[ACE_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

}  // namespace

// Accessors the plan layer uses (defined in ace_api.cu).
ace_status ace_internal_plan_info(const ace_plan* p, int* device, int* n_occ, long long* ng, long long* ld,
                                  double* dv, int* f64, int* real);
ace_status ace_internal_set_error(ace_status s, const char* msg);

extern "C" ace_status ace_apply_static(ace_plan* p, const void* Xi, const void* Psi, int nb, void* Y,
                                       void* stream) {
  int device = 0, N = 0, f64 = 0, real = 0;
  long long ng = 0, ld = 0;
  double dv = 0.0;
  if (!p) return ace_internal_set_error(ACE_ERR_ARG, "plan is NULL");
  ace_internal_plan_info(p, &device, &N, &ng, &ld, &dv, &f64, &real);
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != device)
    return ace_internal_set_error(ACE_ERR_ARG, "current device differs from the plan's device");
  if (cur < 0 || cur >= kMaxDevices) return ace_internal_set_error(ACE_ERR_ARG, "device index out of range");
  if (nb < 0) return ace_internal_set_error(ACE_ERR_ARG, "n_b must be >= 0");
  if (nb == 0) return ACE_OK;
  if (!Xi || !Psi || !Y) return ace_internal_set_error(ACE_ERR_ARG, "NULL vector pointer");
  if (((uintptr_t)Xi | (uintptr_t)Psi | (uintptr_t)Y) & 15u)
    return ace_internal_set_error(ACE_ERR_ARG, "vectors must be 16-byte aligned");
  if (Y == Xi || Y == Psi) return ace_internal_set_error(ACE_ERR_ARG, "Y must not alias Xi or Psi");
  // scratch: `splits` partial N x nb complex FP64 matrices plus C itself
  const size_t mat = (size_t)N * (size_t)nb * 2 * sizeof(double);
  const size_t fit = ACE_STATIC_SCRATCH_BYTES / mat;
  if (fit < 2)
    return ace_internal_set_error(
        ACE_ERR_ARG, ("n_occ * n_b = " + std::to_string((long long)N * nb) +
                      " exceeds the static scratch (max " +
                      std::to_string(ACE_STATIC_SCRATCH_BYTES / (4 * sizeof(double))) + ")").c_str());
  int splits = ace::gram_splits(ng, N, nb);
  if ((size_t)splits > fit - 1) splits = (int)(fit - 1);

  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[cur]) {
      const cudaError_t e = cudaGetSymbolAddress(&g_addr[cur], g_apply_scratch);
      if (e != cudaSuccess) {
        g_addr[cur] = nullptr;
        return ace_internal_set_error(ACE_ERR_CUDA, (std::string("cudaGetSymbolAddress: ") +
                                                     cudaGetErrorString(e)).c_str());
      }
    }
    base = g_addr[cur];
  }
  double* part = static_cast<double*>(base);
  double* Cm = part + (size_t)splits * N * nb * 2;
  cudaStream_t st = (cudaStream_t)stream;
  ace::launch_gram(f64 != 0, real != 0, Xi, N, Psi, nb, ld, ng, part, splits, st);
  ace::launch_gram_reduce(part, splits, N, nb, dv, false, false, Cm, nullptr, st);
  ace::launch_outer(f64 != 0, real != 0, Xi, N, Cm, nb, ld, ng, -1.0, Y, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return ace_internal_set_error(ACE_ERR_CUDA, (std::string("ace_apply_static: ") + cudaGetErrorString(e)).c_str());
  return ACE_OK;
}
