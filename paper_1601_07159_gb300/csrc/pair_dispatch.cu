// Grid edge -> compiled instance of the pair passes (pair_edge.cu).
#include "ace_internal.h"

// Keep in step with EDGES_F32 / EDGES_F64 in build_lib.py.
#define ACE_EDGES_F32(X) X(8) X(12) X(16) X(20) X(24) X(32) X(36) X(40) X(48) X(64) X(96)
#define ACE_EDGES_F64(X) X(8) X(12) X(16) X(20) X(24) X(32) X(36) X(40) X(48) X(64) X(96)

namespace ace {

#define DECL(P, E)                                                                           \
  bool edge_launch_##P##_##E(const PairLaunch&, const Batch&, cudaStream_t);                \
  void edge_prepare_##P##_##E(EngineInfo&);                                                  \
  void edge_tasks_##P##_##E(const Batch&, int nt[4]);                                        \
  bool edge_engine_##P##_##E(const PairLaunch&, const EngineLaunch&, cudaStream_t);
#define DECL32(E) DECL(f32, E)
#define DECL64(E) DECL(f64, E)
ACE_EDGES_F32(DECL32)
ACE_EDGES_F64(DECL64)

bool pair_edge_supported_f32(int n) {
#define CASE(E) if (n == E) return true;
  ACE_EDGES_F32(CASE)
#undef CASE
  return false;
}
bool pair_edge_supported_f64(int n) {
#define CASE(E) if (n == E) return true;
  ACE_EDGES_F64(CASE)
#undef CASE
  return false;
}
bool launch_pair_batch_f32(const PairLaunch& L, const Batch& b, cudaStream_t st) {
#define CASE(E) if (L.n == E) return edge_launch_f32_##E(L, b, st);
  ACE_EDGES_F32(CASE)
#undef CASE
  return false;
}
bool launch_pair_batch_f64(const PairLaunch& L, const Batch& b, cudaStream_t st) {
#define CASE(E) if (L.n == E) return edge_launch_f64_##E(L, b, st);
  ACE_EDGES_F64(CASE)
#undef CASE
  return false;
}
bool engine_prepare_f32(int n, EngineInfo& info) {
#define CASE(E) if (n == E) { edge_prepare_f32_##E(info); return true; }
  ACE_EDGES_F32(CASE)
#undef CASE
  return false;
}
bool engine_prepare_f64(int n, EngineInfo& info) {
#define CASE(E) if (n == E) { edge_prepare_f64_##E(info); return true; }
  ACE_EDGES_F64(CASE)
#undef CASE
  return false;
}
bool engine_tasks_f32(int n, const Batch& b, int nt[4]) {
#define CASE(E) if (n == E) { edge_tasks_f32_##E(b, nt); return true; }
  ACE_EDGES_F32(CASE)
#undef CASE
  return false;
}
bool engine_tasks_f64(int n, const Batch& b, int nt[4]) {
#define CASE(E) if (n == E) { edge_tasks_f64_##E(b, nt); return true; }
  ACE_EDGES_F64(CASE)
#undef CASE
  return false;
}
bool launch_engine_f32(const PairLaunch& L, const EngineLaunch& E, cudaStream_t st) {
#define CASE(E_) if (L.n == E_) return edge_engine_f32_##E_(L, E, st);
  ACE_EDGES_F32(CASE)
#undef CASE
  return false;
}
bool launch_engine_f64(const PairLaunch& L, const EngineLaunch& E, cudaStream_t st) {
#define CASE(E_) if (L.n == E_) return edge_engine_f64_##E_(L, E, st);
  ACE_EDGES_F64(CASE)
#undef CASE
  return false;
}

int energy_blocks(int n, int npairs, bool f64) {
  (void)f64;
  // pass B: one slot per block (256 pencils; 128 for the two-lane form of n >= 64)
  return (int)(((long long)npairs * n * n + 127) / 128);
}

}  // namespace ace
