// Grid shape -> compiled instances of the pair passes: plane passes A and C
// per (n_x, n_y) (pair_plane.cu), pass B per n_z (pair_pencil.cu), pass D per
// precision (pair_point.cu), and the persistent engine per cubic edge
// (pair_edge.cu). A grid n_x x n_y x n_z is supported when its plane and its
// pencil length are compiled in.
#include "ace_internal.h"

// Edges (FFT lengths of radices 2, 3, 4, 5): every square plane, every pencil
// length and every cubic engine. build_lib.py reads these lists to decide which
// instances to compile.
#define ACE_EDGES_F32(X) X(8) X(12) X(16) X(20) X(24) X(32) X(36) X(40) X(48) X(64) X(96)
#define ACE_EDGES_F64(X) X(8) X(12) X(16) X(20) X(24) X(32) X(36) X(40) X(48) X(64) X(96)
// Non-square planes (n_x, n_y) compiled beside the square ones.
#define ACE_PLANES_F32(X) X(12, 16) X(16, 12) X(16, 24) X(24, 16) X(40, 48) X(48, 40)
#define ACE_PLANES_F64(X) X(12, 16) X(16, 12) X(16, 24) X(24, 16) X(40, 48) X(48, 40)
// FP32 edges and planes also compiled with the odd-radix-first order
// (ACE_RADIX_ORDER = 1): the lengths with a factor 3 or 5 beside a power of
// two, where the two orders differ.
#define ACE_EDGES_F32_R1(X) X(12) X(20) X(24) X(36) X(40) X(48) X(96)
#define ACE_PLANES_F32_R1(X) X(12, 16) X(16, 12) X(16, 24) X(24, 16) X(40, 48) X(48, 40)

namespace ace {

using PlaneFn = bool (*)(const PairLaunch&, const Batch&, int, cudaStream_t);
using PencilFn = bool (*)(const PairLaunch&, const Batch&, cudaStream_t);

#define DECL_SQ(P, E)                                                                      \
  bool plane_launch_##P##_##E##_##E(const PairLaunch&, const Batch&, int, cudaStream_t);  \
  bool pencil_launch_##P##_##E(const PairLaunch&, const Batch&, cudaStream_t);            \
  bool point_cube_launch_##P##_##E(const PairLaunch&, const Batch&, cudaStream_t);        \
  void edge_prepare_##P##_##E(EngineInfo&);                                                \
  void edge_tasks_##P##_##E(const Batch&, int nt[4]);                                      \
  bool edge_engine_##P##_##E(const PairLaunch&, const EngineLaunch&, cudaStream_t);
#define DECL_PL(P, X_, Y_) bool plane_launch_##P##_##X_##_##Y_(const PairLaunch&, const Batch&, int, cudaStream_t);
#define DECL_SQ32(E) DECL_SQ(f32, E)
#define DECL_SQ64(E) DECL_SQ(f64, E)
#define DECL_PL32(X_, Y_) DECL_PL(f32, X_, Y_)
#define DECL_PL64(X_, Y_) DECL_PL(f64, X_, Y_)
ACE_EDGES_F32(DECL_SQ32)
ACE_EDGES_F64(DECL_SQ64)
ACE_PLANES_F32(DECL_PL32)
ACE_PLANES_F64(DECL_PL64)
#define DECL_SQ32R1(E)                                                                      \
  bool plane_launch_f32_##E##_##E##_r1(const PairLaunch&, const Batch&, int, cudaStream_t); \
  bool pencil_launch_f32_##E##_r1(const PairLaunch&, const Batch&, cudaStream_t);
#define DECL_PL32R1(X_, Y_) bool plane_launch_f32_##X_##_##Y_##_r1(const PairLaunch&, const Batch&, int, cudaStream_t);
ACE_EDGES_F32_R1(DECL_SQ32R1)
ACE_PLANES_F32_R1(DECL_PL32R1)

bool launch_point_f32(const PairLaunch& L, const Batch& b, cudaStream_t st);
bool launch_point_f64(const PairLaunch& L, const Batch& b, cudaStream_t st);

namespace {

// radix order 1 falls back to order 0 where no such instance is compiled (the
// two orders coincide there)
PlaneFn find_plane(bool f64, int nx, int ny, int radix) {
  if (!f64 && radix == 1) {
#define SQ32R1(E) if (nx == E && ny == E) return plane_launch_f32_##E##_##E##_r1;
#define PL32R1(X_, Y_) if (nx == X_ && ny == Y_) return plane_launch_f32_##X_##_##Y_##_r1;
    ACE_EDGES_F32_R1(SQ32R1)
    ACE_PLANES_F32_R1(PL32R1)
#undef SQ32R1
#undef PL32R1
  }
#define SQ32(E) if (nx == E && ny == E) return plane_launch_f32_##E##_##E;
#define SQ64(E) if (nx == E && ny == E) return plane_launch_f64_##E##_##E;
#define PL32(X_, Y_) if (nx == X_ && ny == Y_) return plane_launch_f32_##X_##_##Y_;
#define PL64(X_, Y_) if (nx == X_ && ny == Y_) return plane_launch_f64_##X_##_##Y_;
  if (f64) {
    ACE_EDGES_F64(SQ64)
    ACE_PLANES_F64(PL64)
  } else {
    ACE_EDGES_F32(SQ32)
    ACE_PLANES_F32(PL32)
  }
#undef SQ32
#undef SQ64
#undef PL32
#undef PL64
  return nullptr;
}

PencilFn find_pencil(bool f64, int nz, int radix) {
  if (!f64 && radix == 1) {
#define PE32R1(E) if (nz == E) return pencil_launch_f32_##E##_r1;
    ACE_EDGES_F32_R1(PE32R1)
#undef PE32R1
  }
#define PE32(E) if (nz == E) return pencil_launch_f32_##E;
#define PE64(E) if (nz == E) return pencil_launch_f64_##E;
  if (f64) {
    ACE_EDGES_F64(PE64)
  } else {
    ACE_EDGES_F32(PE32)
  }
#undef PE32
#undef PE64
  return nullptr;
}

// Pass D for the grid: the cubic instance (N_g compiled in) when there is one.
PencilFn find_point(bool f64, int nx, int ny, int nz) {
  if (nx == ny && ny == nz) {
#define PC32(E) if (nz == E) return point_cube_launch_f32_##E;
#define PC64(E) if (nz == E) return point_cube_launch_f64_##E;
    if (f64) {
      ACE_EDGES_F64(PC64)
    } else {
      ACE_EDGES_F32(PC32)
    }
#undef PC32
#undef PC64
  }
  return f64 ? launch_point_f64 : launch_point_f32;
}

// Passes A-D of one batch (or, with prepare_only, the kernels' attributes),
// with the profiling events around each pass when L.ev is set.
bool launch_batch(bool f64, const PairLaunch& L, const Batch& b, cudaStream_t st) {
  const PlaneFn plane = find_plane(f64, L.nx, L.ny, L.radix);
  const PencilFn pencil = find_pencil(f64, L.nz, L.radix);
  if (!plane || !pencil) return false;
  if (L.prepare_only) return plane(L, b, 0, st) && pencil(L, b, st);
  auto mark = [&](int k) { if (L.ev) cudaEventRecord(L.ev[k], st); };
  const int mask = L.pass_mask ? L.pass_mask : 15;
  bool ok = true;
  mark(0);
  if (mask & 1) ok = ok && plane(L, b, 0, st);
  mark(1);
  if (mask & 2) ok = ok && pencil(L, b, st);
  mark(2);
  if (L.mode == 1) {
    mark(3);
    mark(4);
    return ok;
  }
  if (mask & 4) ok = ok && plane(L, b, 2, st);
  mark(3);
  if (mask & 8) ok = ok && find_point(f64, L.nx, L.ny, L.nz)(L, b, st);
  mark(4);
  return ok;
}

}  // namespace

bool pair_grid_supported(bool f64, int nx, int ny, int nz) {
  return find_plane(f64, nx, ny, 0) != nullptr && find_pencil(f64, nz, 0) != nullptr;
}

bool launch_pair_batch_f32(const PairLaunch& L, const Batch& b, cudaStream_t st) { return launch_batch(false, L, b, st); }
bool launch_pair_batch_f64(const PairLaunch& L, const Batch& b, cudaStream_t st) { return launch_batch(true, L, b, st); }

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
  if (L.nx != L.ny || L.ny != L.nz) return false;
#define CASE(E_) if (L.nx == E_) return edge_engine_f32_##E_(L, E, st);
  ACE_EDGES_F32(CASE)
#undef CASE
  return false;
}
bool launch_engine_f64(const PairLaunch& L, const EngineLaunch& E, cudaStream_t st) {
  if (L.nx != L.ny || L.ny != L.nz) return false;
#define CASE(E_) if (L.nx == E_) return edge_engine_f64_##E_(L, E, st);
  ACE_EDGES_F64(CASE)
#undef CASE
  return false;
}

int energy_blocks(int nx, int ny, int nz, int npairs) {
  // pass B: one energy partial per block (256 pencils; 128 for the two-lane form of
  // n_z >= 64; 32 for the four-warp form of n_z = 64 and 96, counted for either
  // precision)
  const long long pencils = (long long)npairs * nx * ny;
  const int per = (nz == 64 || nz == 96) ? 32 : (nz >= 64 && nz % 4 == 0) ? 128 : 256;
  return (int)((pencils + per - 1) / per);
}

}  // namespace ace
