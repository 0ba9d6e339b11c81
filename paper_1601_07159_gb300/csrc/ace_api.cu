// C ABI of the ACE hot path: plan creation (kernel table, twiddles, pair-tile
// schedule), workspace sizing, CUDA-graph replay of the pair-solve section and
// the entry points of include/ace.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <deque>
#include <mutex>
#include <limits>
#include <string>
#include <vector>

#include "../../include/ace.h"
#include "ace_internal.h"

using namespace ace;

namespace {

thread_local std::string g_last_error;

// Allocation-failure injection (ace_debug_fail_alloc): when g_fail_at > 0 the
// g_fail_at-th device allocation counted from the hook's last call fails as if
// the device were out of memory.
std::atomic<long long> g_fail_at{0};
std::atomic<long long> g_alloc_count{0};

cudaError_t dev_alloc(void** ptr, size_t bytes) {
  const long long c = ++g_alloc_count;
  if (g_fail_at.load() > 0 && c == g_fail_at.load()) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(ptr, bytes);
}

ace_status fail(ace_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

ace_status cuda_check(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ACE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return ACE_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kMaxLanes = 8;
constexpr int kMaxGraphs = 8;

// Batches in the order they run; batches of one round write disjoint outputs
// and may run concurrently.
struct Schedule {
  std::vector<Batch> batches;
  std::vector<int> round;
  std::vector<int> toff;        // offset of each batch's tiles in dtiles
  TileDesc* dtiles = nullptr;   // device copy of all tile descriptors
  EngineBatch* deng[2] = {nullptr, nullptr};   // engine task tables: [0] Poisson, [1] energy only
  long long ntasks[2] = {0, 0};
  std::vector<long long> soff;  // first pair slot of each batch in a store of all pair potentials
};

void free_schedule(Schedule& sc) {
  cudaFree(sc.dtiles);
  cudaFree(sc.deng[0]);
  cudaFree(sc.deng[1]);
  sc.dtiles = nullptr;
  sc.deng[0] = sc.deng[1] = nullptr;
}

struct GraphEntry {
  uintptr_t key[8] = {};
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
  unsigned long long last_use = 0;
};

struct ProfRec {
  size_t first;   // index of the first event
  int kind;       // 0: 5 events around passes A..D of one batch; 1: 2 events around a section
};

}  // namespace

struct ace_plan {
  ace_desc d{};
  int device = 0;
  int nx = 0, ny = 0, nz = 0;    // grid points along x, y, z
  bool cubic = false;            // nx == ny == nz (the persistent engine needs it)
  long long ng = 0;              // grid points N_g
  long long ld = 0;              // elements from one vector to the next
  int xi = 0;                    // Xi = W L^{-*}: 0 the plan's GEMM, 1 FP16 Ozaki slices, 2 FP64 CUDA cores
  double vol = 0.0, dv = 0.0;
  bool f64 = false, real = false;
  size_t csize = 0;              // bytes per complex scratch element
  size_t vsize = 0;              // bytes per stored vector element
  int max_pairs = 0, tile = 0, lanes = 1;
  bool graphs = true;
  bool engine = true;            // persistent pair engine (else four kernels per batch)
  bool tc = false;               // tensor-core GEMMs (complex FP32 storage)
  bool bf16 = false;             // M and the apply with BF16 operands (ACE_PREC_SPLIT_BF16)
  bool overlap = false;          // graph mode: pass A of batch k+1 overlaps pass D of batch k
  int radix = 0;                 // line-transform radix order (ACE_FLAG_RADIX_ODD_FIRST)
  unsigned eng_polls = kEngineSpinDefault;   // engine wait limit (ace_debug_engine_wait)
  unsigned eng_bias = 0;
  cudaEvent_t ov_ev[2] = {};

  EngineInfo einfo;
  std::vector<double> tw[3];     // per axis x, y, z: 2n doubles, exp(-2 pi i k / n)
  Schedule build;                // symmetric schedule of the W build
  std::deque<std::pair<int, Schedule>> rect;   // one-sided schedules by n_b
  std::deque<std::pair<int, Schedule>> pois;   // one-sided schedules of one constant orbital, by n_b
  void* ones = nullptr;          // N_g vector of ones (the left factor of the Poisson solves)
  void* Kt = nullptr;            // kernel table (float or double)
  double* Mc = nullptr;          // 2 N^2, M (complex, row-major)
  double* work = nullptr;        // 4 N^2, Cholesky work (global fallback)
  double* LinvH = nullptr;       // 2 N^2, L^{-*}
  int* status = nullptr;         // [code, pivot]
  cudaStream_t cap = nullptr;    // capture stream
  cudaStream_t lane[kMaxLanes] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kMaxLanes] = {};
  std::vector<GraphEntry> graph_cache;
  unsigned long long use_clock = 0;
  long long launches = 0;        // kernel launches issued (instrumentation)
  std::vector<cudaEvent_t> ev;   // profiling events
  size_t ev_used = 0;
  long long ev_dropped = 0;
  std::vector<ProfRec> prof;
};

namespace {

// Copy the tile descriptors of every batch to one device array (kernels read
// them from there, which keeps the launch parameter block small), and build
// the persistent engine's task tables (Poisson and energy-only).
cudaError_t upload(const ace_plan* p, Schedule& sc) {
  std::vector<TileDesc> all;
  std::vector<EngineBatch> eng[2];
  long long t0[2] = {0, 0};
  long long slots = 0;
  for (const Batch& b : sc.batches) {
    sc.soff.push_back(slots);
    slots += b.npairs;
    sc.toff.push_back((int)all.size());
    int nt[4] = {0, 0, 0, 0};
    if (p->cubic) {
      if (p->f64) engine_tasks_f64(p->nx, b, nt);
      else engine_tasks_f32(p->nx, b, nt);
    }
    for (int m = 0; m < 2; ++m) {
      EngineBatch e{};
      e.toff = (int)all.size();
      e.ntiles = b.ntiles;
      e.npairs = b.npairs;
      e.task0 = t0[m];
      for (int q = 0; q < 4; ++q) e.n[q] = (m == 1 && q >= 2) ? 0 : nt[q];
      t0[m] += e.n[0] + e.n[1] + e.n[2] + e.n[3];
      eng[m].push_back(e);
    }
    for (int t = 0; t < b.ntiles; ++t) all.push_back(b.t[t]);
  }
  sc.ntasks[0] = t0[0];
  sc.ntasks[1] = t0[1];
  if (all.empty()) return cudaSuccess;
  cudaError_t e = dev_alloc((void**)&sc.dtiles, all.size() * sizeof(TileDesc));
  if (e == cudaSuccess) e = cudaMemcpy(sc.dtiles, all.data(), all.size() * sizeof(TileDesc), cudaMemcpyHostToDevice);
  for (int m = 0; m < 2 && e == cudaSuccess; ++m) {
    e = dev_alloc((void**)&sc.deng[m], eng[m].size() * sizeof(EngineBatch));
    if (e == cudaSuccess)
      e = cudaMemcpy(sc.deng[m], eng[m].data(), eng[m].size() * sizeof(EngineBatch), cudaMemcpyHostToDevice);
  }
  return e;
}

// Tournament ("circle") schedule over orbital blocks: every round pairs each
// block with exactly one other, so the tiles of a round write disjoint outputs.
Schedule make_sym_schedule(int N, int b, int max_pairs, bool real) {
  const int B = (N + b - 1) / b;
  auto blk = [&](int I, int& o0, int& no) { o0 = I * b; no = (I * b + b <= N) ? b : N - I * b; };
  std::vector<std::vector<TileDesc>> rounds;
  const int Bp = (B % 2) ? B + 1 : B;
  std::vector<int> arr(Bp);
  for (int i = 0; i < Bp; ++i) arr[i] = i;
  for (int round = 0; round + 1 < Bp; ++round) {
    std::vector<TileDesc> tiles;
    for (int i = 0; i < Bp / 2; ++i) {
      int I = arr[i], J = arr[Bp - 1 - i];
      if (I >= B || J >= B) continue;   // bye
      if (I > J) std::swap(I, J);
      TileDesc t{};
      blk(I, t.l0, t.nl);
      blk(J, t.r0, t.nr);
      t.kind = 0;
      tiles.push_back(t);
    }
    rounds.push_back(tiles);
    const int last = arr[Bp - 1];   // rotate all but the first entry
    for (int i = Bp - 1; i > 1; --i) arr[i] = arr[i - 1];
    arr[1] = last;
  }
  std::vector<TileDesc> diag;
  for (int I = 0; I < B; ++I) {
    TileDesc t{};
    blk(I, t.l0, t.nl);
    t.r0 = t.l0;
    t.nr = t.nl;
    t.kind = 1;
    diag.push_back(t);
  }
  rounds.push_back(diag);
  Schedule out;
  int rid = 0;
  for (auto& r : rounds) {
    Batch cur{};
    for (auto& t : r) {
      const int np = tile_slots(t, real);
      if (cur.ntiles > 0 && (cur.npairs + np > max_pairs || cur.ntiles == kMaxTiles)) {
        out.batches.push_back(cur);
        out.round.push_back(rid);
        cur = Batch{};
      }
      t.slot0 = cur.npairs;
      cur.t[cur.ntiles++] = t;
      cur.npairs += np;
    }
    if (cur.ntiles > 0) {
      out.batches.push_back(cur);
      out.round.push_back(rid);
    }
    ++rid;
  }
  return out;
}

// Orbitals of Phi per l-chunk of a one-sided schedule: as many as fill a batch
// of max_pairs slots with r-blocks of b (b / 2 slots per orbital for real vectors).
int rect_chunk(int N, int b, int max_pairs, bool real) {
  int lc = max_pairs / (real ? (b + 1) / 2 : b);
  if (lc < 1) lc = 1;
  if (lc > N) lc = N;
  return lc;
}

// One-sided schedule for V_X[Phi] Psi: r-blocks of Psi (<= b), l-chunks of Phi;
// a round holds the tiles of one l-chunk, which write distinct Psi blocks.
Schedule make_rect_schedule(int N, int nb, int b, int max_pairs, bool real) {
  Schedule out;
  const int nrb = (nb + b - 1) / b;
  const int lc = rect_chunk(N, b, max_pairs, real);
  int rid = 0;
  for (int l0 = 0; l0 < N; l0 += lc, ++rid) {
    const int nl = (l0 + lc <= N) ? lc : N - l0;
    Batch cur{};
    for (int R = 0; R < nrb; ++R) {
      TileDesc t{};
      t.l0 = l0;
      t.nl = nl;
      t.r0 = R * b;
      t.nr = (R * b + b <= nb) ? b : nb - R * b;
      t.kind = 2;
      const int np = tile_slots(t, real);
      if (cur.ntiles > 0 && (cur.npairs + np > max_pairs || cur.ntiles == kMaxTiles)) {
        out.batches.push_back(cur);
        out.round.push_back(rid);
        cur = Batch{};
      }
      t.slot0 = cur.npairs;
      cur.t[cur.ntiles++] = t;
      cur.npairs += np;
    }
    if (cur.ntiles > 0) {
      out.batches.push_back(cur);
      out.round.push_back(rid);
    }
  }
  return out;
}

struct WsLayout {
  char* S = nullptr;
  double* Epart = nullptr;
  double* part = nullptr;
  double* Cm = nullptr;
  char* Wtmp = nullptr;
  char* ctr = nullptr;          // engine queue head + per-batch counters
  double* work = nullptr;       // oversampled build: Cholesky work and L^{-*} of N_phi
  double* LinvH = nullptr;
  char* xis = nullptr;          // FP64-accurate Xi: row/column exponents and C slices
  char* store = nullptr;        // pair potentials kept between calls (ACE_OP_ENERGY_GRAD_STORE)
  size_t total = 0;
};

// Split-K partial matrices of a gram product (the tensor-core or CUDA-core one).
int gram_parts(const ace_plan* p, int na, int nb) {
  return p->tc ? gram_tc_splits(p->ng, na, nb) : gram_splits(p->ng, na, nb);
}

// Upper bound on the batches of the one-sided schedule for n_b vectors.
long long rect_batch_bound(const ace_plan* p, int nb) {
  const int N = p->d.n_occ, b = p->tile;
  const int lc = rect_chunk(N, b, p->max_pairs, p->real);
  return (long long)((N + lc - 1) / lc) * ((nb + b - 1) / b);
}

int epart_per_lane(const ace_plan* p) { return energy_blocks(p->nx, p->ny, p->nz, p->max_pairs) + 1; }
size_t slot_bytes(const ace_plan* p) { return (size_t)p->ng * p->csize; }
size_t lane_bytes(const ace_plan* p) { return align256((size_t)p->max_pairs * slot_bytes(p)); }

WsLayout layout(const ace_plan* p, int op, int nb, char* base) {
  WsLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) { char* r = base ? base + off : nullptr; off += align256(bytes); return r; };
  const int N = p->d.n_occ;
  const int splits = op == ACE_OP_BUILD_OVERSAMPLED ? gram_parts(p, nb, nb) : gram_parts(p, N, op == ACE_OP_APPLY ? nb : N);
  if (op == ACE_OP_EXCHANGE_APPLY || op == ACE_OP_BUILD || op == ACE_OP_ENERGY_GRAD || op == ACE_OP_BUILD_OVERSAMPLED ||
      op == ACE_OP_POISSON || op == ACE_OP_ENERGY_GRAD_STORE) {
    L.S = take((size_t)p->lanes * lane_bytes(p));
    long long nbat = op == ACE_OP_EXCHANGE_APPLY ? rect_batch_bound(p, nb) : (long long)p->build.batches.size();
    if (op == ACE_OP_POISSON) nbat = (nb + p->tile - 1) / p->tile;
    if (op == ACE_OP_BUILD_OVERSAMPLED && nb > N && rect_batch_bound(p, nb - N) > nbat) nbat = rect_batch_bound(p, nb - N);
    L.ctr = take(engine_ctr_bytes(nbat));
  }
  if (op == ACE_OP_BUILD_OVERSAMPLED) {
    const size_t pd = (size_t)splits * nb * nb * 2;
    L.part = (double*)take((pd > diag_dot_part_doubles(nb) ? pd : diag_dot_part_doubles(nb)) * sizeof(double));
    L.Wtmp = take((size_t)nb * p->ld * p->vsize);
    L.Cm = (double*)take((size_t)nb * nb * 2 * sizeof(double));
    if (p->xi == 1) L.xis = take(xi_oz_scratch_bytes(p->ng, nb, nb, false));
    L.work = (double*)take(cholesky_work_doubles(nb) * sizeof(double));
    L.LinvH = (double*)take((size_t)nb * nb * 2 * sizeof(double));
  }
  if (op == ACE_OP_ENERGY_GRAD || op == ACE_OP_ENERGY_GRAD_STORE)
    L.Epart = (double*)take((size_t)p->lanes * epart_per_lane(p) * sizeof(double));
  if (op == ACE_OP_ENERGY_GRAD_STORE) {   // every unique pair potential of the build schedule
    long long slots = 0;
    for (const Batch& b : p->build.batches) slots += b.npairs;
    L.store = take((size_t)slots * slot_bytes(p));
  }
  if (op == ACE_OP_BUILD) {
    const size_t pd = (size_t)splits * N * N * 2;
    L.part = (double*)take((pd > diag_dot_part_doubles(N) ? pd : diag_dot_part_doubles(N)) * sizeof(double));
    L.Wtmp = take((size_t)N * p->ld * p->vsize);
    if (p->xi == 1) L.xis = take(xi_oz_scratch_bytes(p->ng, N, N, false));
  }
  if (op == ACE_OP_APPLY) {
    L.part = (double*)take((size_t)splits * N * nb * 2 * sizeof(double));
    L.Cm = (double*)take((size_t)N * nb * 2 * sizeof(double));
  }
  L.total = off;
  return L;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

ace_status check_common(ace_plan* p, void* ws, size_t ws_bytes, int op, int nb) {
  if (!p) return fail(ACE_ERR_ARG, "plan is NULL");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device)
    return fail(ACE_ERR_ARG, "current device differs from the plan's device");
  const size_t need = layout(p, op, nb, nullptr).total;
  if (ws_bytes < need)
    return fail(ACE_ERR_WORKSPACE, "workspace too small: need " + std::to_string(need) + " bytes");
  if (need > 0 && (!ws || ((uintptr_t)ws & 255u)))
    return fail(ACE_ERR_ARG, "workspace NULL or not 256-byte aligned");
  return ACE_OK;
}

bool launch_one(const ace_plan* p, const PairLaunch& L, const Batch& b, cudaStream_t st) {
  return p->f64 ? launch_pair_batch_f64(L, b, st) : launch_pair_batch_f32(L, b, st);
}

cudaEvent_t* take_events(ace_plan* p, int count, int kind) {
  if (p->ev.empty()) return nullptr;
  if (p->ev_used + (size_t)count > p->ev.size()) {
    ++p->ev_dropped;
    return nullptr;
  }
  cudaEvent_t* e = &p->ev[p->ev_used];
  p->prof.push_back(ProfRec{p->ev_used, kind});
  p->ev_used += (size_t)count;
  return e;
}

// Enqueue the pair-solve section on `cs`. Eager mode (graphs off): batches in
// order on `cs` with lane-0 scratch and, when profiling, events around every
// pass. Graph mode (called while capturing `cs`): the batches of one round
// are spread over the plan's lanes (fork/join through events), consecutive
// rounds are joined. Returns the kernel count, or -1 if the edge is not built.
//
// With `store` set, batch k works in its own part of a store of every pair
// potential (slots sc.soff[k] ..), nothing is reused, and base.pass_mask
// selects the passes (A-C to fill the store, D to consume it); the persistent
// engine is not used then.
long long issue_pairs(ace_plan* p, const PairLaunch& base, const Schedule& sc, char* S0, double* E0,
                      char* ctr, cudaStream_t cs, bool reset_status = true, char* store = nullptr) {
  long long kernels = 0;
  if (reset_status) cudaMemsetAsync(p->status, 0, 2 * sizeof(int), cs);
  if (sc.batches.empty()) return 0;
  const int gmask = base.pass_mask ? base.pass_mask : 15;
  auto scratch = [&](size_t k, char* dflt) { return store ? store + (size_t)sc.soff[k] * slot_bytes(p) : dflt; };
  auto launches = [&](int mask, int mode) {   // kernels one batch issues for a pass mask
    int c = 0;
    for (int b = 0; b < 4; ++b) c += (mask >> b) & 1;
    return mode == 1 ? std::min(c, 2) : c;
  };
  if (p->engine && !store) {   // one persistent launch for the whole schedule
    const int m = base.mode == 1 ? 1 : 0;
    cudaMemsetAsync(ctr, 0, engine_ctr_bytes((long long)sc.batches.size()), cs);
    PairLaunch L = base;
    L.S = S0;
    L.Epart = E0;
    L.ev = nullptr;
    L.dtiles = sc.dtiles;
    EngineLaunch E{};
    E.dtiles = sc.dtiles;
    E.batches = sc.deng[m];
    E.nbatches = (int)sc.batches.size();
    E.ntasks = sc.ntasks[m];
    E.head = reinterpret_cast<unsigned long long*>(ctr);
    E.done = reinterpret_cast<unsigned*>(ctr + 128);
    E.status = p->status;
    E.blocks = p->einfo.blocks;
    E.smem = p->einfo.smem;
    E.spin_limit = p->eng_polls;
    E.wait_bias = p->eng_bias;
    const bool ok = p->f64 ? launch_engine_f64(L, E, cs) : launch_engine_f32(L, E, cs);
    return ok ? 1 : -1;
  }
  if (!p->graphs) {
    for (const Batch& b : sc.batches) {
      const size_t k = (size_t)(&b - sc.batches.data());
      PairLaunch L = base;
      L.S = scratch(k, S0);
      L.Epart = E0;
      L.ev = take_events(p, 5, 0);
      L.dtiles = sc.dtiles + sc.toff[k];
      kernels += launches(gmask, L.mode);
      if (!launch_one(p, L, b, cs)) return -1;
    }
    return kernels;
  }
  if (p->overlap && base.mode != 1) {
    // Two streams: lane 0 runs pass A of every batch, lane 1 runs B, C and D.
    // A(k+1) waits for C(k), so it overlaps D(k) and fills D's tail; the
    // scratch alternates between two buffers, and C(k) completes after D(k-1)
    // (same stream), so a buffer is free before A rewrites it. Letting A run
    // further ahead, or moving B or C to lane 0, measured slower.
    cudaStream_t la = p->lane[0], lb = p->lane[1];
    cudaEventRecord(p->fork_ev, cs);
    cudaStreamWaitEvent(la, p->fork_ev, 0);
    cudaStreamWaitEvent(lb, p->fork_ev, 0);
    bool ok = true;
    for (size_t k = 0; k < sc.batches.size(); ++k) {
      PairLaunch L = base;
      L.S = scratch(k, S0 + (k & 1) * lane_bytes(p));
      L.Epart = E0;
      L.ev = nullptr;
      L.dtiles = sc.dtiles + sc.toff[k];
      L.pass_mask = 1 & gmask;
      if (L.pass_mask) ok = ok && launch_one(p, L, sc.batches[k], la);
      cudaEventRecord(p->ov_ev[0], la);
      cudaStreamWaitEvent(lb, p->ov_ev[0], 0);
      L.pass_mask = (2 | 4) & gmask;
      if (L.pass_mask) ok = ok && launch_one(p, L, sc.batches[k], lb);
      cudaEventRecord(p->ov_ev[1], lb);
      cudaStreamWaitEvent(la, p->ov_ev[1], 0);
      L.pass_mask = 8 & gmask;
      if (L.pass_mask) ok = ok && launch_one(p, L, sc.batches[k], lb);
      kernels += launches(gmask, L.mode);
    }
    cudaEventRecord(p->join_ev[0], la);
    cudaStreamWaitEvent(cs, p->join_ev[0], 0);
    cudaEventRecord(p->join_ev[1], lb);
    cudaStreamWaitEvent(cs, p->join_ev[1], 0);
    return ok ? kernels : -1;
  }
  const int nl = p->lanes;
  auto fork = [&]() {
    cudaEventRecord(p->fork_ev, cs);
    for (int i = 0; i < nl; ++i) cudaStreamWaitEvent(p->lane[i], p->fork_ev, 0);
  };
  auto join = [&]() {
    for (int i = 0; i < nl; ++i) {
      cudaEventRecord(p->join_ev[i], p->lane[i]);
      cudaStreamWaitEvent(cs, p->join_ev[i], 0);
    }
  };
  fork();
  int cur = sc.round.empty() ? 0 : sc.round[0], k_in_round = 0;
  bool ok = true;
  for (size_t k = 0; k < sc.batches.size(); ++k) {
    if (sc.round[k] != cur) {
      join();
      fork();
      cur = sc.round[k];
      k_in_round = 0;
    }
    const int ln = k_in_round++ % nl;
    PairLaunch L = base;
    L.S = scratch(k, S0 + (size_t)ln * lane_bytes(p));
    L.Epart = E0 ? E0 + (size_t)ln * epart_per_lane(p) : nullptr;
    L.ev = nullptr;
    L.dtiles = sc.dtiles + sc.toff[k];
    kernels += launches(gmask, L.mode);
    ok = ok && launch_one(p, L, sc.batches[k], p->lane[ln]);
  }
  join();
  return ok ? kernels : -1;
}

// Run `issue(stream)` (which enqueues work and returns its kernel count, or
// -1): eagerly on `st` when graphs are off, else by replaying the graph cached
// under `key`, capturing it on the plan's capture stream on first use. With
// `timed`, profiling events bracket the graph launch.
template <typename F>
ace_status run_graph(ace_plan* p, const uintptr_t key[8], cudaStream_t st, bool timed, F&& issue) {
  if (!p->graphs) {
    const long long k = issue(st);
    if (k < 0) return fail(ACE_ERR_UNSUPPORTED, "edge not built");
    p->launches += k;
    return cuda_check("eager section");
  }
  GraphEntry* hit = nullptr;
  for (auto& g : p->graph_cache)
    if (std::memcmp(g.key, key, sizeof(g.key)) == 0) hit = &g;
  if (!hit) {
    if ((int)p->graph_cache.size() >= kMaxGraphs) {
      size_t victim = 0;
      for (size_t i = 1; i < p->graph_cache.size(); ++i)
        if (p->graph_cache[i].last_use < p->graph_cache[victim].last_use) victim = i;
      cudaGraphExecDestroy(p->graph_cache[victim].exec);
      p->graph_cache.erase(p->graph_cache.begin() + victim);
    }
    GraphEntry g;
    std::memcpy(g.key, key, sizeof(g.key));
    cudaStream_t cs = p->cap;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return cuda_check("graph capture begin");
    g.kernels = issue(cs);
    const bool ok = g.kernels >= 0;
    cudaGraph_t graph = nullptr;
    const cudaError_t e1 = cudaStreamEndCapture(cs, &graph);
    if (!ok || e1 != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return ok ? fail(ACE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e1))
                : fail(ACE_ERR_UNSUPPORTED, "edge not built");
    }
    const cudaError_t e2 = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) return fail(ACE_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
    p->graph_cache.push_back(g);
    hit = &p->graph_cache.back();
  }
  hit->last_use = ++p->use_clock;
  cudaEvent_t* ev = timed ? take_events(p, 2, 1) : nullptr;
  if (ev) cudaEventRecord(ev[0], st);
  if (cudaGraphLaunch(hit->exec, st) != cudaSuccess) return cuda_check("graph launch");
  if (ev) cudaEventRecord(ev[1], st);
  p->launches += hit->kernels;
  return cuda_check("graph section");
}

PairLaunch base_launch(const ace_plan* p) {
  PairLaunch L{};
  L.nx = p->nx;
  L.ny = p->ny;
  L.nz = p->nz;
  L.ld = p->ld;
  L.Kt = p->Kt;
  L.twx = p->tw[0].data();
  L.twy = p->tw[1].data();
  L.twz = p->tw[2].data();
  L.real_io = p->real;
  L.scale = 1.0;
  L.prepare_only = false;
  L.no_pdl = (p->d.flags & ACE_FLAG_NO_PDL) != 0;
  L.radix = p->radix;
  return L;
}

// The one-sided schedule for n_b target vectors: the plan keeps one per n_b
// seen; the first call with an n_b builds and uploads it (a small allocation).
const Schedule* rect_schedule(ace_plan* p, int nb) {
  for (auto& c : p->rect)
    if (c.first == nb) return &c.second;
  p->rect.emplace_back(nb, make_rect_schedule(p->d.n_occ, nb, p->tile, p->max_pairs, p->real));
  if (upload(p, p->rect.back().second) != cudaSuccess) {
    free_schedule(p->rect.back().second);
    p->rect.pop_back();
    return nullptr;
  }
  return &p->rect.back().second;
}

// The one-sided schedule of the Poisson solves (one constant left orbital).
const Schedule* poisson_schedule(ace_plan* p, int nb) {
  for (auto& c : p->pois)
    if (c.first == nb) return &c.second;
  p->pois.emplace_back(nb, make_rect_schedule(1, nb, p->tile, p->max_pairs, p->real));
  if (upload(p, p->pois.back().second) != cudaSuccess) {
    free_schedule(p->pois.back().second);
    p->pois.pop_back();
    return nullptr;
  }
  return &p->pois.back().second;
}

void drop_graphs(ace_plan* p) {
  for (auto& g : p->graph_cache) cudaGraphExecDestroy(g.exec);
  p->graph_cache.clear();
}

// Zero `count` vectors of the plan's layout (only the N_g elements of each).
void zero_vectors(const ace_plan* p, void* X, long long count, cudaStream_t st) {
  const size_t row = (size_t)p->ng * p->vsize;
  if (p->ld == p->ng) cudaMemsetAsync(X, 0, (size_t)count * row, st);
  else cudaMemset2DAsync(X, (size_t)p->ld * p->vsize, 0, row, (size_t)count, st);
}

// Xi = W L^{-*} (Eq. Wtilde) for `nk` vectors on `cs` by the plan's Xi mode;
// returns the kernel count.
// c32: scratch of nk * nk * 8 bytes for the TF32 product's FP32 copy of L^{-*}
// (the gram partials, dead by then).
int issue_xi(ace_plan* p, const void* W, int nk, const double* LinvH, void* Xi, char* xis, void* c32,
             cudaStream_t cs) {
  if (p->xi == 1) return launch_xi_oz(W, nk, LinvH, nk, p->ld, p->ng, Xi, false, xis, p->status, cs);
  if (p->xi == 2) {
    launch_outer_f64acc(W, nk, LinvH, nk, p->ld, p->ng, Xi, false, cs);
    return 1;
  }
  if (p->tc) {
    launch_outer_tc(W, nk, LinvH, nk, p->ld, p->ng, 1.0, Xi, c32, p->status, cs);
    return 2;
  }
  launch_outer(p->f64, p->real, W, nk, LinvH, nk, p->ld, p->ng, 1.0, Xi, cs);
  return 1;
}

// The W build's pair section on `cs`: W = 0, then W = V_X[Phi] Phi over the
// unique pairs (Eq. W). Returns the kernel count, or -1.
long long issue_build_pairs(ace_plan* p, const void* Phi, void* W, const WsLayout& Wl, cudaStream_t cs) {
  PairLaunch L = base_launch(p);
  L.X = Phi;
  L.Y = Phi;
  L.OutX = W;
  L.OutY = W;
  L.mode = 0;
  zero_vectors(p, W, p->d.n_occ, cs);
  return issue_pairs(p, L, p->build, Wl.S, nullptr, Wl.ctr, cs);
}

// The build's dense section on `cs`: M = dV Phi^* W, Hermitian part (Eq.
// ACEconstruct2); -M = L L^* and L^{-*} in FP64; Xi = W L^{-*} (Eq. Wtilde).
long long issue_build_dense(ace_plan* p, const void* Phi, const void* W, void* Xi, const WsLayout& Wl,
                            cudaStream_t cs) {
  const int N = p->d.n_occ;
  const int splits = gram_parts(p, N, N);
  if (p->tc) launch_gram_tc(Phi, N, W, N, p->ld, p->ng, Wl.part, splits, p->status, cs, p->bf16);
  else launch_gram(p->f64, p->real, Phi, N, W, N, p->ld, p->ng, Wl.part, splits, cs);
  const int kr = launch_gram_reduce(Wl.part, splits, N, N, p->dv, true, false, p->Mc, nullptr, cs);
  if (p->tc) launch_diag_exact(Phi, W, N, p->ld, p->ng, p->dv, Wl.part, p->Mc, cs);
  const int kc = launch_cholesky_inv(p->Mc, N, p->work, p->LinvH, p->status, cs);
  const int kx = issue_xi(p, W, N, p->LinvH, Xi, Wl.xis, Wl.part, cs);
  return 1 + kr + (p->tc ? 2 : 0) + kc + kx;
}

// Tuned schedules (ace_autotune, ace_tuning_register), process-wide, keyed by
// the problem shape; ace_plan_create takes the registered schedule when the
// descriptor leaves max_pairs, tile and lanes at 0.
std::mutex g_tune_mu;
std::vector<ace_desc> g_tuned;
constexpr int kScheduleFlags = ACE_FLAG_NO_OVERLAP | ACE_FLAG_RADIX_ODD_FIRST;

bool same_problem(const ace_desc& a, const ace_desc& b) {
  return a.n[0] == b.n[0] && a.n[1] == b.n[1] && a.n[2] == b.n[2] && a.n_occ == b.n_occ && a.dtype == b.dtype &&
         a.prec == b.prec && a.kernel == b.kernel;
}

void register_tuned(const ace_desc& t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& e : g_tuned)
    if (same_problem(e, t)) {
      e = t;
      return;
    }
  g_tuned.push_back(t);
}

// One captured graph per batch of systems (ace_build_batched), shared by all
// plans of the process and keyed by every pointer the graph bakes in.
struct BatchGraph {
  std::vector<uintptr_t> key;
  std::vector<ace_plan*> plans;
  std::vector<long long> kernels;   // per system
  cudaGraphExec_t exec = nullptr;
  unsigned long long last_use = 0;
};
std::mutex g_batch_mu;
std::vector<BatchGraph> g_batch_graphs;
unsigned long long g_batch_clock = 0;
constexpr int kMaxBatchGraphs = 4;

void drop_batch_graphs_of(const ace_plan* p) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (size_t i = 0; i < g_batch_graphs.size();) {
    auto& g = g_batch_graphs[i];
    if (std::find(g.plans.begin(), g.plans.end(), p) != g.plans.end()) {
      cudaGraphExecDestroy(g.exec);
      g_batch_graphs.erase(g_batch_graphs.begin() + i);
    } else {
      ++i;
    }
  }
}

// Estimated cost of one system's build (pair solves x grid points), used to
// balance the chains of a batch (longest-processing-time-first).
double build_cost(const ace_plan* p) {
  const double N = p->d.n_occ;
  return 0.5 * N * (N + 1.0) * (double)p->ng + N * N * (double)p->ng * 0.05;
}

}  // namespace

ace_status ace_internal_plan_info(const ace_plan* p, int* device, int* n_occ, long long* ng, long long* ld,
                                  double* dv, int* f64, int* real) {
  *device = p->device;
  *n_occ = p->d.n_occ;
  *ng = p->ng;
  *ld = p->ld;
  *dv = p->dv;
  *f64 = p->f64 ? 1 : 0;
  *real = p->real ? 1 : 0;
  return ACE_OK;
}

ace_status ace_internal_set_error(ace_status s, const char* msg) { return fail(s, msg); }

extern "C" {

int ace_supported_grid(const int n[3], int dtype) {
  if (!n || dtype < ACE_DTYPE_R64 || dtype > ACE_DTYPE_C64) return 0;
  return pair_grid_supported(dtype != ACE_DTYPE_C64, n[0], n[1], n[2]) ? 1 : 0;
}

int ace_supported_edge(int n, int dtype) {
  const int g[3] = {n, n, n};
  return ace_supported_grid(g, dtype);
}

const char* ace_last_error(void) { return g_last_error.c_str(); }

ace_status ace_plan_create(const ace_desc* d, ace_plan** out) {
  if (!out) return fail(ACE_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!d) return fail(ACE_ERR_ARG, "desc is NULL");
  if (d->dtype < ACE_DTYPE_R64 || d->dtype > ACE_DTYPE_C64) return fail(ACE_ERR_ARG, "bad dtype");
  if (d->kernel != ACE_KERNEL_BARE && d->kernel != ACE_KERNEL_ERFC && d->kernel != ACE_KERNEL_KINETIC)
    return fail(ACE_ERR_ARG, "bad kernel");
  if (d->n_occ < 1) return fail(ACE_ERR_ARG, "n_occ must be >= 1");
  if (d->n_occ > 1024) return fail(ACE_ERR_UNSUPPORTED, "n_occ > 1024 not supported");
  if (!(d->L[0] > 0 && d->L[1] > 0 && d->L[2] > 0)) return fail(ACE_ERR_ARG, "cell edges must be > 0");
  if (d->kernel == ACE_KERNEL_ERFC && !(d->omega > 0)) return fail(ACE_ERR_ARG, "omega must be > 0");
  if (!std::isfinite(d->alpha)) return fail(ACE_ERR_ARG, "alpha must be finite");
  if (d->n[0] < 1 || d->n[1] < 1 || d->n[2] < 1) return fail(ACE_ERR_ARG, "grid sizes must be >= 1");
  if (!ace_supported_grid(d->n, d->dtype))
    return fail(ACE_ERR_UNSUPPORTED, "grid " + std::to_string(d->n[0]) + "x" + std::to_string(d->n[1]) + "x" +
                                         std::to_string(d->n[2]) + " not built for this dtype");
  const long long ng_ = (long long)d->n[0] * d->n[1] * d->n[2];
  if (d->ld != 0 && (d->ld < ng_ || (d->ld & 1)))
    return fail(ACE_ERR_ARG, "ld must be 0 or an even count >= N_g");
  if (d->prec < ACE_PREC_DEFAULT || d->prec > ACE_PREC_SPLIT_BF16) return fail(ACE_ERR_ARG, "bad prec");
  if (d->dtype != ACE_DTYPE_C64 && d->prec != ACE_PREC_DEFAULT)
    return fail(ACE_ERR_UNSUPPORTED, "FP64 plans compute in FP64: prec must be ACE_PREC_DEFAULT");
  if ((d->flags & ACE_FLAG_SIMT_GEMM) && d->prec != ACE_PREC_DEFAULT && d->prec != ACE_PREC_FP32)
    return fail(ACE_ERR_ARG, "ACE_FLAG_SIMT_GEMM conflicts with prec");
  if (d->tile < 0 || d->tile > kTileMax) return fail(ACE_ERR_ARG, "tile must be 0..8");
  if (d->max_pairs < 0) return fail(ACE_ERR_ARG, "max_pairs must be >= 0");
  if (d->lanes < 0 || d->lanes > kMaxLanes) return fail(ACE_ERR_ARG, "lanes must be 0..8");

  ace_desc dd = *d;
  if (dd.max_pairs == 0 && dd.tile == 0 && dd.lanes == 0) {   // a registered tuned schedule, if any
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& t : g_tuned)
      if (same_problem(t, dd)) {
        dd.max_pairs = t.max_pairs;
        dd.tile = t.tile;
        dd.lanes = t.lanes;
        dd.flags = (dd.flags & ~kScheduleFlags) | (t.flags & kScheduleFlags);
        break;
      }
  }
  d = &dd;
  ace_plan* p = new ace_plan();
  p->d = *d;
  cudaGetDevice(&p->device);
  p->nx = d->n[0];
  p->ny = d->n[1];
  p->nz = d->n[2];
  p->cubic = p->nx == p->ny && p->ny == p->nz;
  p->ng = ng_;
  p->ld = d->ld ? d->ld : ng_;
  p->vol = d->L[0] * d->L[1] * d->L[2];
  p->dv = p->vol / (double)p->ng;
  p->f64 = d->dtype != ACE_DTYPE_C64;
  p->real = d->dtype == ACE_DTYPE_R64;
  p->csize = p->f64 ? 16 : 8;
  p->vsize = p->real ? 8 : p->csize;
  p->tile = d->tile ? d->tile : kTileMax;
  p->lanes = d->lanes ? d->lanes : 2;
  p->graphs = !(d->flags & ACE_FLAG_NO_GRAPH);
  p->engine = (d->flags & ACE_FLAG_ENGINE) != 0 && p->cubic;
  p->tc = !p->f64 && !(d->flags & ACE_FLAG_SIMT_GEMM) && d->prec != ACE_PREC_FP32;
  // C64 default: Xi to FP64 accuracy on the FP16 tensor cores (the triangular
  // product stays FP64-accurate, as the Cholesky factor it applies)
  p->bf16 = p->tc && d->prec == ACE_PREC_SPLIT_BF16;
  const bool xi_slices = d->prec == ACE_PREC_XI_FP64 || d->prec == ACE_PREC_SPLIT_BF16 ||
                         (d->prec == ACE_PREC_DEFAULT && p->tc);
  p->xi = xi_slices ? 1 : (d->prec == ACE_PREC_XI_FP64_SIMT ? 2 : 0);
  p->overlap = p->graphs && !p->engine && !(d->flags & ACE_FLAG_NO_OVERLAP);
  if (p->overlap && p->lanes < 2) p->lanes = 2;
  p->radix = (!p->f64 && (d->flags & ACE_FLAG_RADIX_ODD_FIRST)) ? 1 : 0;
  const size_t slot = (size_t)p->ng * p->csize;
  const int tt = p->tile * p->tile;
  if (d->max_pairs) {
    p->max_pairs = d->max_pairs;
  } else {
    // a batch whose scratch (~72 MB per lane, at least one whole tile) stays
    // in L2 between the passes; at 48^3 FP32 that is one off-diagonal tile
    // (64 pairs) or two diagonal ones (2 x 36)
    const long long budget = (72ll << 20) / (long long)slot;
    p->max_pairs = (int)(budget > (long long)kMaxTiles * tt ? (long long)kMaxTiles * tt : budget);
  }
  if (p->max_pairs < tt) p->max_pairs = tt;

  // twiddles exp(-2 pi i k/n) in FP64, per axis
  const int nax[3] = {p->nx, p->ny, p->nz};
  for (int a = 0; a < 3; ++a) {
    p->tw[a].resize(2 * nax[a]);
    for (int k = 0; k < nax[a]; ++k) {
      const double t = 2.0 * M_PI * (double)k / (double)nax[a];
      p->tw[a][2 * k] = std::cos(t);
      p->tw[a][2 * k + 1] = -std::sin(t);
    }
  }
  // kernel table K(G) alpha / N_g, folded: every kernel depends on |G|^2 only,
  // and |G|^2 at index n - k equals that at k on each axis (the wrapped
  // frequency k - n = -k), so the table holds indices 0..n/2 per axis,
  // [kz][kx][ky] with (n_z/2 + 1)(n_x/2 + 1)(n_y/2 + 1) entries (62.5 KB at 48^3
  // FP32, L1-sized)
  const double g0_default = d->kernel == ACE_KERNEL_ERFC ? M_PI / (d->omega * d->omega) : 0.0;
  const double g0 = std::isnan(d->g0_value) ? g0_default : d->g0_value;
  const int nhx = p->nx / 2 + 1, nhy = p->ny / 2 + 1, nhz = p->nz / 2 + 1;
  std::vector<double> kt((size_t)nhz * nhx * nhy);
  for (int kz = 0; kz < nhz; ++kz)
    for (int kx = 0; kx < nhx; ++kx)
      for (int ky = 0; ky < nhy; ++ky) {
        const double gx = 2.0 * M_PI * kx / d->L[0];
        const double gy = 2.0 * M_PI * ky / d->L[1];
        const double gz = 2.0 * M_PI * kz / d->L[2];
        const double g2 = gx * gx + gy * gy + gz * gz;
        double k;
        if (g2 == 0.0) k = g0;
        else if (d->kernel == ACE_KERNEL_BARE) k = 4.0 * M_PI / g2;
        else if (d->kernel == ACE_KERNEL_KINETIC) k = 0.5 * g2;
        else k = 4.0 * M_PI / g2 * (1.0 - std::exp(-g2 / (4.0 * d->omega * d->omega)));
        kt[((size_t)kz * nhx + kx) * nhy + ky] = d->alpha * k / (double)p->ng;
      }
  const int N = d->n_occ;
  cudaError_t e = cudaSuccess;
  if (p->f64) {
    e = dev_alloc(&p->Kt, kt.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(p->Kt, kt.data(), kt.size() * sizeof(double), cudaMemcpyHostToDevice);
  } else {
    std::vector<float> kf(kt.begin(), kt.end());
    e = dev_alloc(&p->Kt, kf.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(p->Kt, kf.data(), kf.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    if (p->vsize == 8 && !p->real) {   // c64: (1.0f, 0.0f) pairs
      std::vector<float> onef((size_t)2 * p->ng, 0.0f);
      for (long long i = 0; i < p->ng; ++i) onef[2 * i] = 1.0f;
      e = dev_alloc(&p->ones, onef.size() * sizeof(float));
      if (e == cudaSuccess) e = cudaMemcpy(p->ones, onef.data(), onef.size() * sizeof(float), cudaMemcpyHostToDevice);
    } else {                           // r64: 1.0; c128: (1.0, 0.0)
      const size_t stride = p->real ? 1 : 2;
      std::vector<double> oned((size_t)p->ng * stride, 0.0);
      for (long long i = 0; i < p->ng; ++i) oned[stride * i] = 1.0;
      e = dev_alloc(&p->ones, oned.size() * sizeof(double));
      if (e == cudaSuccess) e = cudaMemcpy(p->ones, oned.data(), oned.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
  }
  if (e == cudaSuccess) e = dev_alloc((void**)&p->Mc, (size_t)2 * N * N * sizeof(double));
  if (e == cudaSuccess) e = dev_alloc((void**)&p->work, cholesky_work_doubles(N) * sizeof(double));
  if (e == cudaSuccess) e = dev_alloc((void**)&p->LinvH, (size_t)2 * N * N * sizeof(double));
  if (e == cudaSuccess) e = dev_alloc((void**)&p->status, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->status, 0, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
  for (int i = 0; i < p->lanes && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&p->lane[i], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming);
  for (int i = 0; i < p->lanes && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&p->join_ev[i], cudaEventDisableTiming);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&p->ov_ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess) {
    PairLaunch prep = base_launch(p);
    prep.prepare_only = true;
    Batch none{};
    launch_one(p, prep, none, nullptr);
    prepare_cholesky(N);
    if (p->tc) tc_gemm_prepare();
    if (p->xi == 1) xi_oz_prepare();
    if (p->engine) {
      if (p->f64) engine_prepare_f64(p->nx, p->einfo);
      else engine_prepare_f32(p->nx, p->einfo);
      if (p->einfo.blocks <= 0) p->engine = false;   // does not fit: four kernels per batch
    }
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    std::string m = std::string("plan set-up: ") + cudaGetErrorString(e);
    ace_plan_destroy(p);
    return fail(ACE_ERR_CUDA, m);
  }
  p->build = make_sym_schedule(N, p->tile, p->max_pairs, p->real);
  e = upload(p, p->build);
  if (e != cudaSuccess) {
    std::string m = std::string("schedule upload: ") + cudaGetErrorString(e);
    ace_plan_destroy(p);
    return fail(ACE_ERR_CUDA, m);
  }
  *out = p;
  return ACE_OK;
}

ace_status ace_plan_destroy(ace_plan* p) {
  if (!p) return ACE_OK;
  cudaDeviceSynchronize();
  drop_graphs(p);
  drop_batch_graphs_of(p);
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  for (int i = 0; i < kMaxLanes; ++i) {
    if (p->lane[i]) cudaStreamDestroy(p->lane[i]);
    if (p->join_ev[i]) cudaEventDestroy(p->join_ev[i]);
  }
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->fork_ev) cudaEventDestroy(p->fork_ev);
  for (cudaEvent_t e : p->ov_ev)
    if (e) cudaEventDestroy(e);
  free_schedule(p->build);
  for (auto& r : p->rect) free_schedule(r.second);
  for (auto& r : p->pois) free_schedule(r.second);
  cudaFree(p->ones);
  cudaFree(p->Kt);
  cudaFree(p->Mc);
  cudaFree(p->work);
  cudaFree(p->LinvH);
  cudaFree(p->status);
  delete p;
  return ACE_OK;
}

size_t ace_workspace_size(const ace_plan* p, int op, int nb) {
  if (!p || op < ACE_OP_EXCHANGE_APPLY || op > ACE_OP_ENERGY_GRAD_STORE) return 0;
  if ((op == ACE_OP_EXCHANGE_APPLY || op == ACE_OP_APPLY || op == ACE_OP_POISSON) && nb < 0) return 0;
  if (op == ACE_OP_BUILD_OVERSAMPLED && (nb < p->d.n_occ || nb > 1024)) return 0;
  return layout(p, op, nb, nullptr).total;
}

ace_status ace_exchange_apply(ace_plan* p, const void* Phi, const void* Psi, int nb, void* Y,
                              void* ws, size_t ws_bytes, void* stream) {
  ace_status s = check_common(p, ws, ws_bytes, ACE_OP_EXCHANGE_APPLY, nb);
  if (s != ACE_OK) return s;
  if (nb < 0) return fail(ACE_ERR_ARG, "n_b must be >= 0");
  if (nb == 0) return ACE_OK;
  if (!Phi || !Psi || !Y) return fail(ACE_ERR_ARG, "NULL vector pointer");
  if (!aligned16(Phi) || !aligned16(Psi) || !aligned16(Y)) return fail(ACE_ERR_ARG, "vectors must be 16-byte aligned");
  if (Y == Phi || Y == Psi) return fail(ACE_ERR_ARG, "Y must not alias Phi or Psi");
  cudaStream_t st = (cudaStream_t)stream;
  const WsLayout W = layout(p, ACE_OP_EXCHANGE_APPLY, nb, (char*)ws);
  PairLaunch L = base_launch(p);
  L.X = Phi;
  L.Y = Psi;
  L.OutX = nullptr;
  L.OutY = Y;
  L.mode = 0;
  const Schedule* sc = rect_schedule(p, nb);
  if (!sc) return cuda_check("schedule upload");
  const uintptr_t key[8] = {(uintptr_t)Phi, (uintptr_t)Psi, (uintptr_t)Y, (uintptr_t)ws, (uintptr_t)nb, 1, 0, 0};
  return run_graph(p, key, st, true, [&](cudaStream_t cs) -> long long {
    zero_vectors(p, Y, nb, cs);
    return issue_pairs(p, L, *sc, W.S, nullptr, W.ctr, cs);
  });
}

ace_status ace_build(ace_plan* p, const void* Phi, void* W_out, void* Xi_out, double* M_out,
                     double* Ex_out, void* ws, size_t ws_bytes, void* stream) {
  ace_status s = check_common(p, ws, ws_bytes, ACE_OP_BUILD, 0);
  if (s != ACE_OK) return s;
  if (!Phi || !Xi_out) return fail(ACE_ERR_ARG, "Phi and Xi_out are required");
  if (!aligned16(Phi) || !aligned16(Xi_out) || (W_out && !aligned16(W_out)))
    return fail(ACE_ERR_ARG, "vectors must be 16-byte aligned");
  if (Xi_out == Phi || W_out == Phi || (W_out && W_out == Xi_out))
    return fail(ACE_ERR_ARG, "outputs must not alias Phi or each other");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = p->d.n_occ;
  const WsLayout Wl = layout(p, ACE_OP_BUILD, 0, (char*)ws);
  void* W = W_out ? W_out : (void*)Wl.Wtmp;
  // W = V_X[Phi] Phi over the unique pairs (Eq. W)
  const uintptr_t kp[8] = {(uintptr_t)Phi, (uintptr_t)W, (uintptr_t)ws, 0, 0, 2, 0, 0};
  s = run_graph(p, kp, st, true, [&](cudaStream_t cs) -> long long {
    return issue_build_pairs(p, Phi, W, Wl, cs);
  });
  if (s != ACE_OK) return s;
  // M, its Cholesky factor, L^{-*} and Xi = W L^{-*}
  const uintptr_t kd[8] = {(uintptr_t)Phi, (uintptr_t)W, (uintptr_t)Xi_out, (uintptr_t)ws, 4, 0, 0, 0};
  s = run_graph(p, kd, st, false, [&](cudaStream_t cs) -> long long {
    return issue_build_dense(p, Phi, W, Xi_out, Wl, cs);
  });
  if (s != ACE_OK) return s;
  // caller-owned small outputs, outside the graph (their pointers vary per call)
  p->launches += launch_m_outputs(p->Mc, N, p->real, M_out, Ex_out, st);
  return cuda_check("ace_build");
}

ace_status ace_build_oversampled(ace_plan* p, const void* Phi, int n_phi, void* W_out, void* Xi_out,
                                 double* M_out, double* Ex_out, void* ws, size_t ws_bytes, void* stream) {
  if (!p) return fail(ACE_ERR_ARG, "plan is NULL");
  const int N = p->d.n_occ;
  if (n_phi < N || n_phi > 1024) return fail(ACE_ERR_ARG, "n_phi must be in [n_occ, 1024]");
  ace_status s = check_common(p, ws, ws_bytes, ACE_OP_BUILD_OVERSAMPLED, n_phi);
  if (s != ACE_OK) return s;
  if (!Phi || !Xi_out) return fail(ACE_ERR_ARG, "Phi and Xi_out are required");
  if (!aligned16(Phi) || !aligned16(Xi_out) || (W_out && !aligned16(W_out)))
    return fail(ACE_ERR_ARG, "vectors must be 16-byte aligned");
  if (Xi_out == Phi || W_out == Phi || (W_out && W_out == Xi_out))
    return fail(ACE_ERR_ARG, "outputs must not alias Phi or each other");
  cudaStream_t st = (cudaStream_t)stream;
  const WsLayout Wl = layout(p, ACE_OP_BUILD_OVERSAMPLED, n_phi, (char*)ws);
  void* W = W_out ? W_out : (void*)Wl.Wtmp;
  const size_t vec = (size_t)p->ld * p->vsize;
  const int nu = n_phi - N;
  const Schedule* sc = nu > 0 ? rect_schedule(p, nu) : nullptr;
  if (nu > 0 && !sc) return cuda_check("schedule upload");
  // W_i = V_X[Phi_occ] Phi_i: unique occupied pairs, then the one-sided pairs
  // of the occupied orbitals with the N_phi - N_e others (Eq. W, Eq. applyVX2)
  const uintptr_t kp[8] = {(uintptr_t)Phi, (uintptr_t)W, (uintptr_t)ws, (uintptr_t)n_phi, 0, 5, 0, 0};
  s = run_graph(p, kp, st, true, [&](cudaStream_t cs) -> long long {
    zero_vectors(p, W, n_phi, cs);
    PairLaunch L = base_launch(p);
    L.X = Phi;
    L.Y = Phi;
    L.OutX = W;
    L.OutY = W;
    L.mode = 0;
    const long long k1 = issue_pairs(p, L, p->build, Wl.S, nullptr, Wl.ctr, cs);
    long long k2 = 0;
    if (nu > 0) {
      PairLaunch R = base_launch(p);
      R.X = Phi;
      R.Y = static_cast<const char*>(Phi) + (size_t)N * vec;
      R.OutX = nullptr;
      R.OutY = static_cast<char*>(W) + (size_t)N * vec;
      R.mode = 0;
      k2 = issue_pairs(p, R, *sc, Wl.S, nullptr, Wl.ctr, cs, false);
    }
    return (k1 < 0 || k2 < 0) ? -1 : k1 + k2;
  });
  if (s != ACE_OK) return s;
  // M = dV Phi^* W (N_phi x N_phi), -M = L L^*, Xi = W L^{-*}
  const uintptr_t kd[8] = {(uintptr_t)Phi, (uintptr_t)W, (uintptr_t)Xi_out, (uintptr_t)ws, (uintptr_t)n_phi, 6, 0, 0};
  s = run_graph(p, kd, st, false, [&](cudaStream_t cs) -> long long {
    const int splits = gram_parts(p, n_phi, n_phi);
    if (p->tc) launch_gram_tc(Phi, n_phi, W, n_phi, p->ld, p->ng, Wl.part, splits, p->status, cs, p->bf16);
    else launch_gram(p->f64, p->real, Phi, n_phi, W, n_phi, p->ld, p->ng, Wl.part, splits, cs);
    const int kr = launch_gram_reduce(Wl.part, splits, n_phi, n_phi, p->dv, true, false, Wl.Cm, nullptr, cs);
    if (p->tc) launch_diag_exact(Phi, W, n_phi, p->ld, p->ng, p->dv, Wl.part, Wl.Cm, cs);
    const int kc = launch_cholesky_inv(Wl.Cm, n_phi, Wl.work, Wl.LinvH, p->status, cs);
    const int kx = issue_xi(p, W, n_phi, Wl.LinvH, Xi_out, Wl.xis, Wl.part, cs);
    return 1 + kr + (p->tc ? 2 : 0) + kc + kx;
  });
  if (s != ACE_OK) return s;
  p->launches += launch_m_outputs(Wl.Cm, n_phi, p->real, M_out, Ex_out, st, N);
  return cuda_check("ace_build_oversampled");
}

ace_status ace_poisson(ace_plan* p, const void* rho, int nb, void* V, void* ws, size_t ws_bytes, void* stream) {
  ace_status s = check_common(p, ws, ws_bytes, ACE_OP_POISSON, nb);
  if (s != ACE_OK) return s;
  if (nb < 0) return fail(ACE_ERR_ARG, "n_b must be >= 0");
  if (nb == 0) return ACE_OK;
  if (!rho || !V) return fail(ACE_ERR_ARG, "NULL vector pointer");
  if (!aligned16(rho) || !aligned16(V)) return fail(ACE_ERR_ARG, "vectors must be 16-byte aligned");
  if (V == rho) return fail(ACE_ERR_ARG, "V must not alias rho");
  cudaStream_t st = (cudaStream_t)stream;
  const WsLayout W = layout(p, ACE_OP_POISSON, nb, (char*)ws);
  const Schedule* sc = poisson_schedule(p, nb);
  if (!sc) return cuda_check("schedule upload");
  // one-sided pair solves of the constant orbital 1 with each rho_b: pass D
  // accumulates Out -= scale * 1 * v, so scale -1 leaves V_b = Poisson[rho_b]
  PairLaunch L = base_launch(p);
  L.X = p->ones;
  L.Y = rho;
  L.OutX = nullptr;
  L.OutY = V;
  L.mode = 0;
  L.scale = -1.0;
  const uintptr_t key[8] = {(uintptr_t)rho, (uintptr_t)V, (uintptr_t)ws, (uintptr_t)nb, 0, 7, 0, 0};
  return run_graph(p, key, st, true, [&](cudaStream_t cs) -> long long {
    zero_vectors(p, V, nb, cs);
    return issue_pairs(p, L, *sc, W.S, nullptr, W.ctr, cs);
  });
}

size_t ace_workspace_size_batched(ace_plan* const* plans, int n_sys) {
  if (!plans || n_sys < 0) return 0;
  size_t total = 0;
  for (int i = 0; i < n_sys; ++i) {
    if (!plans[i]) return 0;
    total += align256(layout(plans[i], ACE_OP_BUILD, 0, nullptr).total);
  }
  return total;
}

ace_status ace_build_batched(ace_plan* const* plans, const void* const* Phi, void* const* Xi, double* Ex,
                             int n_sys, int chains, void* ws, size_t ws_bytes, void* stream) {
  if (n_sys < 0 || chains < 0) return fail(ACE_ERR_ARG, "n_sys and chains must be >= 0");
  if (n_sys == 0) return ACE_OK;
  if (!plans || !Phi || !Xi) return fail(ACE_ERR_ARG, "plans, Phi and Xi are required");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(ACE_ERR_CUDA, "no current device");
  for (int i = 0; i < n_sys; ++i) {
    ace_plan* p = plans[i];
    if (!p) return fail(ACE_ERR_ARG, "plan " + std::to_string(i) + " is NULL");
    if (p->device != dev) return fail(ACE_ERR_ARG, "plan " + std::to_string(i) + " is on another device");
    for (int j = 0; j < i; ++j)
      if (plans[j] == p) return fail(ACE_ERR_ARG, "a plan appears twice in the batch");
    if (!Phi[i] || !Xi[i] || !aligned16(Phi[i]) || !aligned16(Xi[i]))
      return fail(ACE_ERR_ARG, "system " + std::to_string(i) + ": Phi/Xi NULL or not 16-byte aligned");
    if (Phi[i] == Xi[i]) return fail(ACE_ERR_ARG, "system " + std::to_string(i) + ": Xi aliases Phi");
  }
  const size_t need = ace_workspace_size_batched(plans, n_sys);
  if (ws_bytes < need) return fail(ACE_ERR_WORKSPACE, "workspace too small: need " + std::to_string(need) + " bytes");
  if (!ws || ((uintptr_t)ws & 255u)) return fail(ACE_ERR_ARG, "workspace NULL or not 256-byte aligned");
  const int K = std::max(1, std::min(chains ? chains : 3, n_sys));
  cudaStream_t st = (cudaStream_t)stream;

  std::vector<uintptr_t> key = {(uintptr_t)n_sys, (uintptr_t)K, (uintptr_t)ws, (uintptr_t)Ex, (uintptr_t)dev};
  for (int i = 0; i < n_sys; ++i) {
    key.push_back((uintptr_t)plans[i]);
    key.push_back((uintptr_t)Phi[i]);
    key.push_back((uintptr_t)Xi[i]);
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  BatchGraph* hit = nullptr;
  for (auto& g : g_batch_graphs)
    if (g.key == key) hit = &g;
  if (!hit) {
    if ((int)g_batch_graphs.size() >= kMaxBatchGraphs) {
      size_t victim = 0;
      for (size_t i = 1; i < g_batch_graphs.size(); ++i)
        if (g_batch_graphs[i].last_use < g_batch_graphs[victim].last_use) victim = i;
      cudaGraphExecDestroy(g_batch_graphs[victim].exec);
      g_batch_graphs.erase(g_batch_graphs.begin() + victim);
    }
    // systems by decreasing cost, each to the chain with the least work so far
    std::vector<int> order(n_sys);
    for (int i = 0; i < n_sys; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return build_cost(plans[a]) > build_cost(plans[b]); });
    std::vector<std::vector<int>> chain(K);
    std::vector<double> load(K, 0.0);
    for (int i : order) {
      const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      chain[c].push_back(i);
      load[c] += build_cost(plans[i]);
    }
    std::vector<size_t> off(n_sys + 1, 0);
    for (int i = 0; i < n_sys; ++i) off[i + 1] = off[i] + align256(layout(plans[i], ACE_OP_BUILD, 0, nullptr).total);

    BatchGraph g;
    g.key = key;
    g.plans.assign(plans, plans + n_sys);
    g.kernels.assign(n_sys, 0);
    cudaStream_t cs = nullptr;
    std::vector<cudaStream_t> cst(K, nullptr);
    std::vector<cudaEvent_t> jev(K, nullptr);
    cudaEvent_t fev = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int c = 0; c < K && e == cudaSuccess; ++c) e = cudaStreamCreateWithFlags(&cst[c], cudaStreamNonBlocking);
    for (int c = 0; c < K && e == cudaSuccess; ++c) e = cudaEventCreateWithFlags(&jev[c], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fev, cudaEventDisableTiming);
    bool ok = e == cudaSuccess;
    cudaGraph_t graph = nullptr;
    if (ok) ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      cudaEventRecord(fev, cs);
      for (int c = 0; c < K; ++c) {
        cudaStreamWaitEvent(cst[c], fev, 0);
        for (int i : chain[c]) {
          ace_plan* p = plans[i];
          const WsLayout Wl = layout(p, ACE_OP_BUILD, 0, (char*)ws + off[i]);
          std::vector<cudaEvent_t> prof_ev;   // no per-pass events inside the batch graph
          prof_ev.swap(p->ev);
          const long long k1 = issue_build_pairs(p, Phi[i], Wl.Wtmp, Wl, cst[c]);
          prof_ev.swap(p->ev);
          const long long k2 = issue_build_dense(p, Phi[i], Wl.Wtmp, Xi[i], Wl, cst[c]);
          const long long k3 = Ex ? launch_m_outputs(p->Mc, p->d.n_occ, p->real, nullptr, Ex + i, cst[c]) : 0;
          if (k1 < 0) ok = false;
          g.kernels[i] = k1 + k2 + k3;
        }
        cudaEventRecord(jev[c], cst[c]);
        cudaStreamWaitEvent(cs, jev[c], 0);
      }
      const cudaError_t e1 = cudaStreamEndCapture(cs, &graph);
      if (e1 != cudaSuccess) ok = false;
    }
    if (ok && graph) ok = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    const cudaError_t ce = cudaGetLastError();
    if (fev) cudaEventDestroy(fev);
    for (int c = 0; c < K; ++c) {
      if (jev[c]) cudaEventDestroy(jev[c]);
      if (cst[c]) cudaStreamDestroy(cst[c]);
    }
    if (cs) cudaStreamDestroy(cs);
    if (!ok) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      return fail(ce != cudaSuccess ? ACE_ERR_CUDA : ACE_ERR_UNSUPPORTED,
                  std::string("batched graph capture failed: ") +
                      (ce != cudaSuccess ? cudaGetErrorString(ce) : "an edge is not built"));
    }
    g_batch_graphs.push_back(std::move(g));
    hit = &g_batch_graphs.back();
  }
  hit->last_use = ++g_batch_clock;
  if (cudaGraphLaunch(hit->exec, st) != cudaSuccess) return cuda_check("batched graph launch");
  for (int i = 0; i < n_sys; ++i) plans[i]->launches += hit->kernels[i];
  return cuda_check("ace_build_batched");
}

ace_status ace_autotune(const ace_desc* d, int reps, ace_desc* best, double* ms_out) {
  if (!d || !best) return fail(ACE_ERR_ARG, "desc and best are required");
  if (reps <= 0) reps = 3;
  // probe the descriptor once (validation, sizes)
  ace_plan* probe = nullptr;
  ace_status s = ace_plan_create(d, &probe);
  if (s != ACE_OK) return s;
  const int N = probe->d.n_occ;
  const long long ng = probe->ng, vstride = probe->ld;
  const size_t vsize = probe->vsize, slot = (size_t)ng * probe->csize;
  const bool f64 = probe->f64;
  ace_plan_destroy(probe);

  // candidates: tile edge x batch scratch budget x pair schedule
  std::vector<ace_desc> cand;
  const int tiles[3] = {8, 6, 4};
  const long long budgets[3] = {72ll << 20, 36ll << 20, 144ll << 20};
  for (int tile : tiles) {
    if (tile > N && tile != tiles[0]) continue;   // tiles wider than N all act as one tile
    const int tt = tile * tile;
    for (long long b : budgets) {
      long long mp = b / (long long)slot;
      if (mp > (long long)kMaxTiles * tt) mp = (long long)kMaxTiles * tt;
      if (mp < tt) mp = tt;
      for (int ov = 1; ov >= 0; --ov) {
        for (int rx = 0; rx < (f64 ? 1 : 2); ++rx) {   // radix orders (FP32 line transforms)
          ace_desc c = *d;
          c.tile = tile;
          c.max_pairs = (int)mp;
          c.lanes = 2;
          c.flags = (d->flags & ~(ACE_FLAG_NO_OVERLAP | ACE_FLAG_NO_GRAPH | ACE_FLAG_ENGINE |
                                  ACE_FLAG_RADIX_ODD_FIRST)) |
                    (ov ? 0 : ACE_FLAG_NO_OVERLAP) | (rx ? ACE_FLAG_RADIX_ODD_FIRST : 0);
          bool dup = false;
          for (const auto& o : cand)
            dup = dup || (o.tile == c.tile && o.max_pairs == c.max_pairs && o.flags == c.flags);
          if (!dup) cand.push_back(c);
        }
      }
    }
  }
  void *Phi = nullptr, *Xi = nullptr, *ws = nullptr;
  size_t ws_cap = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const size_t vbytes = (size_t)N * vstride * vsize;
  cudaError_t e = dev_alloc(&Phi, vbytes);
  if (e == cudaSuccess) e = dev_alloc(&Xi, vbytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) launch_fill_random(Phi, (long long)(vbytes / (f64 ? 8 : 4)), f64, 1601071590ull, st);
  double best_ms = -1.0;
  s = e == cudaSuccess ? ACE_OK : fail(ACE_ERR_CUDA, std::string("autotune setup: ") + cudaGetErrorString(e));
  for (size_t i = 0; i < cand.size() && s == ACE_OK; ++i) {
    ace_plan* p = nullptr;
    if (ace_plan_create(&cand[i], &p) != ACE_OK) continue;   // e.g. out of memory for a large budget
    const size_t need = layout(p, ACE_OP_BUILD, 0, nullptr).total;
    if (need > ws_cap) {
      cudaFree(ws);
      ws = nullptr;
      ws_cap = 0;
      if (dev_alloc(&ws, need) != cudaSuccess) {
        cudaGetLastError();
        ace_plan_destroy(p);
        continue;
      }
      ws_cap = need;
    }
    s = ace_build(p, Phi, nullptr, Xi, nullptr, nullptr, ws, ws_cap, st);   // capture + warm-up
    if (s == ACE_OK) s = ace_status_sync(p, st, nullptr);
    if (s == ACE_OK) {
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && s == ACE_OK; ++r) s = ace_build(p, Phi, nullptr, Xi, nullptr, nullptr, ws, ws_cap, st);
      cudaEventRecord(e1, st);
      if (s == ACE_OK) s = ace_status_sync(p, st, nullptr);
      float ms = 0.f;
      if (s == ACE_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
        const double per = (double)ms / reps;
        if (best_ms < 0 || per < best_ms) {
          best_ms = per;
          *best = cand[i];
        }
      }
    }
    ace_plan_destroy(p);
  }
  cudaFree(ws);
  cudaFree(Phi);
  cudaFree(Xi);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (s != ACE_OK) return s;
  if (best_ms < 0) return fail(ACE_ERR_CUDA, "autotune: no candidate could be timed");
  if (ms_out) *ms_out = best_ms;
  register_tuned(*best);
  return ACE_OK;
}

ace_status ace_tuning_register(const ace_desc* tuned) {
  if (!tuned) return fail(ACE_ERR_ARG, "tuned is NULL");
  if (tuned->tile < 1 || tuned->tile > kTileMax || tuned->max_pairs < 1 || tuned->lanes < 0 || tuned->lanes > kMaxLanes)
    return fail(ACE_ERR_ARG, "a tuned schedule needs tile 1..8, max_pairs >= 1 and lanes 0..8");
  register_tuned(*tuned);
  return ACE_OK;
}

ace_status ace_tuning_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned.clear();
  return ACE_OK;
}

ace_status ace_plan_desc(const ace_plan* p, ace_desc* out) {
  if (!p || !out) return fail(ACE_ERR_ARG, "plan and out are required");
  *out = p->d;
  out->max_pairs = p->max_pairs;
  out->tile = p->tile;
  out->lanes = p->lanes;
  out->ld = p->ld;
  return ACE_OK;
}

ace_status ace_apply(ace_plan* p, const void* Xi, const void* Psi, int nb, void* Y, void* ws,
                     size_t ws_bytes, void* stream) {
  ace_status s = check_common(p, ws, ws_bytes, ACE_OP_APPLY, nb);
  if (s != ACE_OK) return s;
  if (nb < 0) return fail(ACE_ERR_ARG, "n_b must be >= 0");
  if (nb == 0) return ACE_OK;
  if (!Xi || !Psi || !Y) return fail(ACE_ERR_ARG, "NULL vector pointer");
  if (!aligned16(Xi) || !aligned16(Psi) || !aligned16(Y)) return fail(ACE_ERR_ARG, "vectors must be 16-byte aligned");
  if (Y == Xi || Y == Psi) return fail(ACE_ERR_ARG, "Y must not alias Xi or Psi");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = p->d.n_occ;
  const WsLayout Wl = layout(p, ACE_OP_APPLY, nb, (char*)ws);
  const int splits = gram_parts(p, N, nb);
  // C = dV Xi^* Psi, Y = -Xi C (Eq. ACE)
  if (p->tc) launch_gram_tc(Xi, N, Psi, nb, p->ld, p->ng, Wl.part, splits, p->status, st, p->bf16);
  else launch_gram(p->f64, p->real, Xi, N, Psi, nb, p->ld, p->ng, Wl.part, splits, st);
  launch_gram_reduce(Wl.part, splits, N, nb, p->dv, false, false, Wl.Cm, nullptr, st);
  if (p->tc) launch_outer_tc(Xi, N, Wl.Cm, nb, p->ld, p->ng, -1.0, Y, Wl.part, p->status, st, p->bf16);
  else launch_outer(p->f64, p->real, Xi, N, Wl.Cm, nb, p->ld, p->ng, -1.0, Y, st);
  p->launches += p->tc ? 4 : 3;
  return cuda_check("ace_apply");
}

ace_status ace_exchange_energy_grad(ace_plan* p, const void* Phi, double* Ex_out, void* grad_out,
                                    double grad_scale, int recompute, void* ws, size_t ws_bytes, void* stream) {
  const int op = recompute ? ACE_OP_ENERGY_GRAD : ACE_OP_ENERGY_GRAD_STORE;
  ace_status s = check_common(p, ws, ws_bytes, op, 0);
  if (s != ACE_OK) return s;
  if (!Phi || (!Ex_out && (recompute || !grad_out))) return fail(ACE_ERR_ARG, "Phi and Ex_out are required");
  if (!aligned16(Phi) || (grad_out && !aligned16(grad_out))) return fail(ACE_ERR_ARG, "vectors must be 16-byte aligned");
  if (grad_out == Phi) return fail(ACE_ERR_ARG, "grad_out must not alias Phi");
  if (!std::isfinite(grad_scale)) return fail(ACE_ERR_ARG, "grad_scale must be finite");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = p->d.n_occ;
  const WsLayout Wl = layout(p, op, 0, (char*)ws);
  const int ecount = p->lanes * epart_per_lane(p);
  const double efac = -0.5 * p->vol / (double)p->ng;   // E = -1/2 Omega/N_g sum_pairs w_p sum_G Kt |F rho|^2
  PairLaunch L = base_launch(p);
  L.X = Phi;
  L.Y = Phi;
  L.OutX = grad_out;
  L.OutY = grad_out;
  L.scale = 2.0 * p->dv;                   // grad = 2 dV W, then * grad_scale
  if (recompute) {
    // one sweep: energy (and, with grad_out, the potentials consumed batch by batch)
    L.mode = grad_out ? 2 : 1;
    const uintptr_t key[8] = {(uintptr_t)Phi, (uintptr_t)grad_out, (uintptr_t)Ex_out, (uintptr_t)ws, 0, 3, 0, 0};
    s = run_graph(p, key, st, true, [&](cudaStream_t cs) -> long long {
      cudaMemsetAsync(Wl.Epart, 0, (size_t)ecount * sizeof(double), cs);
      if (grad_out) zero_vectors(p, grad_out, N, cs);
      const long long k = issue_pairs(p, L, p->build, Wl.S, Wl.Epart, Wl.ctr, cs);
      launch_energy_reduce(Wl.Epart, ecount, efac, Ex_out, cs);
      return k < 0 ? k : k + 1;
    });
  } else if (!grad_out) {
    // the energy, and every unique pair potential into the workspace's store
    L.mode = 2;
    L.pass_mask = 1 | 2 | 4;
    const uintptr_t key[8] = {(uintptr_t)Phi, 0, (uintptr_t)Ex_out, (uintptr_t)ws, 0, 3, 1, 0};
    s = run_graph(p, key, st, true, [&](cudaStream_t cs) -> long long {
      cudaMemsetAsync(Wl.Epart, 0, (size_t)ecount * sizeof(double), cs);
      const long long k = issue_pairs(p, L, p->build, Wl.S, Wl.Epart, Wl.ctr, cs, true, Wl.store);
      launch_energy_reduce(Wl.Epart, ecount, efac, Ex_out, cs);
      return k < 0 ? k : k + 1;
    });
  } else {
    // the gradient from the stored potentials (pass D only); E_x again from
    // the stored energy partials
    L.mode = 0;
    L.pass_mask = 8;
    const uintptr_t key[8] = {(uintptr_t)Phi, (uintptr_t)grad_out, (uintptr_t)Ex_out, (uintptr_t)ws, 0, 3, 2, 0};
    s = run_graph(p, key, st, true, [&](cudaStream_t cs) -> long long {
      zero_vectors(p, grad_out, N, cs);
      const long long k = issue_pairs(p, L, p->build, Wl.S, nullptr, Wl.ctr, cs, true, Wl.store);
      if (Ex_out) launch_energy_reduce(Wl.Epart, ecount, efac, Ex_out, cs);
      return k < 0 ? k : k + (Ex_out ? 1 : 0);
    });
  }
  if (s != ACE_OK) return s;
  if (grad_out && grad_scale != 1.0) {   // outside the graph: the scale varies per call
    launch_scale(p->f64, p->real, grad_out, N, p->ng, p->ld, grad_scale, st);
    p->launches += 1;
  }
  return cuda_check("ace_exchange_energy_grad");
}

ace_status ace_profile_begin(ace_plan* p, int max_events) {
  if (!p) return fail(ACE_ERR_ARG, "plan is NULL");
  if (max_events < 5) return fail(ACE_ERR_ARG, "max_events must be >= 5");
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  p->ev.assign((size_t)max_events, nullptr);
  for (auto& e : p->ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      p->ev.clear();
      return cuda_check("ace_profile_begin");
    }
  p->ev_used = 0;
  p->ev_dropped = 0;
  p->prof.clear();
  p->launches = 0;
  return ACE_OK;
}

ace_status ace_profile_end(ace_plan* p, double* ms_out, long long* counts_out) {
  if (!p) return fail(ACE_ERR_ARG, "plan is NULL");
  if (cudaDeviceSynchronize() != cudaSuccess) return cuda_check("ace_profile_end");
  double ms[5] = {0, 0, 0, 0, 0};
  bool per_pass = false;
  long long recs = 0;
  for (const ProfRec& r : p->prof) {
    ++recs;
    if (r.kind == 0) {
      per_pass = true;
      for (int k = 0; k < 4; ++k) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p->ev[r.first + k], p->ev[r.first + k + 1]) == cudaSuccess) ms[k] += t;
      }
    } else {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p->ev[r.first], p->ev[r.first + 1]) == cudaSuccess) ms[4] += t;
    }
  }
  if (per_pass) ms[4] += ms[0] + ms[1] + ms[2] + ms[3];
  else ms[0] = ms[1] = ms[2] = ms[3] = std::numeric_limits<double>::quiet_NaN();
  if (ms_out)
    for (int k = 0; k < 5; ++k) ms_out[k] = ms[k];
  if (counts_out) {
    counts_out[0] = recs;
    counts_out[1] = p->launches;
    counts_out[2] = p->ev_dropped;
  }
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  p->ev.clear();
  p->prof.clear();
  p->ev_used = 0;
  return cuda_check("ace_profile_end");
}

long long ace_debug_fail_alloc(long long k) {
  const long long seen = g_alloc_count.exchange(0);
  g_fail_at.store(k > 0 ? k : 0);
  return seen;
}

ace_status ace_debug_engine_wait(ace_plan* p, unsigned polls, int unreachable) {
  if (!p) return fail(ACE_ERR_ARG, "plan is NULL");
  p->eng_polls = polls ? polls : kEngineSpinDefault;
  p->eng_bias = unreachable ? 1u : 0u;
  drop_graphs(p);   // captured engine launches carry the old limits
  return ACE_OK;
}

ace_status ace_debug_xi_product(ace_plan* p, const void* W, void* Xi_out, int method, void* stream) {
  if (!p) return fail(ACE_ERR_ARG, "plan is NULL");
  if (p->f64) return fail(ACE_ERR_UNSUPPORTED, "complex FP32 plans only");
  if (!W || !Xi_out || !aligned16(W) || !aligned16(Xi_out)) return fail(ACE_ERR_ARG, "W / Xi NULL or unaligned");
  if (method != 1 && method != 2) return fail(ACE_ERR_ARG, "method must be 1 or 2");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return fail(ACE_ERR_ARG, "wrong device");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = p->d.n_occ;
  if (method == 2) {
    launch_outer_f64acc(W, N, p->LinvH, N, p->ld, p->ng, Xi_out, true, st);
    return cuda_check("ace_debug_xi_product");
  }
  void* scratch = nullptr;
  if (dev_alloc(&scratch, xi_oz_scratch_bytes(p->ng, N, N, true)) != cudaSuccess)
    return fail(ACE_ERR_CUDA, "ace_debug_xi_product: out of memory");
  xi_oz_prepare();
  launch_xi_oz(W, N, p->LinvH, N, p->ld, p->ng, Xi_out, true, scratch, p->status, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(scratch);
  if (e != cudaSuccess) return fail(ACE_ERR_CUDA, std::string("ace_debug_xi_product: ") + cudaGetErrorString(e));
  return cuda_check("ace_debug_xi_product");
}

ace_status ace_status_sync(ace_plan* p, void* stream, int* info) {
  if (!p) return fail(ACE_ERR_ARG, "plan is NULL");
  int h[2] = {0, 0};
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("ace_status_sync");
  if (cudaMemcpy(h, p->status, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_check("ace_status_sync");
  cudaMemset(p->status, 0, sizeof(h));
  if (info) *info = h[1];
  if (h[0] == ACE_ERR_NOT_POSDEF) return fail(ACE_ERR_NOT_POSDEF, "-M is not positive definite at pivot " + std::to_string(h[1]));
  if (h[0] == ACE_ERR_NONFINITE) return fail(ACE_ERR_NONFINITE, "non-finite Cholesky pivot " + std::to_string(h[1]));
  if (h[0] == ACE_ERR_TIMEOUT) return fail(ACE_ERR_TIMEOUT, "pair engine wait ran out at task " + std::to_string(h[1]));
  return ACE_OK;
}

}  // extern "C"
