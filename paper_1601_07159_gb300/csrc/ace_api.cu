// C ABI of the ACE hot path: plan creation (kernel table, twiddles, pair-tile
// schedule), workspace sizing and the four entry points of include/ace.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ace.h"
#include "ace_internal.h"

using namespace ace;

namespace {

thread_local std::string g_last_error;

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

}  // namespace

struct ace_plan {
  ace_desc d{};
  int device = 0;
  int n = 0;
  long long ng = 0;
  double vol = 0.0, dv = 0.0;
  bool f64 = false, real = false;
  size_t csize = 0;              // bytes per complex scratch element
  size_t vsize = 0;              // bytes per stored vector element
  int max_pairs = 0, tile = 0;
  std::vector<double> tw;        // 2n doubles, exp(-2 pi i k / n)
  std::vector<Batch> build_batches;
  void* Kt = nullptr;            // kernel table (float or double)
  double* Mc = nullptr;          // 2 N^2, M (complex, row-major)
  double* work = nullptr;        // 4 N^2, Cholesky factor + inverse
  double* LinvH = nullptr;       // 2 N^2, L^{-*}
  int* status = nullptr;         // [code, pivot]
  long long launches = 0;        // kernel launches issued (instrumentation)
  std::vector<cudaEvent_t> ev;   // profiling events (5 per recorded batch)
  size_t ev_used = 0;
  long long ev_dropped = 0;
};

namespace {

// Tournament ("circle") schedule over orbital blocks: every round pairs each
// block with exactly one other, so the tiles of a round write disjoint outputs.
std::vector<Batch> make_sym_schedule(int N, int b, int max_pairs) {
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
    // rotate all but the first entry
    const int last = arr[Bp - 1];
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
  std::vector<Batch> out;
  for (auto& r : rounds) {
    Batch cur{};
    for (auto& t : r) {
      const int np = tile_pairs(t);
      if (cur.ntiles > 0 && (cur.npairs + np > max_pairs || cur.ntiles == kMaxTiles)) {
        out.push_back(cur);
        cur = Batch{};
      }
      t.slot0 = cur.npairs;
      cur.t[cur.ntiles++] = t;
      cur.npairs += np;
    }
    if (cur.ntiles > 0) out.push_back(cur);
  }
  return out;
}

// One-sided schedule for V_X[Phi] Psi: r-blocks of Psi (<= b), l-chunks of Phi;
// a batch holds tiles of one l-chunk, so its tiles write distinct Psi blocks.
std::vector<Batch> make_rect_schedule(int N, int nb, int b, int max_pairs) {
  std::vector<Batch> out;
  const int nrb = (nb + b - 1) / b;
  int lc = max_pairs / b;
  if (lc < 1) lc = 1;
  if (lc > N) lc = N;
  for (int l0 = 0; l0 < N; l0 += lc) {
    const int nl = (l0 + lc <= N) ? lc : N - l0;
    Batch cur{};
    for (int R = 0; R < nrb; ++R) {
      TileDesc t{};
      t.l0 = l0;
      t.nl = nl;
      t.r0 = R * b;
      t.nr = (R * b + b <= nb) ? b : nb - R * b;
      t.kind = 2;
      const int np = tile_pairs(t);
      if (cur.ntiles > 0 && (cur.npairs + np > max_pairs || cur.ntiles == kMaxTiles)) {
        out.push_back(cur);
        cur = Batch{};
      }
      t.slot0 = cur.npairs;
      cur.t[cur.ntiles++] = t;
      cur.npairs += np;
    }
    if (cur.ntiles > 0) out.push_back(cur);
  }
  return out;
}

struct WsLayout {
  char* S = nullptr;
  double* Epart = nullptr;
  double* part = nullptr;
  double* Cm = nullptr;
  char* Wtmp = nullptr;
  size_t total = 0;
};

int epart_count(const ace_plan* p) { return energy_blocks(p->n, p->max_pairs, p->f64) + 1; }

WsLayout layout(const ace_plan* p, int op, int nb, char* base) {
  WsLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) { char* r = base ? base + off : nullptr; off += align256(bytes); return r; };
  const int N = p->d.n_occ;
  const int splits = gram_splits(p->ng);
  if (op == ACE_OP_EXCHANGE_APPLY || op == ACE_OP_BUILD || op == ACE_OP_ENERGY_GRAD)
    L.S = take((size_t)p->max_pairs * p->ng * p->csize);
  if (op == ACE_OP_ENERGY_GRAD) L.Epart = (double*)take((size_t)epart_count(p) * sizeof(double));
  if (op == ACE_OP_BUILD) {
    L.part = (double*)take((size_t)splits * N * N * 2 * sizeof(double));
    L.Wtmp = take((size_t)N * p->ng * p->vsize);
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

bool launch_batch(ace_plan* p, const PairLaunch& L0, const Batch& b, cudaStream_t st) {
  PairLaunch L = L0;
  L.ev = nullptr;
  if (!p->ev.empty()) {
    if (p->ev_used + 5 <= p->ev.size()) {
      L.ev = &p->ev[p->ev_used];
      p->ev_used += 5;
    } else {
      ++p->ev_dropped;
    }
  }
  p->launches += pair_batch_launches(L.mode);
  return p->f64 ? launch_pair_batch_f64(L, b, st) : launch_pair_batch_f32(L, b, st);
}

PairLaunch base_launch(const ace_plan* p) {
  PairLaunch L{};
  L.n = p->n;
  L.ld = p->ng;
  L.Kt = p->Kt;
  L.tw = p->tw.data();
  L.real_io = p->real;
  L.scale = 1.0;
  return L;
}

}  // namespace

ace_status ace_internal_plan_info(const ace_plan* p, int* device, int* n_occ, long long* ng,
                                  double* dv, int* f64, int* real) {
  *device = p->device;
  *n_occ = p->d.n_occ;
  *ng = p->ng;
  *dv = p->dv;
  *f64 = p->f64 ? 1 : 0;
  *real = p->real ? 1 : 0;
  return ACE_OK;
}

ace_status ace_internal_set_error(ace_status s, const char* msg) { return fail(s, msg); }

extern "C" {

int ace_supported_edge(int n, int dtype) {
  if (dtype == ACE_DTYPE_C64) return pair_edge_supported_f32(n) ? 1 : 0;
  if (dtype == ACE_DTYPE_C128 || dtype == ACE_DTYPE_R64) return pair_edge_supported_f64(n) ? 1 : 0;
  return 0;
}

const char* ace_last_error(void) { return g_last_error.c_str(); }

ace_status ace_plan_create(const ace_desc* d, ace_plan** out) {
  if (!out) return fail(ACE_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!d) return fail(ACE_ERR_ARG, "desc is NULL");
  if (d->dtype < ACE_DTYPE_R64 || d->dtype > ACE_DTYPE_C64) return fail(ACE_ERR_ARG, "bad dtype");
  if (d->kernel != ACE_KERNEL_BARE && d->kernel != ACE_KERNEL_ERFC) return fail(ACE_ERR_ARG, "bad kernel");
  if (d->n_occ < 1) return fail(ACE_ERR_ARG, "n_occ must be >= 1");
  if (!(d->L[0] > 0 && d->L[1] > 0 && d->L[2] > 0)) return fail(ACE_ERR_ARG, "cell edges must be > 0");
  if (d->kernel == ACE_KERNEL_ERFC && !(d->omega > 0)) return fail(ACE_ERR_ARG, "omega must be > 0");
  if (!std::isfinite(d->alpha)) return fail(ACE_ERR_ARG, "alpha must be finite");
  if (!ace_supported_edge(d->n, d->dtype))
    return fail(ACE_ERR_UNSUPPORTED, "grid edge " + std::to_string(d->n) + " not built for this dtype");
  if (d->tile < 0 || d->tile > kTileMax) return fail(ACE_ERR_ARG, "tile must be 0..8");
  if (d->max_pairs < 0) return fail(ACE_ERR_ARG, "max_pairs must be >= 0");

  ace_plan* p = new ace_plan();
  p->d = *d;
  cudaGetDevice(&p->device);
  p->n = d->n;
  p->ng = (long long)d->n * d->n * d->n;
  p->vol = d->L[0] * d->L[1] * d->L[2];
  p->dv = p->vol / (double)p->ng;
  p->f64 = d->dtype != ACE_DTYPE_C64;
  p->real = d->dtype == ACE_DTYPE_R64;
  p->csize = p->f64 ? 16 : 8;
  p->vsize = p->real ? 8 : p->csize;
  p->tile = d->tile ? d->tile : kTileMax;
  const size_t slot = (size_t)p->ng * p->csize;
  if (d->max_pairs) {
    p->max_pairs = d->max_pairs;
  } else {
    const long long budget = (512ll << 20) / (long long)slot;
    p->max_pairs = (int)(budget > 1 ? budget : 1);
    const long long total = (long long)d->n_occ * (d->n_occ + 1) / 2;
    if (p->max_pairs > total) p->max_pairs = (int)total;
  }
  if (p->max_pairs < p->tile * p->tile) p->max_pairs = p->tile * p->tile;

  // twiddles exp(-2 pi i k/n) in FP64
  const int n = p->n;
  p->tw.resize(2 * n);
  for (int k = 0; k < n; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)n;
    p->tw[2 * k] = std::cos(a);
    p->tw[2 * k + 1] = -std::sin(a);
  }
  // kernel table K(G) alpha / N_g in the spectrum layout [kz][kx][ky]
  const double g0_default = d->kernel == ACE_KERNEL_BARE ? 0.0 : M_PI / (d->omega * d->omega);
  const double g0 = std::isnan(d->g0_value) ? g0_default : d->g0_value;
  std::vector<double> kt((size_t)p->ng);
  auto freq = [n](int i) { return (i <= n / 2) ? i : i - n; };   // |G| symmetric at n/2
  for (int kz = 0; kz < n; ++kz)
    for (int kx = 0; kx < n; ++kx)
      for (int ky = 0; ky < n; ++ky) {
        const double gx = 2.0 * M_PI * freq(kx) / d->L[0];
        const double gy = 2.0 * M_PI * freq(ky) / d->L[1];
        const double gz = 2.0 * M_PI * freq(kz) / d->L[2];
        const double g2 = gx * gx + gy * gy + gz * gz;
        double k;
        if (g2 == 0.0) k = g0;
        else if (d->kernel == ACE_KERNEL_BARE) k = 4.0 * M_PI / g2;
        else k = 4.0 * M_PI / g2 * (1.0 - std::exp(-g2 / (4.0 * d->omega * d->omega)));
        kt[((size_t)kz * n + kx) * n + ky] = d->alpha * k / (double)p->ng;
      }
  const int N = d->n_occ;
  cudaError_t e = cudaSuccess;
  if (p->f64) {
    e = cudaMalloc(&p->Kt, kt.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(p->Kt, kt.data(), kt.size() * sizeof(double), cudaMemcpyHostToDevice);
  } else {
    std::vector<float> kf(kt.begin(), kt.end());
    e = cudaMalloc(&p->Kt, kf.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(p->Kt, kf.data(), kf.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMalloc(&p->Mc, (size_t)2 * N * N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&p->work, (size_t)4 * N * N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&p->LinvH, (size_t)2 * N * N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&p->status, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->status, 0, 2 * sizeof(int));
  if (e != cudaSuccess) {
    std::string m = std::string("plan allocation: ") + cudaGetErrorString(e);
    ace_plan_destroy(p);
    return fail(ACE_ERR_CUDA, m);
  }
  p->build_batches = make_sym_schedule(N, p->tile, p->max_pairs);
  *out = p;
  return ACE_OK;
}

ace_status ace_plan_destroy(ace_plan* p) {
  if (!p) return ACE_OK;
  cudaDeviceSynchronize();
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  cudaFree(p->Kt);
  cudaFree(p->Mc);
  cudaFree(p->work);
  cudaFree(p->LinvH);
  cudaFree(p->status);
  delete p;
  return ACE_OK;
}

size_t ace_workspace_size(const ace_plan* p, int op, int nb) {
  if (!p || op < ACE_OP_EXCHANGE_APPLY || op > ACE_OP_ENERGY_GRAD) return 0;
  if ((op == ACE_OP_EXCHANGE_APPLY || op == ACE_OP_APPLY) && nb < 0) return 0;
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
  cudaMemsetAsync(Y, 0, (size_t)nb * p->ng * p->vsize, st);
  PairLaunch L = base_launch(p);
  L.X = Phi;
  L.Y = Psi;
  L.OutX = nullptr;
  L.OutY = Y;
  L.S = W.S;
  L.mode = 0;
  for (const Batch& b : make_rect_schedule(p->d.n_occ, nb, p->tile, p->max_pairs))
    if (!launch_batch(p, L, b, st)) return fail(ACE_ERR_UNSUPPORTED, "edge not built");
  return cuda_check("ace_exchange_apply");
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
  cudaMemsetAsync(W, 0, (size_t)N * p->ng * p->vsize, st);
  cudaMemsetAsync(p->status, 0, 2 * sizeof(int), st);
  // W = V_X[Phi] Phi over the unique pairs (Eq. W)
  PairLaunch L = base_launch(p);
  L.X = Phi;
  L.Y = Phi;
  L.OutX = W;
  L.OutY = W;
  L.S = Wl.S;
  L.mode = 0;
  for (const Batch& b : p->build_batches)
    if (!launch_batch(p, L, b, st)) return fail(ACE_ERR_UNSUPPORTED, "edge not built");
  // M = dV Phi^* W, Hermitian part (Eq. ACEconstruct2); E_x = 1/2 Re tr M
  const int splits = gram_splits(p->ng);
  launch_gram(p->f64, p->real, Phi, N, W, N, p->ng, p->ng, Wl.part, splits, st);
  launch_gram_reduce(Wl.part, splits, N, N, p->dv, true, false, p->Mc, Ex_out, st);
  if (M_out) launch_gram_reduce(Wl.part, splits, N, N, p->dv, true, p->real, M_out, nullptr, st);
  // -M = L L^* and L^{-*} in FP64; Xi = W L^{-*} (Eq. Wtilde)
  launch_cholesky_inv(p->Mc, N, p->work, p->LinvH, p->status, st);
  launch_outer(p->f64, p->real, W, N, p->LinvH, N, p->ng, p->ng, 1.0, Xi_out, st);
  p->launches += 2 + (Ex_out ? 1 : 0) + (M_out ? 1 : 0) + 2 + 1;
  return cuda_check("ace_build");
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
  const int splits = gram_splits(p->ng);
  // C = dV Xi^* Psi, Y = -Xi C (Eq. ACE)
  launch_gram(p->f64, p->real, Xi, N, Psi, nb, p->ng, p->ng, Wl.part, splits, st);
  launch_gram_reduce(Wl.part, splits, N, nb, p->dv, false, false, Wl.Cm, nullptr, st);
  launch_outer(p->f64, p->real, Xi, N, Wl.Cm, nb, p->ng, p->ng, -1.0, Y, st);
  p->launches += 3;
  return cuda_check("ace_apply");
}

ace_status ace_exchange_energy_grad(ace_plan* p, const void* Phi, double* Ex_out, void* grad_out,
                                    double grad_scale, void* ws, size_t ws_bytes, void* stream) {
  ace_status s = check_common(p, ws, ws_bytes, ACE_OP_ENERGY_GRAD, 0);
  if (s != ACE_OK) return s;
  if (!Phi || !Ex_out) return fail(ACE_ERR_ARG, "Phi and Ex_out are required");
  if (!aligned16(Phi) || (grad_out && !aligned16(grad_out))) return fail(ACE_ERR_ARG, "vectors must be 16-byte aligned");
  if (grad_out == Phi) return fail(ACE_ERR_ARG, "grad_out must not alias Phi");
  if (!std::isfinite(grad_scale)) return fail(ACE_ERR_ARG, "grad_scale must be finite");
  cudaStream_t st = (cudaStream_t)stream;
  const int N = p->d.n_occ;
  const WsLayout Wl = layout(p, ACE_OP_ENERGY_GRAD, 0, (char*)ws);
  const int ecount = epart_count(p);
  cudaMemsetAsync(Wl.Epart, 0, (size_t)ecount * sizeof(double), st);
  if (grad_out) cudaMemsetAsync(grad_out, 0, (size_t)N * p->ng * p->vsize, st);
  PairLaunch L = base_launch(p);
  L.X = Phi;
  L.Y = Phi;
  L.OutX = grad_out;
  L.OutY = grad_out;
  L.S = Wl.S;
  L.Epart = Wl.Epart;
  L.mode = grad_out ? 2 : 1;
  L.scale = 2.0 * p->dv * grad_scale;     // grad = grad_scale * 2 dV W
  for (const Batch& b : p->build_batches)
    if (!launch_batch(p, L, b, st)) return fail(ACE_ERR_UNSUPPORTED, "edge not built");
  // E = -1/2 Omega/N_g sum_pairs w_p sum_G Kt |F rho|^2  (Kt = alpha K / N_g)
  launch_energy_reduce(Wl.Epart, ecount, -0.5 * p->vol / (double)p->ng, Ex_out, st);
  p->launches += 1;
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
  p->launches = 0;
  return ACE_OK;
}

ace_status ace_profile_end(ace_plan* p, double* ms_out, long long* counts_out) {
  if (!p) return fail(ACE_ERR_ARG, "plan is NULL");
  if (cudaDeviceSynchronize() != cudaSuccess) return cuda_check("ace_profile_end");
  double ms[5] = {0, 0, 0, 0, 0};
  const size_t batches = p->ev_used / 5;
  for (size_t b = 0; b < batches; ++b) {
    for (int k = 0; k < 4; ++k) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p->ev[5 * b + k], p->ev[5 * b + k + 1]) == cudaSuccess) ms[k] += t;
    }
  }
  ms[4] = ms[0] + ms[1] + ms[2] + ms[3];
  if (ms_out)
    for (int k = 0; k < 5; ++k) ms_out[k] = ms[k];
  if (counts_out) {
    counts_out[0] = (long long)batches;
    counts_out[1] = p->launches;
    counts_out[2] = p->ev_dropped;
  }
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  p->ev.clear();
  p->ev_used = 0;
  return cuda_check("ace_profile_end");
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
  return ACE_OK;
}

}  // extern "C"
