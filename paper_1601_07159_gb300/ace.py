"""ctypes binding over the C ABI of include/ace.h.

Argument marshalling only: every step of the exchange / ACE path runs in the
CUDA kernels of libace.so. PyTorch supplies device memory and the current
stream. Importing this module loads the library and raises ImportError when it
has not been built (``paper_1601_07159_gb300.build_lib``); there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libace.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libace.so not built ({LIB_PATH}); run python -m paper_1601_07159_gb300.build_lib")
_lib = ctypes.CDLL(LIB_PATH)

ACE_OK = 0
ACE_ERR_ARG = -1
ACE_ERR_NOT_POSDEF = -2
ACE_ERR_NONFINITE = -3
ACE_ERR_WORKSPACE = -4
ACE_ERR_CUDA = -5
ACE_ERR_TIMEOUT = -6
ACE_ERR_UNSUPPORTED = -7

DTYPES = {"r64": 0, "c128": 1, "c64": 2}
TORCH_DTYPES = {"r64": torch.float64, "c128": torch.complex128, "c64": torch.complex64}
KERNELS = {"bare": 0, "erfc": 1, "kinetic": 2}
OP_EXCHANGE_APPLY, OP_BUILD, OP_APPLY, OP_ENERGY_GRAD, OP_BUILD_OVERSAMPLED, OP_POISSON = 0, 1, 2, 3, 4, 5
OP_ENERGY_GRAD_STORE = 6


PRECS = {"default": 0, "split_tf32": 1, "fp32": 2, "xi_fp64": 3, "xi_fp64_simt": 4, "split_bf16": 5}


class Desc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("L", ctypes.c_double * 3),
        ("n_occ", ctypes.c_int),
        ("dtype", ctypes.c_int),
        ("prec", ctypes.c_int),
        ("kernel", ctypes.c_int),
        ("omega", ctypes.c_double),
        ("g0_value", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("ld", ctypes.c_longlong),
        ("max_pairs", ctypes.c_int),
        ("tile", ctypes.c_int),
        ("lanes", ctypes.c_int),
        ("flags", ctypes.c_int),
    ]


def _grid(n):
    """(n_x, n_y, n_z) from an edge or a 3-sequence."""
    if isinstance(n, int):
        return (n, n, n)
    n = tuple(int(v) for v in n)
    if len(n) != 3:
        raise ValueError("grid must be an int or three ints (n_x, n_y, n_z)")
    return n


_vp = ctypes.c_void_p
_lib.ace_supported_edge.argtypes = [ctypes.c_int, ctypes.c_int]
_lib.ace_supported_edge.restype = ctypes.c_int
_lib.ace_supported_grid.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_int]
_lib.ace_supported_grid.restype = ctypes.c_int
_lib.ace_last_error.argtypes = []
_lib.ace_last_error.restype = ctypes.c_char_p
_lib.ace_plan_create.argtypes = [ctypes.POINTER(Desc), ctypes.POINTER(_vp)]
_lib.ace_plan_create.restype = ctypes.c_int
_lib.ace_plan_destroy.argtypes = [_vp]
_lib.ace_plan_destroy.restype = ctypes.c_int
_lib.ace_workspace_size.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
_lib.ace_workspace_size.restype = ctypes.c_size_t
_lib.ace_exchange_apply.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_size_t, _vp]
_lib.ace_exchange_apply.restype = ctypes.c_int
_lib.ace_build.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]
_lib.ace_build.restype = ctypes.c_int
_lib.ace_apply.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_size_t, _vp]
_lib.ace_apply.restype = ctypes.c_int
_lib.ace_exchange_energy_grad.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _vp, ctypes.c_size_t,
                                          _vp]
_lib.ace_exchange_energy_grad.restype = ctypes.c_int
_lib.ace_status_sync.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_int)]
_lib.ace_status_sync.restype = ctypes.c_int
_lib.ace_apply_static.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp]
_lib.ace_apply_static.restype = ctypes.c_int
_lib.ace_profile_begin.argtypes = [_vp, ctypes.c_int]
_lib.ace_profile_begin.restype = ctypes.c_int
_lib.ace_profile_end.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
_lib.ace_profile_end.restype = ctypes.c_int
_lib.ace_build_oversampled.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]
_lib.ace_build_oversampled.restype = ctypes.c_int
_lib.ace_poisson.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_size_t, _vp]
_lib.ace_poisson.restype = ctypes.c_int
_lib.ace_workspace_size_batched.argtypes = [ctypes.POINTER(_vp), ctypes.c_int]
_lib.ace_workspace_size_batched.restype = ctypes.c_size_t
_lib.ace_build_batched.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp,
                                   ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _vp]
_lib.ace_build_batched.restype = ctypes.c_int
_lib.ace_autotune.argtypes = [ctypes.POINTER(Desc), ctypes.c_int, ctypes.POINTER(Desc),
                              ctypes.POINTER(ctypes.c_double)]
_lib.ace_autotune.restype = ctypes.c_int
_lib.ace_tuning_register.argtypes = [ctypes.POINTER(Desc)]
_lib.ace_tuning_register.restype = ctypes.c_int
_lib.ace_tuning_clear.argtypes = []
_lib.ace_tuning_clear.restype = ctypes.c_int
_lib.ace_plan_desc.argtypes = [_vp, ctypes.POINTER(Desc)]
_lib.ace_plan_desc.restype = ctypes.c_int
_lib.ace_debug_engine_wait.argtypes = [_vp, ctypes.c_uint, ctypes.c_int]
_lib.ace_debug_engine_wait.restype = ctypes.c_int
_lib.ace_debug_xi_product.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp]
_lib.ace_debug_xi_product.restype = ctypes.c_int
_lib.ace_debug_fail_alloc.argtypes = [ctypes.c_longlong]
_lib.ace_debug_fail_alloc.restype = ctypes.c_longlong


class AceError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ace error {code}: {msg}")
        self.code = code


def _check(code: int):
    if code != ACE_OK:
        raise AceError(code, _lib.ace_last_error().decode())


def supported_edge(n: int, dtype: str) -> bool:
    return bool(_lib.ace_supported_edge(n, DTYPES[dtype]))


def supported_grid(n, dtype: str) -> bool:
    g = (ctypes.c_int * 3)(*_grid(n))
    return bool(_lib.ace_supported_grid(g, DTYPES[dtype]))


def lib():
    """The loaded ctypes library (for tests that call the C ABI directly)."""
    return _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Plan:
    """An ACE plan on the current CUDA device (see ace_plan_create)."""

    def __init__(self, n, L, n_occ: int, dtype: str = "c64", kernel: str = "bare",
                 omega: float = 0.0, g0: float | None = None, alpha: float = 1.0,
                 max_pairs: int = 0, tile: int = 0, lanes: int = 0, graphs: bool = True,
                 engine: bool = False, pdl: bool = True, tensor_cores: bool = True,
                 overlap: bool = True, prec: str = "default", ld: int = 0, radix: int = 0):
        """n: grid edge or (n_x, n_y, n_z); L: cell edge or (L_x, L_y, L_z);
        ld: elements from one vector to the next (0 = N_g); radix: order of
        the FP32 line transforms (0: radix 4 first, 1: odd radix first)."""
        if isinstance(L, (int, float)):
            L = (float(L),) * 3
        grid = _grid(n)
        d = Desc()
        d.n[0], d.n[1], d.n[2] = grid
        d.L[0], d.L[1], d.L[2] = L
        d.n_occ = n_occ
        d.dtype = DTYPES[dtype]
        d.prec = PRECS[prec]
        d.kernel = KERNELS[kernel]
        d.omega = omega
        d.g0_value = math.nan if g0 is None else g0
        d.alpha = alpha
        d.ld = ld
        d.max_pairs = max_pairs
        d.tile = tile
        d.lanes = lanes
        d.flags = ((0 if graphs else 1) | (2 if engine else 0) | (0 if pdl else 4) | (0 if tensor_cores else 8) |
                   (0 if overlap else 16) | (32 if radix else 0))
        self.schedule = {"tile": tile, "max_pairs": max_pairs, "lanes": lanes, "overlap": overlap, "radix": radix}
        h = _vp()
        _check(_lib.ace_plan_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.grid = grid
        self.n = grid[0] if grid[0] == grid[1] == grid[2] else grid
        self.L, self.n_occ, self.dtype = tuple(L), n_occ, dtype
        self.ng = grid[0] * grid[1] * grid[2]
        self.ld = ld if ld else self.ng
        self.shape = (grid[2], grid[1], grid[0])     # [z][y][x]
        self.volume = L[0] * L[1] * L[2]
        self.dv = self.volume / self.ng
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.tdtype = TORCH_DTYPES[dtype]
        self._ws = {}

    def close(self):
        if getattr(self, "_h", None):
            _lib.ace_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- helpers
    def workspace_size(self, op: int, n_b: int = 0) -> int:
        return int(_lib.ace_workspace_size(self._h, op, n_b))

    def workspace(self, op: int, n_b: int = 0) -> torch.Tensor:
        nbytes = max(self.workspace_size(op, n_b), 256)
        ws = self._ws.get(op)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self._ws[op] = ws
        return ws

    def _vec(self, t: torch.Tensor, name: str) -> torch.Tensor:
        if t.dtype != self.tdtype:
            raise TypeError(f"{name}: expected {self.tdtype}, got {t.dtype}")
        if t.device != self.device:
            raise ValueError(f"{name}: expected device {self.device}")
        if t.dim() != 4 or tuple(t.shape[1:]) != self.shape:
            raise ValueError(f"{name}: expected shape (count, {self.shape[0]}, {self.shape[1]}, {self.shape[2]})")
        nz, ny, nx = self.shape
        want = (self.ld, ny * nx, nx, 1)
        if t.shape[0] > 1 and t.stride() != want or t.shape[0] <= 1 and t.stride()[1:] != want[1:]:
            raise ValueError(f"{name}: expected strides {want} (vectors {self.ld} elements apart)")
        return t

    def empty(self, count: int) -> torch.Tensor:
        """`count` vectors of the plan's layout: (count, n_z, n_y, n_x), vectors ld
        elements apart."""
        if self.ld == self.ng:
            return torch.empty((count,) + self.shape, dtype=self.tdtype, device=self.device)
        flat = torch.empty((max(count, 1), self.ld), dtype=self.tdtype, device=self.device)
        nz, ny, nx = self.shape
        return flat.as_strided((count,) + self.shape, (self.ld, ny * nx, nx, 1))

    # ---------------------------------------------------------------- entry points
    def exchange_apply(self, phi, psi, out=None):
        """Y = V_X[phi] psi (Eq. applyVX2)."""
        self._vec(phi, "phi")
        self._vec(psi, "psi")
        nb = psi.shape[0]
        y = self.empty(nb) if out is None else self._vec(out, "out")
        ws = self.workspace(OP_EXCHANGE_APPLY, nb)
        _check(_lib.ace_exchange_apply(self._h, _ptr(phi), _ptr(psi), nb, _ptr(y), _ptr(ws),
                                       ws.numel(), _stream()))
        return y

    def build(self, phi, want_w: bool = True, want_m: bool = True, xi=None, w=None):
        """ACE construction: W, M, Xi and E_x = 1/2 Re tr M (Alg. 2 steps 2-3)."""
        self._vec(phi, "phi")
        N = self.n_occ
        if phi.shape[0] != N:
            raise ValueError("phi must hold n_occ vectors")
        xi = self.empty(N) if xi is None else self._vec(xi, "xi")
        if want_w and w is None:
            w = self.empty(N)
        m = None
        if want_m:
            mshape = (N, N) if self.dtype == "r64" else (N, N, 2)
            m = torch.empty(mshape, dtype=torch.float64, device=self.device)
        ex = torch.empty((), dtype=torch.float64, device=self.device)
        ws = self.workspace(OP_BUILD)
        _check(_lib.ace_build(self._h, _ptr(phi), _ptr(w), _ptr(xi), _ptr(m), _ptr(ex), _ptr(ws),
                              ws.numel(), _stream()))
        if m is not None and self.dtype != "r64":
            m = torch.view_as_complex(m)
        return {"Xi": xi, "W": w, "M": m, "Ex": ex}

    def build_oversampled(self, phi, want_w: bool = True, want_m: bool = True, xi=None, w=None):
        """ACE with oversampling (Sec. 3): phi holds N_phi >= n_occ orbitals, the
        n_occ occupied ones first; V_X is that of the occupied ones and Xi has
        N_phi vectors. E_x is that of the occupied block."""
        self._vec(phi, "phi")
        n_phi = phi.shape[0]
        if n_phi < self.n_occ:
            raise ValueError("phi must hold at least n_occ vectors")
        xi = self.empty(n_phi) if xi is None else self._vec(xi, "xi")
        if want_w and w is None:
            w = self.empty(n_phi)
        m = None
        if want_m:
            mshape = (n_phi, n_phi) if self.dtype == "r64" else (n_phi, n_phi, 2)
            m = torch.empty(mshape, dtype=torch.float64, device=self.device)
        ex = torch.empty((), dtype=torch.float64, device=self.device)
        ws = self.workspace(OP_BUILD_OVERSAMPLED, n_phi)
        _check(_lib.ace_build_oversampled(self._h, _ptr(phi), n_phi, _ptr(w), _ptr(xi), _ptr(m), _ptr(ex),
                                          _ptr(ws), ws.numel(), _stream()))
        if m is not None and self.dtype != "r64":
            m = torch.view_as_complex(m)
        return {"Xi": xi, "W": w, "M": m, "Ex": ex}

    def poisson(self, rho, out=None):
        """V_b = sum_G K(G) rho_hat_b(G) e^{iG.r} with the plan's kernel: the
        Hartree potential of Eq. HF for the bare kernel and the density."""
        self._vec(rho, "rho")
        nb = rho.shape[0]
        v = self.empty(nb) if out is None else self._vec(out, "out")
        ws = self.workspace(OP_POISSON, nb)
        _check(_lib.ace_poisson(self._h, _ptr(rho), nb, _ptr(v), _ptr(ws), ws.numel(), _stream()))
        return v

    def apply(self, xi, psi, out=None):
        """Y = V_ACE psi = -Xi (dV Xi^* psi) (Eq. ACE)."""
        self._vec(xi, "xi")
        self._vec(psi, "psi")
        nb = psi.shape[0]
        y = self.empty(nb) if out is None else self._vec(out, "out")
        ws = self.workspace(OP_APPLY, nb)
        _check(_lib.ace_apply(self._h, _ptr(xi), _ptr(psi), nb, _ptr(y), _ptr(ws), ws.numel(),
                              _stream()))
        return y

    def apply_static(self, xi, psi, out):
        """ace_apply_static: the apply without a workspace (the library's own
        static device scratch; calls on one device must not overlap)."""
        self._vec(xi, "xi")
        self._vec(psi, "psi")
        self._vec(out, "out")
        _check(_lib.ace_apply_static(self._h, _ptr(xi), _ptr(psi), psi.shape[0], _ptr(out), _stream()))
        return out

    def energy_grad(self, phi, grad: bool = False, grad_scale: float = 1.0, out=None, recompute: bool = True):
        """E_x (Eq. EX) and optionally grad_scale * 2 dV W. With recompute=False
        the plan's store workspace keeps the pair potentials: a call without
        grad stores them, a later call with grad (same phi) uses them."""
        self._vec(phi, "phi")
        ex = torch.empty((), dtype=torch.float64, device=self.device)
        g = None
        if grad:
            g = self.empty(self.n_occ) if out is None else self._vec(out, "out")
        ws = self.workspace(OP_ENERGY_GRAD if recompute else OP_ENERGY_GRAD_STORE)
        _check(_lib.ace_exchange_energy_grad(self._h, _ptr(phi), _ptr(ex), _ptr(g), grad_scale,
                                             1 if recompute else 0, _ptr(ws), ws.numel(), _stream()))
        return ex, g

    def profile_begin(self, max_events: int = 4096):
        _check(_lib.ace_profile_begin(self._h, max_events))

    def profile_end(self) -> dict:
        """Pass durations (ms) over the recorded batches and the launch count."""
        ms = (ctypes.c_double * 5)()
        cnt = (ctypes.c_longlong * 3)()
        _check(_lib.ace_profile_end(self._h, ms, cnt))
        return {"pass_ms": {"A": ms[0], "B": ms[1], "C": ms[2], "D": ms[3]}, "pair_ms": ms[4],
                "batches": cnt[0], "launches": cnt[1], "dropped": cnt[2]}

    def effective_schedule(self) -> dict:
        """The schedule the plan runs (after any registered tuned schedule)."""
        d = Desc()
        _check(_lib.ace_plan_desc(self._h, ctypes.byref(d)))
        return {"tile": d.tile, "max_pairs": d.max_pairs, "lanes": d.lanes, "overlap": not (d.flags & 16),
                "radix": 1 if d.flags & 32 else 0, "ld": d.ld}

    def debug_engine_wait(self, polls: int = 0, unreachable: bool = False):
        """ace_debug_engine_wait: bound (or make unreachable) the engine's waits."""
        _check(_lib.ace_debug_engine_wait(self._h, polls, 1 if unreachable else 0))

    def debug_xi_product(self, w, method: int):
        """ace_debug_xi_product: Xi = W L^{-*} of the last build in FP64 (complex128),
        method 1 = tensor-core slices, 2 = FP64 CUDA cores."""
        self._vec(w, "w")
        out = torch.empty((self.n_occ, self.ld), dtype=torch.complex128, device=self.device)
        _check(_lib.ace_debug_xi_product(self._h, _ptr(w), _ptr(out), method, _stream()))
        nz, ny, nx = self.shape
        return out.as_strided((self.n_occ,) + self.shape, (self.ld, ny * nx, nx, 1))

    def status(self) -> tuple[int, int]:
        """(code, pivot) of the device status word after synchronising."""
        info = ctypes.c_int(0)
        code = _lib.ace_status_sync(self._h, _stream(), ctypes.byref(info))
        return code, info.value


def debug_fail_alloc(k: int) -> int:
    """ace_debug_fail_alloc: make the k-th library allocation from now fail
    (k <= 0: off); returns the allocations counted since the previous call."""
    return int(_lib.ace_debug_fail_alloc(k))


def _desc(n, L, n_occ, dtype, kernel, omega, g0, alpha) -> Desc:
    if isinstance(L, (int, float)):
        L = (float(L),) * 3
    d = Desc()
    d.n[0], d.n[1], d.n[2] = _grid(n)
    d.L[0], d.L[1], d.L[2] = L
    d.n_occ = n_occ
    d.dtype = DTYPES[dtype]
    d.kernel = KERNELS[kernel]
    d.omega = omega
    d.g0_value = math.nan if g0 is None else g0
    d.alpha = alpha
    return d


def autotune(n: int, L, n_occ: int, dtype: str = "c64", kernel: str = "bare", omega: float = 0.0,
             g0: float | None = None, alpha: float = 1.0, reps: int = 3) -> dict:
    """ace_autotune: the fastest schedule for this problem shape on the current
    device, as Plan keyword arguments plus the measured ms per build."""
    d = _desc(n, L, n_occ, dtype, kernel, omega, g0, alpha)
    best = Desc()
    ms = ctypes.c_double(0.0)
    _check(_lib.ace_autotune(ctypes.byref(d), reps, ctypes.byref(best), ctypes.byref(ms)))
    return {"tile": best.tile, "max_pairs": best.max_pairs, "lanes": best.lanes,
            "overlap": not (best.flags & 16), "radix": 1 if best.flags & 32 else 0, "ms": ms.value}


def tuning_register(n, L, n_occ: int, dtype: str, kernel: str, tile: int, max_pairs: int, lanes: int,
                    overlap: bool, omega: float = 0.0, prec: str = "default", radix: int = 0):
    """ace_tuning_register: later plans of this problem with default schedule
    knobs run this schedule."""
    d = _desc(n, L, n_occ, dtype, kernel, omega, None, 1.0)
    d.prec = PRECS[prec]
    d.tile, d.max_pairs, d.lanes = tile, max_pairs, lanes
    d.flags = (0 if overlap else 16) | (32 if radix else 0)
    _check(_lib.ace_tuning_register(ctypes.byref(d)))


def tuning_clear():
    _check(_lib.ace_tuning_clear())


class TuningTable:
    """Autotuner results keyed by problem shape (n, N, dtype, kernel), kept in
    a JSON file so that a shape is timed once per machine. Loading a table
    registers its entries with the library, so plans created with the default
    schedule knobs run the tuned schedules."""

    def __init__(self, path: str | None = None):
        self.path = path
        self.table = {}
        if path and os.path.exists(path):
            import json
            with open(path) as f:
                self.table = json.load(f)
            for k, t in self.table.items():
                n, n_occ, dtype, kernel = k.split("|")
                tuning_register(tuple(int(v) for v in n.split("x")), 1.0, int(n_occ), dtype, kernel,
                                t["tile"], t["max_pairs"], t["lanes"], t["overlap"], radix=t.get("radix", 0))

    @staticmethod
    def key(n, n_occ, dtype, kernel) -> str:
        """'n_x x n_y x n_z|N|dtype|kernel', e.g. '48x48x48|128|c64|erfc'."""
        return "x".join(str(v) for v in _grid(n)) + f"|{n_occ}|{dtype}|{kernel}"

    def schedule(self, n, L, n_occ, dtype="c64", kernel="bare", omega=0.0, g0=None, alpha=1.0) -> dict:
        k = self.key(n, n_occ, dtype, kernel)
        if k not in self.table:
            self.table[k] = autotune(n, L, n_occ, dtype, kernel, omega, g0, alpha)
            if self.path:
                import json
                os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
                with open(self.path, "w") as f:
                    json.dump(self.table, f, indent=1, sort_keys=True)
        return self.table[k]

    def plan(self, n, L, n_occ, dtype="c64", kernel="bare", omega=0.0, g0=None, alpha=1.0) -> "Plan":
        t = self.schedule(n, L, n_occ, dtype, kernel, omega, g0, alpha)
        return Plan(n, L, n_occ, dtype=dtype, kernel=kernel, omega=omega, g0=g0, alpha=alpha,
                    tile=t["tile"], max_pairs=t["max_pairs"], lanes=t["lanes"], overlap=t["overlap"],
                    radix=t.get("radix", 0))


class Batch:
    """ace_build_batched over a fixed list of plans (one per system), with the
    batch workspace allocated once so that the captured graph is replayed."""

    def __init__(self, plans, chains: int = 0):
        self.plans = list(plans)
        self.chains = chains
        n = len(self.plans)
        self._hp = (_vp * n)(*[p._h for p in self.plans])
        nbytes = int(_lib.ace_workspace_size_batched(self._hp, n))
        self.ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.plans[0].device) if n else None
        self.ex = torch.empty(n, dtype=torch.float64, device=self.plans[0].device) if n else None

    def build(self, phis, xis=None):
        """Xi_i and E_x,i = 1/2 Re tr M_i for every system (Alg. 2 steps 2-3)."""
        n = len(self.plans)
        if len(phis) != n:
            raise ValueError("one phi per plan")
        if xis is None:
            xis = [p.empty(p.n_occ) for p in self.plans]
        for p, phi, xi in zip(self.plans, phis, xis):
            p._vec(phi, "phi")
            p._vec(xi, "xi")
            if phi.shape[0] != p.n_occ or xi.shape[0] != p.n_occ:
                raise ValueError("phi and xi must hold n_occ vectors")
        hphi = (_vp * n)(*[t.data_ptr() for t in phis])
        hxi = (_vp * n)(*[t.data_ptr() for t in xis])
        _check(_lib.ace_build_batched(self._hp, hphi, hxi, _ptr(self.ex), n, self.chains, _ptr(self.ws),
                                      self.ws.numel() if self.ws is not None else 0, _stream()))
        return xis, self.ex


class ExchangeEnergy(torch.autograd.Function):
    """E_x[Phi] with a hand-written adjoint: backward returns grad_output * 2 dV
    W, the gradient dE/dRe(phi) + i dE/dIm(phi). When the N(N+1)/2 N_g pair
    potentials fit in the free device memory (with `store`, by default half of
    it), forward keeps them in the plan's store workspace and backward only
    accumulates; otherwise backward recomputes them through the pair kernels."""

    @staticmethod
    def forward(ctx, phi, plan: Plan, store=None):
        if store is None:
            need = plan.workspace_size(OP_ENERGY_GRAD_STORE)
            have = plan._ws.get(OP_ENERGY_GRAD_STORE)
            free = torch.cuda.mem_get_info(plan.device)[0] + (have.numel() if have is not None else 0)
            store = need <= free // 2
        ex, _ = plan.energy_grad(phi, grad=False, recompute=not store)
        plan._store_token = getattr(plan, "_store_token", 0) + 1
        ctx.plan = plan
        ctx.store = store
        ctx.token = plan._store_token
        ctx.save_for_backward(phi)
        return ex

    @staticmethod
    def backward(ctx, g_out):
        # the gradient with unit scale from the adjoint kernels, then the chain
        # rule's upstream factor applied on the device (no host synchronisation)
        (phi,) = ctx.saved_tensors
        plan = ctx.plan
        from_store = ctx.store and plan._store_token == ctx.token   # no other forward since
        _, g = plan.energy_grad(phi, grad=True, recompute=not from_store)
        g.mul_(g_out.to(g.real.dtype))
        return g, None, None


def exchange_energy(phi: torch.Tensor, plan: Plan, store=None) -> torch.Tensor:
    """E_x[phi] as a differentiable scalar; store=None picks storing the pair
    potentials when they fit, True / False forces one way."""
    return ExchangeEnergy.apply(phi, plan, store)
