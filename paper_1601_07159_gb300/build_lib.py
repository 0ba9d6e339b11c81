"""Build libace.so in-tree: one nvcc process per translation unit (the pair
kernels once per precision and plane, pencil length or cubic edge), run in
parallel, then a shared link. sm_103a only (GB300).

    python -m paper_1601_07159_gb300.build_lib [--force]
"""
from __future__ import annotations

import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libace.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
PLAIN = ["pair_dispatch.cu", "pair_point.cu", "dense.cu", "chol.cu", "tc_gemm.cu", "xi_oz.cu", "ace_api.cu",
         "apply_static.cu"]


def shape_lists():
    """The compiled edges and non-square planes per precision (and, as
    "f32_r1", the FP32 ones also compiled with the odd-radix-first order), read
    from the lists in csrc/pair_dispatch.cu (the one place they are written
    down)."""
    text = open(os.path.join(CSRC, "pair_dispatch.cu")).read()
    out = {}
    for prec in ("F32", "F64", "F32_R1"):
        edges = re.search(rf"#define ACE_EDGES_{prec}\(X\)(.*)", text).group(1)
        planes = re.search(rf"#define ACE_PLANES_{prec}\(X\)(.*)", text).group(1)
        out[prec.lower()] = (tuple(int(v) for v in re.findall(r"X\((\d+)\)", edges)),
                             tuple((int(a), int(b)) for a, b in re.findall(r"X\((\d+),\s*(\d+)\)", planes)))
    return out


def units():
    """(source, object name, extra flags) for every translation unit."""
    out = [(s, s.replace(".cu", ".o"), []) for s in PLAIN]
    lists = shape_lists()
    r1_edges, r1_planes = lists.pop("f32_r1")
    for nx, ny in [(n, n) for n in r1_edges] + list(r1_planes):   # odd-radix-first FP32 instances
        tag = f"f32_{nx}_{ny}_r1"
        out.append(("pair_plane.cu", f"pair_plane_{tag}.o",
                    ["-DACE_PLANE_R=float", f"-DACE_PX={nx}", f"-DACE_PY={ny}", f"-DACE_PLANE_TAG={tag}",
                     "-DACE_RADIX_ORDER=1"]))
    for n in r1_edges:
        tag = f"f32_{n}_r1"
        out.append(("pair_pencil.cu", f"pair_pencil_{tag}.o",
                    ["-DACE_PENCIL_R=float", f"-DACE_PZ={n}", f"-DACE_PENCIL_TAG={tag}", "-DACE_RADIX_ORDER=1"]))
    for prec, (edges, planes) in lists.items():
        typ = "float" if prec == "f32" else "double"
        for nx, ny in [(n, n) for n in edges] + list(planes):
            tag = f"{prec}_{nx}_{ny}"
            out.append(("pair_plane.cu", f"pair_plane_{tag}.o",
                        [f"-DACE_PLANE_R={typ}", f"-DACE_PX={nx}", f"-DACE_PY={ny}", f"-DACE_PLANE_TAG={tag}"]))
        for n in edges:
            tag = f"{prec}_{n}"
            out.append(("pair_pencil.cu", f"pair_pencil_{tag}.o",
                        [f"-DACE_PENCIL_R={typ}", f"-DACE_PZ={n}", f"-DACE_PENCIL_TAG={tag}"]))
            out.append(("pair_edge.cu", f"pair_edge_{tag}.o",
                        [f"-DACE_EDGE_R={typ}", f"-DACE_EDGE_N={n}", f"-DACE_EDGE_TAG={tag}"]))
    return out


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _stamp(path: str) -> float:
    return os.path.getmtime(path) if os.path.exists(path) else -1.0


def _deps_mtime() -> float:
    t = _stamp(os.path.abspath(__file__))
    for d in (CSRC, os.path.join(os.path.dirname(PKG), "include")):
        for f in os.listdir(d):
            t = max(t, os.path.getmtime(os.path.join(d, f)))
    return t


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    deps = _deps_mtime()
    if not force and _stamp(LIB) > deps:
        return LIB
    cc = nvcc()
    todo = []
    objs = []
    for src, obj, extra in units():
        path = os.path.join(BUILD, obj)
        objs.append(path)
        if force or _stamp(path) <= deps:
            todo.append([cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", path])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        return cmd, r.returncode, r.stdout.decode(errors="replace")

    workers = max(1, min(len(todo), os.cpu_count() or 1))
    failed = []
    with ThreadPoolExecutor(max_workers=workers) as ex:
        for cmd, rc, out in ex.map(run, todo):
            if rc != 0:
                failed.append((cmd[-3], out))
            elif verbose and out.strip():
                print(out)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"--- {s}\n{o}" for s, o in failed))
    tmp = LIB + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
