"""All-core float64 oracle of Algorithm 2: ctypes binding of omp_oracle.c (plain C + OpenMP).

Test infrastructure (only tests, smoke() and the benchmark's CPU legs use it).  The C code
restates oracle/spectral.py, oracle/kmeans.py and oracle/rng.py step for step with parallel loops
over rows and points; the CPU tests pin it against them on small graphs.  It is the oracle timed
on all host cores (the sequential numpy oracle is the parity reference).

build() compiles it with gcc (-O2 -fopenmp -ffp-contract=off); load() builds on first use when
the shared object is missing or older than its source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "omp_oracle.c")
LIB = os.path.join(HERE, "_omp_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", LIB, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError("building the OpenMP oracle failed:\n" + r.stdout + r.stderr)
    return LIB


def load() -> C.CDLL:
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, i64, i32, u64 = C.c_void_p, C.c_int64, C.c_int, C.c_uint64
        L.orc_threads.restype = i32
        L.orc_set_threads.argtypes = [i32]
        L.orc_set_threads.restype = None
        L.orc_gaussian_block.argtypes = [i64, i32, u64, vp]
        L.orc_kmeanspp_uniform.argtypes = [u64, i64]
        L.orc_kmeanspp_uniform.restype = C.c_double
        L.orc_degrees.argtypes = [i64, vp, vp, vp, vp, vp]
        L.orc_power_method.argtypes = [i64, vp, vp, vp, vp, vp, i32, i32, vp, vp]
        L.orc_embedding_f32.argtypes = [i64, i32, vp, vp, vp]
        L.orc_kmeanspp.argtypes = [i64, i32, vp, i32, i32, u64, vp, vp, vp]
        L.orc_lloyd.argtypes = [i64, i32, vp, i32, vp, i32, vp, vp, vp, vp, vp, vp]
        L.orc_lloyd.restype = i32
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def threads() -> int:
    return int(load().orc_threads())


def set_threads(n: int) -> None:
    """Number of OpenMP threads for the following calls."""
    load().orc_set_threads(int(n))


class Csr:
    """The graph's CSR arrays in the dtypes the C code reads (kept alive by this object)."""

    def __init__(self, g):
        self.n = int(g.n)
        self.rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(g.col, dtype=np.int32)
        self.w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.float32)


def degrees(csr: Csr):
    deg = np.empty(csr.n)
    dinv = np.empty(csr.n)
    load().orc_degrees(csr.n, _p(csr.rp), _p(csr.col), _p(csr.w), _p(deg), _p(dinv))
    return deg, dinv


def gaussian_block(n: int, l: int, seed: int) -> np.ndarray:
    out = np.empty((n, l))
    load().orc_gaussian_block(n, l, seed, _p(out))
    return out


def power_method(csr: Csr, deg, dinv, x: np.ndarray, t: int) -> np.ndarray:
    """t steps of Algorithm 1 on the block x (n x l), in place; returns x."""
    assert x.flags.c_contiguous and x.dtype == np.float64 and x.shape[1] <= 64
    tmp = np.empty_like(x)
    load().orc_power_method(csr.n, _p(csr.rp), _p(csr.col), _p(csr.w), _p(deg), _p(dinv), x.shape[1], t,
                            _p(x), _p(tmp))
    return x


def embedding_f32(dinv, y: np.ndarray) -> np.ndarray:
    out = np.empty(y.shape, dtype=np.float32)
    load().orc_embedding_f32(y.shape[0], y.shape[1], _p(dinv), _p(y), _p(out))
    return out


def embed(g, l: int, t: int, seed: int) -> np.ndarray:
    """D^-1/2 M^t X0 rounded to float32 (Algorithm 2 up to k-means)."""
    csr = Csr(g)
    deg, dinv = degrees(csr)
    x = gaussian_block(csr.n, l, seed)
    power_method(csr, deg, dinv, x, t)
    return embedding_f32(dinv, x)


def kmeanspp(X: np.ndarray, k: int, seed: int, rounds: int | None = None) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    n, l = X.shape
    seeds = np.full(k, -1, dtype=np.int64)
    D2 = np.empty(n, dtype=np.float32)
    prefix = np.empty(n)
    load().orc_kmeanspp(n, l, _p(X), k, k if rounds is None else rounds, seed, _p(seeds), _p(D2), _p(prefix))
    return seeds


def lloyd(X: np.ndarray, seeds: np.ndarray, max_iter: int = 100):
    X = np.ascontiguousarray(X, dtype=np.float32)
    n, l = X.shape
    k = len(seeds)
    seeds = np.ascontiguousarray(seeds, dtype=np.int64)
    labels = np.empty(n, dtype=np.int32)
    c64 = np.empty((k, l))
    inertia = C.c_double(0.0)
    changed = C.c_int64(0)
    best = np.empty(n, dtype=np.float32)
    second = np.empty(n, dtype=np.float32)
    it = load().orc_lloyd(n, l, _p(X), k, _p(seeds), max_iter, _p(labels), _p(c64), C.byref(inertia),
                          C.byref(changed), _p(best), _p(second))
    return {"labels": labels, "centroids": c64, "iters": int(it), "inertia": float(inertia.value),
            "changed": int(changed.value), "best": best, "second": second}


def kmeans(X: np.ndarray, k: int, seed: int, max_iter: int = 100):
    seeds = kmeanspp(X, k, seed)
    out = lloyd(X, seeds, max_iter)
    out["seeds"] = seeds
    return out


def fast_spectral_cluster(g, k: int, l: int, t: int, seed: int, max_iter: int = 100):
    """Algorithm 2 end to end on all host cores."""
    B = embed(g, l, t, seed)
    out = kmeans(B, k, seed, max_iter)
    out["embedding"] = B
    return out
