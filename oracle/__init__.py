"""ORACLE -- test infrastructure only.

A plain CPU implementation of EVOKE's per-vertex orbit counts (brute force by
ESU enumeration, and the paper's equations), written from the paper and
sharing nothing with the CUDA path.  Only ``tests/``, ``__graft_entry__.smoke``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  ``build()`` compiles ``evoke_oracle.cpp`` with g++ (OpenMP).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "evoke_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libevoke_oracle.so")
_lock = threading.Lock()
_lib = None

NORB = 73


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++ -O2 -fopenmp)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.oracle_tables_ok.restype = ctypes.c_int
            lib.oracle_pattern_orbits.argtypes = [ip, ip, ip]
            lib.oracle_pattern_adj.argtypes = [ip]
            lib.oracle_A_matrix.argtypes = [i64p]
            lib.oracle_brute_force.argtypes = [i64p, u32p, ctypes.c_uint32, i64p, i64p, ctypes.c_int]
            lib.oracle_formulas.argtypes = [i64p, u32p, ctypes.c_uint32, i64p, i64p, ctypes.c_int]
            lib.oracle_edge_counts.argtypes = [i64p, u32p, ctypes.c_uint32] + [i64p] * 5 + [ctypes.c_int]
            lib.oracle_edge_orbits_brute.argtypes = [i64p, u32p, ctypes.c_uint32, i64p, ctypes.c_int]
            lib.oracle_edge_orbits_formula.argtypes = [i64p, u32p, ctypes.c_uint32, i64p, ctypes.c_int]
            lib.oracle_formulas4.argtypes = [i64p, u32p, ctypes.c_uint32, i64p, ctypes.c_int]
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _csr(g):
    rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.uint32)
    return rp, col


def tables_ok() -> bool:
    return _load().oracle_tables_ok() == 0


def pattern_orbits():
    """(k[30], orbit_of[30,5], orbit_size[73]) from the automorphism computation."""
    k = np.zeros(30, np.int32)
    orb = np.zeros(150, np.int32)
    sz = np.zeros(73, np.int32)
    rc = _load().oracle_pattern_orbits(_p(k, ctypes.c_int), _p(orb, ctypes.c_int), _p(sz, ctypes.c_int))
    if rc:
        raise RuntimeError("oracle pattern tables inconsistent")
    return k, orb.reshape(30, 5), sz


def pattern_adjacency():
    adj = np.zeros(30 * 25, np.int32)
    if _load().oracle_pattern_adj(_p(adj, ctypes.c_int)):
        raise RuntimeError("oracle pattern tables inconsistent")
    return adj.reshape(30, 5, 5)


def A_matrix() -> np.ndarray:
    A = np.zeros(73 * 73, np.int64)
    if _load().oracle_A_matrix(_p(A, ctypes.c_int64)):
        raise RuntimeError("oracle pattern tables inconsistent")
    return A.reshape(73, 73)


def brute_force(g, noninduced: bool = False, threads: int = 0):
    """Induced counts int64[n,73] by ESU; with ``noninduced`` also the
    non-induced counts by spanning-subgraph enumeration (tiny graphs only)."""
    rp, col = _csr(g)
    dim = np.zeros(g.n * NORB, np.int64)
    dm = np.zeros(g.n * NORB, np.int64) if noninduced else None
    rc = _load().oracle_brute_force(_p(rp, ctypes.c_int64), _p(col, ctypes.c_uint32), g.n,
                                    _p(dim, ctypes.c_int64),
                                    _p(dm, ctypes.c_int64) if dm is not None else None, threads)
    if rc:
        raise RuntimeError(f"oracle brute force failed ({rc})")
    dim = dim.reshape(g.n, NORB)
    return (dim, dm.reshape(g.n, NORB)) if noninduced else dim


def formulas(g, threads: int = 0):
    """(non-induced DM, induced DIM), both int64[n,73], by the paper's method."""
    rp, col = _csr(g)
    dm = np.zeros(g.n * NORB, np.int64)
    dim = np.zeros(g.n * NORB, np.int64)
    rc = _load().oracle_formulas(_p(rp, ctypes.c_int64), _p(col, ctypes.c_uint32), g.n,
                                 _p(dm, ctypes.c_int64), _p(dim, ctypes.c_int64), threads)
    if rc == 7:
        raise OverflowError("an orbit count leaves int64")
    if rc:
        raise RuntimeError(f"oracle formulas failed ({rc})")
    return dm.reshape(g.n, NORB), dim.reshape(g.n, NORB)


def induced(g, threads: int = 0) -> np.ndarray:
    return formulas(g, threads)[1]


def formulas4(g, threads: int = 0):
    """Induced counts of the 4-vertex orbits 0..14 only (Thm. 4orbit), int64[n,15]."""
    rp, col = _csr(g)
    dim = np.zeros(g.n * 15, np.int64)
    rc = _load().oracle_formulas4(_p(rp, ctypes.c_int64), _p(col, ctypes.c_uint32), g.n,
                                  _p(dim, ctypes.c_int64), threads)
    if rc:
        raise RuntimeError(f"oracle 4-vertex formulas failed ({rc})")
    return dim.reshape(g.n, 15)


def edge_counts(g, threads: int = 0):
    """Per-slot T, C4, K4, E7, E9<u,v> (slot = position of v in row u)."""
    rp, col = _csr(g)
    S = int(rp[-1])
    outs = [np.zeros(S, np.int64) for _ in range(5)]
    rc = _load().oracle_edge_counts(_p(rp, ctypes.c_int64), _p(col, ctypes.c_uint32), g.n,
                                    *[_p(o, ctypes.c_int64) for o in outs], threads)
    if rc:
        raise RuntimeError(f"oracle edge counts failed ({rc})")
    return dict(zip(["T", "C4", "K4", "E7", "E9"], outs))


def _edge_orbits(fn, what, g, threads):
    rp, col = _csr(g)
    S = int(rp[-1])
    out = np.zeros((S, 12), np.int64)
    rc = fn(_p(rp, ctypes.c_int64), _p(col, ctypes.c_uint32), g.n, _p(out, ctypes.c_int64), threads)
    if rc:
        raise RuntimeError(f"oracle {what} failed ({rc})")
    return out


def edge_orbits_brute(g, threads: int = 0):
    """E0..E11<u,v> per slot by the definition (tiny graphs): int64 [2m, 12]."""
    return _edge_orbits(_load().oracle_edge_orbits_brute, "edge-orbit brute force", g, threads)


def edge_orbits_formula(g, threads: int = 0):
    """E0..E11<u,v> per slot by Lem. 4edgeorbit: int64 [2m, 12]."""
    return _edge_orbits(_load().oracle_edge_orbits_formula, "edge-orbit formulas", g, threads)


def max_threads() -> int:
    return int(_load().oracle_max_threads())
