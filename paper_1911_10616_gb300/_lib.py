"""ctypes binding of libevoke (include/evoke.h).  Argument marshalling only:
every step of the orbit-counting path runs in the library's CUDA kernels.
There is no CPU fallback: if the library is not built or no GPU is present,
the calls raise."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

EVOKE_OK = 0
NORB = 73

_ERRORS = {
    1: "EVOKE_EINVAL", 2: "EVOKE_ENOTSIMPLE", 3: "EVOKE_ERANGE", 4: "EVOKE_ENOMEM",
    5: "EVOKE_ECUDA", 6: "EVOKE_ETIMEOUT", 7: "EVOKE_EOVERFLOW", 8: "EVOKE_EINCONSISTENT",
}

# exported symbols of include/evoke.h
SYMBOLS = ("evoke_count_orbits", "evoke_count_batch", "evoke_build_dag",
           "evoke_build_dag_noalloc", "evoke_edge_orbits", "evoke_edge_orbit_counts",
           "evoke_graphlet_totals",
           "evoke_orbit_matrix",
           "evoke_plan_create", "evoke_plan_create_batch", "evoke_plan_execute",
           "evoke_plan_launch_graph", "evoke_plan_execute_profiled", "evoke_plan_info", "evoke_plan_set_tuning",
           "evoke_plan_status", "evoke_plan_set_schedule",
           "evoke_plan_destroy", "evoke_plan_set_model", "evoke_plan_features",
           "evoke_plan_root_timing", "evoke_mlp_forward", "evoke_mlp_grad", "evoke_mlp_train",
           "evoke_profile_enable", "evoke_profile_read", "evoke_profile_reset",
           "evoke_launch_count", "evoke_strerror", "evoke_version")


class EvokeError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {_ERRORS.get(code, code)} ({strerror(code)})")


class PhaseTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int32),
                ("calls", ctypes.c_int32), ("ms", ctypes.c_double)]


class PlanStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("m", ctypes.c_uint64), ("triangles", ctypes.c_uint64),
                ("max_degree", ctypes.c_uint32), ("max_out_degree", ctypes.c_uint32),
                ("max_component", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64),
                ("kernels_per_execution", ctypes.c_int32), ("root_threads", ctypes.c_int32),
                ("root_ctas", ctypes.c_int32), ("root_ctas_max", ctypes.c_int32),
                ("link_warps", ctypes.c_int32), ("orbits", ctypes.c_int32)]


class EvokeOpts(ctypes.Structure):
    _fields_ = [("validate", ctypes.c_int32), ("root_ctas", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("orbits", ctypes.c_int32),
                ("noninduced", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libevoke.so (building it first if asked and needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libevoke is not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        lib.evoke_count_orbits.argtypes = [vp, vp, u32, u64, vp, ctypes.POINTER(EvokeOpts), vp]
        lib.evoke_count_orbits.restype = ctypes.c_int
        lib.evoke_build_dag.argtypes = [vp, vp, u32, u64, vp, vp, vp]
        lib.evoke_build_dag.restype = ctypes.c_int
        lib.evoke_build_dag_noalloc.argtypes = [vp, vp, u32, u64, vp, vp, vp]
        lib.evoke_build_dag_noalloc.restype = ctypes.c_int
        lib.evoke_edge_orbits.argtypes = [vp, vp, u32, u64, vp, vp, vp, vp, vp, vp]
        lib.evoke_edge_orbits.restype = ctypes.c_int
        lib.evoke_edge_orbit_counts.argtypes = [vp, vp, u32, u64, vp, vp]
        lib.evoke_edge_orbit_counts.restype = ctypes.c_int
        lib.evoke_graphlet_totals.argtypes = [vp, u32, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int64), vp]
        lib.evoke_graphlet_totals.restype = ctypes.c_int
        lib.evoke_orbit_matrix.argtypes = [ctypes.POINTER(ctypes.c_int64)]
        lib.evoke_orbit_matrix.restype = ctypes.c_int
        lib.evoke_strerror.argtypes = [ctypes.c_int]
        lib.evoke_strerror.restype = ctypes.c_char_p
        lib.evoke_version.restype = ctypes.c_int
        pp = ctypes.POINTER(ctypes.c_void_p)
        lib.evoke_count_batch.argtypes = [vp, vp, vp, vp, u32, vp, ctypes.POINTER(EvokeOpts), vp]
        lib.evoke_count_batch.restype = ctypes.c_int
        lib.evoke_plan_create.argtypes = [vp, vp, u32, u64, ctypes.POINTER(EvokeOpts), vp, pp]
        lib.evoke_plan_create.restype = ctypes.c_int
        lib.evoke_plan_create_batch.argtypes = [vp, vp, vp, vp, u32, ctypes.POINTER(EvokeOpts),
                                                vp, pp]
        lib.evoke_plan_create_batch.restype = ctypes.c_int
        lib.evoke_plan_execute.argtypes = [vp, vp, vp]
        lib.evoke_plan_launch_graph.argtypes = [vp, vp, vp]
        lib.evoke_plan_execute_profiled.argtypes = [vp, vp, vp]
        lib.evoke_plan_info.argtypes = [vp, ctypes.POINTER(PlanStats)]
        lib.evoke_plan_status.argtypes = [vp, vp]
        lib.evoke_plan_set_schedule.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
        lib.evoke_plan_set_schedule.restype = ctypes.c_int
        lib.evoke_plan_status.restype = ctypes.c_int
        lib.evoke_plan_set_tuning.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
        lib.evoke_plan_destroy.argtypes = [vp]
        lib.evoke_plan_set_model.argtypes = [vp, vp]
        lib.evoke_plan_features.argtypes = [vp, vp, vp]
        lib.evoke_plan_root_timing.argtypes = [vp, vp, vp, vp, vp]
        lib.evoke_mlp_forward.argtypes = [vp, u32, vp, vp, vp]
        lib.evoke_mlp_grad.argtypes = [vp, vp, u32, vp, vp, vp, vp]
        lib.evoke_mlp_train.argtypes = [vp, vp, u32, vp, vp, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_float, ctypes.POINTER(ctypes.c_float), vp, vp]
        lib.evoke_profile_enable.argtypes = [ctypes.c_int]
        lib.evoke_profile_read.argtypes = [ctypes.POINTER(PhaseTime), ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int)]
        lib.evoke_launch_count.restype = ctypes.c_uint64
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load(False).evoke_strerror(code).decode()
    except Exception:
        return "?"


def _check(rc: int, what: str):
    if rc != EVOKE_OK:
        raise EvokeError(rc, what)


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def to_device(graph, device="cuda"):
    """Upload a graphgen.Graph as (rowptr, colidx) uint32 bit patterns held in
    int32 tensors on `device`."""
    import torch
    rp = np.ascontiguousarray(graph.rowptr.astype(np.uint32)).view(np.int32)
    col = np.ascontiguousarray(graph.col.astype(np.uint32)).view(np.int32)
    return (torch.from_numpy(rp).to(device, non_blocking=False),
            torch.from_numpy(col).to(device, non_blocking=False))


def _check_graph(rowptr, colidx, n):
    import torch
    if not (rowptr.is_cuda and colidx.is_cuda):
        raise ValueError("rowptr / colidx must be CUDA tensors")
    if rowptr.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)) or \
            colidx.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
        raise ValueError("rowptr / colidx must hold 32-bit ids")
    if rowptr.numel() != n + 1 or not rowptr.is_contiguous() or not colidx.is_contiguous():
        raise ValueError("rowptr must be contiguous with n+1 entries")


def _orbits(orbits: int) -> int:
    if orbits not in (15, 73):
        raise ValueError("orbits must be 73 (all) or 15 (the 4-vertex orbits 0..14)")
    return orbits


def count_orbits(rowptr, colidx, n: int, m: int, out=None, validate: bool = False,
                 root_ctas: int = 0, stream=None, orbits: int = 73, induced: bool = True,
                 schedule: int = 0):
    """Orbit counts, int64 tensor [n, orbits] on the graph's device (orbits =
    73: all; 15: the 4-vertex orbits 0..14 only); induced=False gives the
    non-induced counts DM."""
    import torch
    _check_graph(rowptr, colidx, n)
    k = _orbits(orbits)
    if out is None:
        out = torch.empty((n, k), dtype=torch.int64, device=rowptr.device)
    elif out.dtype != torch.int64 or out.numel() != n * k or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous int64 tensor with n*{k} entries")
    opts = EvokeOpts(1 if validate else 0, int(root_ctas), int(schedule), k, 0 if induced else 1)
    rc = load().evoke_count_orbits(_ptr(rowptr), _ptr(colidx), n, m, _ptr(out),
                                   ctypes.byref(opts), _stream_handle(stream))
    _check(rc, "evoke_count_orbits")
    return out


def batch_to_device(graphs, device="cuda"):
    """Concatenate graphgen.Graph objects for evoke_count_batch: returns
    (rowptr_cat, colidx_cat, vtx_off, edge_off) CUDA tensors."""
    import torch
    from . import graphgen
    rp, col, vo, eo = graphgen.concat_batch(graphs)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    return (t(rp.astype(np.uint32).view(np.int32)), t(col.astype(np.uint32).view(np.int32)),
            t(vo.astype(np.int64)), t(eo.astype(np.int64)))


def count_batch(rowptr_cat, colidx_cat, vtx_off, edge_off, out=None, validate: bool = False,
                stream=None, orbits: int = 73, induced: bool = True):
    """Induced orbit counts of a batch of graphs, int64 [sum n_g, orbits]."""
    import torch
    G = vtx_off.numel() - 1
    N = int(vtx_off[-1].item())
    k = _orbits(orbits)
    if out is None:
        out = torch.empty((N, k), dtype=torch.int64, device=vtx_off.device)
    opts = EvokeOpts(1 if validate else 0, 0, 0, k, 0 if induced else 1)
    rc = load().evoke_count_batch(_ptr(rowptr_cat), _ptr(colidx_cat), _ptr(vtx_off),
                                  _ptr(edge_off), G, _ptr(out), ctypes.byref(opts),
                                  _stream_handle(stream))
    _check(rc, "evoke_count_batch")
    return out


class Plan:
    """A sized, allocated execution plan (evoke_plan_*).  Keep the input
    tensors alive and unchanged while the plan exists."""

    def __init__(self, handle, inputs, n, orbits=73):
        self._h = handle
        self._inputs = inputs
        self.n = n
        self.orbits = orbits

    @classmethod
    def single(cls, rowptr, colidx, n: int, m: int, validate: bool = False, stream=None,
               orbits: int = 73, induced: bool = True):
        _check_graph(rowptr, colidx, n)
        h = ctypes.c_void_p()
        opts = EvokeOpts(1 if validate else 0, 0, 0, _orbits(orbits), 0 if induced else 1)
        _check(load().evoke_plan_create(_ptr(rowptr), _ptr(colidx), n, m, ctypes.byref(opts),
                                        _stream_handle(stream), ctypes.byref(h)),
               "evoke_plan_create")
        return cls(h, (rowptr, colidx), n, orbits)

    @classmethod
    def batch(cls, rowptr_cat, colidx_cat, vtx_off, edge_off, validate: bool = False,
              stream=None, orbits: int = 73, induced: bool = True):
        h = ctypes.c_void_p()
        opts = EvokeOpts(1 if validate else 0, 0, 0, _orbits(orbits), 0 if induced else 1)
        G = vtx_off.numel() - 1
        _check(load().evoke_plan_create_batch(_ptr(rowptr_cat), _ptr(colidx_cat), _ptr(vtx_off),
                                              _ptr(edge_off), G, ctypes.byref(opts),
                                              _stream_handle(stream), ctypes.byref(h)),
               "evoke_plan_create_batch")
        return cls(h, (rowptr_cat, colidx_cat, vtx_off, edge_off), int(vtx_off[-1].item()),
                   orbits)

    def new_output(self):
        import torch
        dev = self._inputs[0].device
        return torch.empty((self.n, self.orbits), dtype=torch.int64, device=dev)

    def execute(self, out, stream=None):
        _check(load().evoke_plan_execute(self._h, _ptr(out), _stream_handle(stream)),
               "evoke_plan_execute")
        return out

    def execute_profiled(self, out, stream=None):
        """execute() with the library's per-phase CUDA events (see
        profile_enable); the same kernels."""
        _check(load().evoke_plan_execute_profiled(self._h, _ptr(out), _stream_handle(stream)),
               "evoke_plan_execute_profiled")
        return out

    def launch_graph(self, out, stream=None):
        _check(load().evoke_plan_launch_graph(self._h, _ptr(out), _stream_handle(stream)),
               "evoke_plan_launch_graph")
        return out

    def status(self, stream=None):
        """Raise EvokeError if the latest execution's device checks failed
        (a wrapped 32-bit 3-path count: EVOKE_EOVERFLOW); synchronises."""
        _check(load().evoke_plan_status(self._h, _stream_handle(stream)), "evoke_plan_status")

    def info(self) -> dict:
        st = PlanStats()
        _check(load().evoke_plan_info(self._h, ctypes.byref(st)), "evoke_plan_info")
        return {f: getattr(st, f) for f, _ in PlanStats._fields_}

    def set_tuning(self, root_threads: int, root_ctas: int):
        _check(load().evoke_plan_set_tuning(self._h, int(root_threads), int(root_ctas)),
               "evoke_plan_set_tuning")

    def set_schedule(self, schedule: int, chunk: int = 8):
        """Root order: 0 degree-bucket, 1 grouped by highest-degree neighbour
        with `chunk` roots per queue grab."""
        _check(load().evoke_plan_set_schedule(self._h, int(schedule), int(chunk)),
               "evoke_plan_set_schedule")

    def set_model(self, params):
        """Attach MLP parameters (float32 CUDA tensor of 1249) or None."""
        self._model = params
        _check(load().evoke_plan_set_model(self._h, _ptr(params) if params is not None else None),
               "evoke_plan_set_model")

    def features(self, stream=None):
        import torch
        X = torch.empty((self.n, 4), dtype=torch.float32, device=self._inputs[0].device)
        _check(load().evoke_plan_features(self._h, _ptr(X), _stream_handle(stream)),
               "evoke_plan_features")
        return X

    def root_timing(self, out=None, stream=None):
        """One execution recording per-vertex root-pass cycles and per-CTA end
        times; returns (cycles int64 [n], cta_end_ns int64 [ctas])."""
        import torch
        dev = self._inputs[0].device
        cyc = torch.zeros(self.n, dtype=torch.int64, device=dev)
        ends = torch.zeros(max(self.info()["root_ctas_max"], 1), dtype=torch.int64, device=dev)
        _check(load().evoke_plan_root_timing(self._h, _ptr(cyc), _ptr(ends), _ptr(out),
                                             _stream_handle(stream)), "evoke_plan_root_timing")
        return cyc, ends[: self.info()["root_ctas"]]

    def destroy(self):
        if self._h:
            load().evoke_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def edge_orbits(rowptr, colidx, n: int, m: int, stream=None):
    """Per-slot T, C4, K4, E7, E9<u,v> as int64 tensors of 2m entries."""
    import torch
    _check_graph(rowptr, colidx, n)
    outs = [torch.empty(2 * m, dtype=torch.int64, device=rowptr.device) for _ in range(5)]
    if m == 0:
        return dict(zip(["T", "C4", "K4", "E7", "E9"], outs))
    rc = load().evoke_edge_orbits(_ptr(rowptr), _ptr(colidx), n, m, *[_ptr(o) for o in outs],
                                  _stream_handle(stream))
    _check(rc, "evoke_edge_orbits")
    return dict(zip(["T", "C4", "K4", "E7", "E9"], outs))


def edge_orbit_counts(rowptr, colidx, n: int, m: int, stream=None):
    """E0..E11<u,v> of Lem. 4edgeorbit: int64 tensor [2m, 12], row = CSR slot."""
    import torch
    _check_graph(rowptr, colidx, n)
    out = torch.empty((2 * m, 12), dtype=torch.int64, device=rowptr.device)
    if m == 0:
        return out
    rc = load().evoke_edge_orbit_counts(_ptr(rowptr), _ptr(colidx), n, m, _ptr(out),
                                        _stream_handle(stream))
    _check(rc, "evoke_edge_orbit_counts")
    return out


def graphlet_totals(counts, stream=None) -> np.ndarray:
    """Global pattern counts from per-vertex orbit counts (int64 CUDA tensor
    [n, 73] or [n, 15]): int64 array of 30 (H0..H29) or 9 (H0..H8) totals."""
    k = _orbits(int(counts.shape[1]) if counts.dim() == 2 else 0)
    if not counts.is_contiguous():
        raise ValueError("counts must be contiguous")
    n = int(counts.shape[0])
    out = (ctypes.c_int64 * (30 if k == 73 else 9))()
    rc = load().evoke_graphlet_totals(_ptr(counts) if n else None, n, k, out,
                                      _stream_handle(stream))
    _check(rc, "evoke_graphlet_totals")
    return np.array(out[:], dtype=np.int64)


def build_dag(rowptr, colidx, n: int, m: int, stream=None):
    import torch
    _check_graph(rowptr, colidx, n)
    dp = torch.empty(n + 1, dtype=torch.int32, device=rowptr.device)
    dc = torch.empty(max(m, 1), dtype=torch.int32, device=rowptr.device)
    rc = load().evoke_build_dag(_ptr(rowptr), _ptr(colidx), n, m, _ptr(dp), _ptr(dc),
                                _stream_handle(stream))
    _check(rc, "evoke_build_dag")
    return dp, dc[:m]


def build_dag_noalloc(rowptr, colidx, n: int, m: int, dag_rowptr, dag_colidx, stream=None):
    """evoke_build_dag_noalloc: fills the caller's dag_rowptr (n+1) and
    dag_colidx (m) int32 CUDA tensors; the library allocates nothing."""
    _check_graph(rowptr, colidx, n)
    rc = load().evoke_build_dag_noalloc(_ptr(rowptr), _ptr(colidx), n, m, _ptr(dag_rowptr),
                                        _ptr(dag_colidx), _stream_handle(stream))
    _check(rc, "evoke_build_dag_noalloc")
    return dag_rowptr, dag_colidx


def orbit_matrix() -> np.ndarray:
    A = np.zeros(73 * 73, dtype=np.int64)
    _check(load().evoke_orbit_matrix(A.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
           "evoke_orbit_matrix")
    return A.reshape(73, 73)


def version() -> int:
    return int(load().evoke_version())


def profile_enable(on: bool = True):
    load().evoke_profile_enable(1 if on else 0)


def profile_reset():
    load().evoke_profile_reset()


def profile_read():
    """{phase: (launches, calls, total_ms)} of the phases run while enabled."""
    lib = load()
    cap = 64
    arr = (PhaseTime * cap)()
    cnt = ctypes.c_int(0)
    _check(lib.evoke_profile_read(arr, cap, ctypes.byref(cnt)), "evoke_profile_read")
    return {arr[i].name.decode(): (arr[i].launches, arr[i].calls, arr[i].ms)
            for i in range(min(cnt.value, cap))}


def launch_count() -> int:
    return int(load().evoke_launch_count())


MLP_PARAMS = 1249


def mlp_forward(X, params, stream=None):
    import torch
    y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    _check(load().evoke_mlp_forward(_ptr(X), X.shape[0], _ptr(params), _ptr(y),
                                    _stream_handle(stream)), "evoke_mlp_forward")
    return y


def mlp_grad(X, T, params, stream=None):
    import torch
    g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=X.device)
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    _check(load().evoke_mlp_grad(_ptr(X), _ptr(T), X.shape[0], _ptr(params), _ptr(g), _ptr(loss),
                                 _stream_handle(stream)), "evoke_mlp_grad")
    return g, loss


def mlp_train(X, T, params, epochs: int, batch: int, lr: float, state=None, stream=None):
    """Adam training on device, params updated in place; returns per-epoch losses."""
    import torch
    if state is None:
        state = torch.zeros(2 * MLP_PARAMS, dtype=torch.float32, device=X.device)
    scratch = torch.zeros(1280 + epochs, dtype=torch.float32, device=X.device)
    losses = (ctypes.c_float * epochs)()
    _check(load().evoke_mlp_train(_ptr(X), _ptr(T), X.shape[0], _ptr(params), _ptr(state),
                                  epochs, batch, float(lr), losses, _ptr(scratch),
                                  _stream_handle(stream)), "evoke_mlp_train")
    return [float(v) for v in losses], state
