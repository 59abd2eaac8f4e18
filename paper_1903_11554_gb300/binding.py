"""Thin Python binding of libttq.so (include/ttq.h): argument marshalling only.

Every step of the quadrature runs in the library's CUDA kernels.  PyTorch is
used for device memory (the plan's workspace) and the current CUDA stream.
There is no CPU fallback: if the library or a GPU is missing, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional

import numpy as np

from . import inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libttq.so")

STATUS_NAMES = {0: "converged", 1: "no_pivot", 2: "rank_cap", 3: "max_sweeps", 4: "pending",
                -1: "invalid_arg", -2: "nonfinite", -3: "singular", -4: "workspace", -5: "cuda",
                -6: "admission", -7: "not_found", -8: "timeout"}

# function name -> (restype, argtypes); the exported surface of include/ttq.h
_c = ctypes
_vp = _c.c_void_p


class TTQProblem(_c.Structure):
    _fields_ = [("family", _c.c_int32), ("form", _c.c_int32), ("n", _c.c_int32), ("d", _c.c_int32),
                ("nodes_per_mode", _c.POINTER(_c.c_int32)), ("nodes", _c.c_void_p), ("weights", _c.c_void_p),
                ("inputs_on_device", _c.c_int32), ("rank_cap", _c.c_int32), ("tol", _c.c_double),
                ("pivot_tol", _c.c_double), ("conv_window", _c.c_int32), ("max_sweeps", _c.c_int32),
                ("seed", _c.c_uint64), ("n_samples", _c.c_int32), ("rook_max", _c.c_int32),
                ("init_samples", _c.c_int32), ("precision", _c.c_int32), ("r0", _c.c_int32),
                ("npiv", _c.c_int32)]


class TTQResult(_c.Structure):
    _fields_ = [("value", _c.c_double), ("value_lo", _c.c_double), ("internal_conv", _c.c_double),
                ("n_eval", _c.c_int64), ("sweeps", _c.c_int32), ("max_rank", _c.c_int32),
                ("status", _c.c_int32), ("d", _c.c_int32), ("ranks", _c.c_int32 * 33)]


class TTQPivot(_c.Structure):
    _fields_ = [("k", _c.c_int32), ("searched", _c.c_int32), ("row", _c.c_int32), ("col", _c.c_int32),
                ("err", _c.c_double), ("accepted", _c.c_int32), ("rounds", _c.c_int32),
                ("evals", _c.c_int64)]


_i32p = _c.POINTER(_c.c_int32)
_dp = _c.POINTER(_c.c_double)
SIGNATURES = {
    "ttq_workspace_bytes": (_c.c_int, [_c.POINTER(TTQProblem), _c.POINTER(_c.c_size_t)]),
    "ttq_plan_create": (_c.c_int, [_c.POINTER(TTQProblem), _vp, _c.c_size_t, _vp, _c.POINTER(_vp)]),
    "ttq_plan_destroy": (_c.c_int, [_vp]),
    "ttq_plan_run": (_c.c_int, [_vp, _c.POINTER(TTQResult)]),
    "ttq_plan_init": (_c.c_int, [_vp]),
    "ttq_plan_launch": (_c.c_int, [_vp, _c.c_int]),
    "ttq_plan_result": (_c.c_int, [_vp, _c.c_int, _c.POINTER(TTQResult)]),
    "ttq_plan_set_state": (_c.c_int, [_vp, _i32p, _i32p, _i32p, _i32p, _i32p]),
    "ttq_plan_get_state": (_c.c_int, [_vp, _i32p, _i32p, _i32p, _i32p, _i32p]),
    "ttq_plan_sweep": (_c.c_int, [_vp, _c.c_int, _c.c_int, _dp, _dp, _c.POINTER(TTQPivot)]),
    "ttq_plan_get_core": (_c.c_int, [_vp, _c.c_int, _dp]),
    "ttq_plan_eval_points": (_c.c_int, [_vp, _vp, _c.c_int64, _vp]),
    "ttq_plan_launches": (_c.c_int64, [_vp]),
    "ttq_plan_transfer_bytes": (_c.c_int, [_vp, _c.POINTER(_c.c_int64), _c.POINTER(_c.c_int64)]),
    "ttq_plan_set_graphs": (_c.c_int, [_vp, _c.c_int]),
    "ttq_plan_set_timing": (_c.c_int, [_vp, _c.c_int]),
    "ttq_plan_set_search": (_c.c_int, [_vp, _c.c_int]),
    "ttq_plan_set_sequential": (_c.c_int, [_vp, _c.c_int]),
    "ttq_plan_set_wait_limit": (_c.c_int, [_vp, _c.c_uint64]),
    "ttq_plan_kernel_times": (_c.c_int, [_vp, _dp, _c.POINTER(_c.c_int64), _dp, _c.c_int]),
    "ttq_integrate_noalloc": (_c.c_int, [_c.POINTER(TTQProblem), _vp, _c.POINTER(TTQResult)]),
    "ttq_batch_workspace_bytes": (_c.c_int, [_c.POINTER(TTQProblem), _c.c_int, _c.POINTER(_c.c_size_t)]),
    "ttq_batch_create": (_c.c_int, [_c.POINTER(TTQProblem), _c.c_int, _vp, _c.c_size_t, _vp, _c.POINTER(_vp)]),
    "ttq_batch_run": (_c.c_int, [_vp, _c.POINTER(TTQResult)]),
    "ttq_batch_autotune": (_c.c_int, [_vp, _c.c_int, _i32p]),
    "ttq_plan_set_config": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int]),
    "ttq_plan_set_rook_rows": (_c.c_int, [_vp, _c.c_int]),
    "ttq_batch_set_groups": (_c.c_int, [_vp, _c.c_int]),
    "ttq_server_create": (_c.c_int, [_vp, _c.c_size_t, _c.c_int, _vp, _c.POINTER(_vp)]),
    "ttq_server_destroy": (_c.c_int, [_vp]),
    "ttq_server_submit": (_c.c_int, [_vp, _c.POINTER(TTQProblem), _c.POINTER(_c.c_uint64)]),
    "ttq_server_step": (_c.c_int, [_vp, _c.c_int, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int),
                                   _c.POINTER(_c.c_int64)]),
    "ttq_server_poll": (_c.c_int, [_vp, _c.c_uint64, _c.POINTER(TTQResult)]),
    "ttq_server_drain": (_c.c_int, [_vp, _c.POINTER(_c.c_uint64), _c.POINTER(TTQResult), _c.c_int,
                                    _c.POINTER(_c.c_int)]),
    "ttq_server_stats": (_c.c_int, [_vp, _c.POINTER(_c.c_int64)]),
    "ttq_server_set_mode": (_c.c_int, [_vp, _c.c_int]),
    "ttq_tt_bytes": (_c.c_int, [_vp, _c.c_int, _c.POINTER(_c.c_size_t)]),
    "ttq_tt_export": (_c.c_int, [_vp, _c.c_int, _vp, _c.c_size_t, _c.POINTER(_vp)]),
    "ttq_tt_get": (_c.c_int, [_vp, _c.c_int, _i32p, _i32p, _i32p, _c.POINTER(_vp), _c.POINTER(_vp),
                              _c.POINTER(_vp)]),
    "ttq_tt_ranks": (_c.c_int, [_vp, _i32p, _i32p]),
    "ttq_tt_free": (_c.c_int, [_vp]),
    "ttq_status_string": (_c.c_char_p, [_c.c_int]),
    "ttq_last_error": (_c.c_char_p, []),
}

KERNELS = ("eval_slabs", "qr", "contract", "samples", "rook_col", "rook_row", "update", "init", "setup",
           "solve", "search")

_lib = None


def load(path: str = LIB_PATH):
    """Load libttq.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libttq.so not built: run __graft_entry__.build() (or python -m "
                               "paper_1903_11554_gb300.build)")
        lib = _c.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class TTQError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc < 0:
        lib = load()
        raise TTQError("%s failed: %s (%s)" % (what, STATUS_NAMES.get(rc, rc),
                                               lib.ttq_last_error().decode(errors="replace")))
    return rc


class _Arrays:
    """Keeps the host arrays a ttq_problem points to alive."""

    def __init__(self, p: inputs.Problem, nodes=None, weights=None):
        self.N = np.ascontiguousarray(p.N, dtype=np.int32)
        if nodes is None:
            self.nodes = np.ascontiguousarray(np.concatenate(p.nodes), dtype=np.float64)
            self.weights = np.ascontiguousarray(np.concatenate(p.weights), dtype=np.float64)
            self.on_device = 0
            self.nptr = self.nodes.ctypes.data
            self.wptr = self.weights.ctypes.data
        else:
            self.nodes, self.weights = nodes, weights
            self.on_device = 1
            self.nptr = nodes.data_ptr()
            self.wptr = weights.data_ptr()


def make_struct(p: inputs.Problem, arrays: _Arrays) -> TTQProblem:
    s = TTQProblem()
    s.family = inputs.FAMILY_CODE[p.family]
    s.form = inputs.FORM_CODE[p.form]
    s.n = p.n
    s.d = p.d
    s.nodes_per_mode = arrays.N.ctypes.data_as(_i32p)
    s.nodes = arrays.nptr
    s.weights = arrays.wptr
    s.inputs_on_device = arrays.on_device
    s.rank_cap = p.rank_cap
    s.tol = p.tol
    s.pivot_tol = p.pivot_tol
    s.conv_window = p.conv_window
    s.max_sweeps = p.sweeps_limit()
    s.seed = p.seed & ((1 << 64) - 1)
    s.n_samples = p.n_samples
    s.rook_max = p.rook_max
    s.init_samples = p.init_samples
    s.r0 = p.r0
    s.npiv = getattr(p, "npiv", 1)
    s.precision = inputs.PREC_CODE[p.precision]
    return s


def workspace_bytes(p: inputs.Problem) -> int:
    lib = load()
    arrays = _Arrays(p)
    st = make_struct(p, arrays)
    out = _c.c_size_t(0)
    _check(lib.ttq_workspace_bytes(_c.byref(st), _c.byref(out)), "ttq_workspace_bytes")
    return int(out.value)


class Plan:
    """One integral on the GPU: workspace (torch) + plan handle (library)."""

    def __init__(self, p: inputs.Problem, workspace=None, stream=None, device_inputs=None):
        import torch
        if not torch.cuda.is_available():
            raise TTQError("no CUDA device: the TT-cross quadrature runs only on the GPU")
        self.lib = load()
        self.problem = p
        self.arrays = _Arrays(p, *(device_inputs or (None, None)))
        self.struct = make_struct(p, self.arrays)
        nbytes = _c.c_size_t(0)
        _check(self.lib.ttq_workspace_bytes(_c.byref(self.struct), _c.byref(nbytes)), "ttq_workspace_bytes")
        self.nbytes = int(nbytes.value)
        if workspace is None:
            workspace = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        if stream is None:
            stream = torch.cuda.Stream()
            stream.wait_stream(torch.cuda.current_stream())     # the workspace allocation is ordered before use
        self.stream = stream
        h = _vp()
        _check(self.lib.ttq_plan_create(_c.byref(self.struct), _vp(workspace.data_ptr()), self.nbytes,
                                        _vp(self.stream.cuda_stream), _c.byref(h)), "ttq_plan_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.ttq_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- full run ---------------------------------------------------------
    def run(self) -> Dict:
        res = TTQResult()
        _check(self.lib.ttq_plan_run(self.h, _c.byref(res)), "ttq_plan_run")
        return _result_dict(res)

    def launch(self, slot: int = 0):
        """Enqueue a whole run; its result lands in `slot` (read with result())."""
        _check(self.lib.ttq_plan_launch(self.h, slot), "ttq_plan_launch")

    def result(self, slot: int = 0) -> Dict:
        res = TTQResult()
        _check(self.lib.ttq_plan_result(self.h, slot, _c.byref(res)), "ttq_plan_result")
        return _result_dict(res)

    # -- stages -----------------------------------------------------------
    def init(self):
        _check(self.lib.ttq_plan_init(self.h), "ttq_plan_init")

    def sweep(self, s: int, search: bool = True):
        v, vlo = _c.c_double(0), _c.c_double(0)
        piv = (TTQPivot * max(1, self.problem.d - 1))()
        _check(self.lib.ttq_plan_sweep(self.h, s, 1 if search else 0, _c.byref(v), _c.byref(vlo), piv),
               "ttq_plan_sweep")
        pivots = [{"k": q.k, "searched": q.searched, "row": q.row, "col": q.col, "err": q.err,
                   "accepted": q.accepted, "rounds": q.rounds, "evals": int(q.evals)}
                  for q in piv[:self.problem.d - 1]]
        return v.value, vlo.value, pivots

    def set_state(self, ranks, lpar, lnode, rpar, rnode):
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.int32)) for a in
                (ranks, np.concatenate([np.asarray(x) for x in lpar]), np.concatenate([np.asarray(x) for x in lnode]),
                 np.concatenate([np.asarray(x) for x in rpar]), np.concatenate([np.asarray(x) for x in rnode]))]
        _check(self.lib.ttq_plan_set_state(self.h, *[a.ctypes.data_as(_i32p) for a in arrs]), "ttq_plan_set_state")

    def get_state(self):
        d = self.problem.d
        cap = self.problem.rank_cap
        ranks = np.zeros(d + 1, dtype=np.int32)
        bufs = [np.zeros(cap * (d - 1), dtype=np.int32) for _ in range(4)]
        _check(self.lib.ttq_plan_get_state(self.h, ranks.ctypes.data_as(_i32p),
                                           *[b.ctypes.data_as(_i32p) for b in bufs]), "ttq_plan_get_state")
        out = {"ranks": ranks.tolist(), "lpar": [], "lnode": [], "rpar": [], "rnode": []}
        o = 0
        for k in range(1, d):
            r = int(ranks[k])
            for name, b in zip(("lpar", "lnode", "rpar", "rnode"), bufs):
                out[name].append(b[o:o + r].copy())
            o += r
        return out

    def get_core(self, k: int, shape) -> np.ndarray:
        out = np.zeros(int(np.prod(shape)), dtype=np.float64)
        _check(self.lib.ttq_plan_get_core(self.h, k, out.ctypes.data_as(_dp)), "ttq_plan_get_core")
        return out.reshape(shape)

    def eval_points(self, idx) -> "object":
        """idx: torch int32 (npts x d) on the GPU -> torch float64 values."""
        import torch
        idx = idx.to(device="cuda", dtype=torch.int32).contiguous()
        out = torch.empty(idx.shape[0], dtype=torch.float64, device="cuda")
        cur = torch.cuda.current_stream()
        self.stream.wait_stream(cur)                 # inputs ready before the plan's stream reads them
        _check(self.lib.ttq_plan_eval_points(self.h, _vp(idx.data_ptr()), idx.shape[0], _vp(out.data_ptr())),
               "ttq_plan_eval_points")
        cur.wait_stream(self.stream)                 # results ready before torch reads them
        idx.record_stream(self.stream)
        out.record_stream(self.stream)
        return out

    def export_tt(self, instance: int = 0) -> "TensorTrain":
        """The tensor train of the last evaluated sweep, copied into a fresh
        device buffer (torch) owned by the returned object."""
        return TensorTrain(self, instance)

    def transfer_bytes(self):
        a, b = _c.c_int64(0), _c.c_int64(0)
        _check(self.lib.ttq_plan_transfer_bytes(self.h, _c.byref(a), _c.byref(b)), "ttq_plan_transfer_bytes")
        return int(a.value), int(b.value)

    def set_graphs(self, on: bool):
        _check(self.lib.ttq_plan_set_graphs(self.h, 1 if on else 0), "ttq_plan_set_graphs")

    def set_timing(self, on: bool):
        _check(self.lib.ttq_plan_set_timing(self.h, 1 if on else 0), "ttq_plan_set_timing")

    def set_search(self, persistent: bool):
        _check(self.lib.ttq_plan_set_search(self.h, 1 if persistent else 0), "ttq_plan_set_search")

    def set_sequential(self, on: bool):
        _check(self.lib.ttq_plan_set_sequential(self.h, 1 if on else 0), "ttq_plan_set_sequential")

    def set_wait_limit(self, ns: int):
        _check(self.lib.ttq_plan_set_wait_limit(self.h, int(ns)), "ttq_plan_set_wait_limit")

    def kernel_times(self, reset: bool = False) -> Dict[str, Dict]:
        ms = (_c.c_double * len(KERNELS))()
        n = (_c.c_int64 * len(KERNELS))()
        fl = (_c.c_double * len(KERNELS))()
        _check(self.lib.ttq_plan_kernel_times(self.h, ms, n, fl, 1 if reset else 0), "ttq_plan_kernel_times")
        return {name: {"ms": ms[q], "launches": int(n[q]), "flops": fl[q]} for q, name in enumerate(KERNELS)}

    @property
    def launches(self) -> int:
        return int(self.lib.ttq_plan_launches(self.h))


class TensorTrain:
    """A TT handle (ttq_tt): cores and nested index sets in a device buffer.
    core(k) returns (core, I<=k-1, I>k) as torch tensors viewing that buffer
    (no copy), shapes (r_{k-1}, N_k, r_k), (r_{k-1}, k-1), (r_k, d-k)."""

    def __init__(self, plan, instance: int = 0):
        import torch
        self.lib = load()
        nb = _c.c_size_t(0)
        _check(self.lib.ttq_tt_bytes(plan.h, instance, _c.byref(nb)), "ttq_tt_bytes")
        self.buffer = torch.empty(max(256, int(nb.value)), dtype=torch.uint8, device="cuda")
        h = _vp()
        _check(self.lib.ttq_tt_export(plan.h, instance, _vp(self.buffer.data_ptr()), int(nb.value), _c.byref(h)),
               "ttq_tt_export")
        self.h = h
        d = _c.c_int32(0)
        ranks = (_c.c_int32 * 33)()
        _check(self.lib.ttq_tt_ranks(self.h, _c.byref(d), ranks), "ttq_tt_ranks")
        self.d = int(d.value)
        self.ranks = [int(x) for x in ranks[:self.d + 1]]

    def _view(self, ptr, count, dtype):
        import torch
        if not ptr or count == 0:
            return torch.empty(0, dtype=dtype, device="cuda")
        off = ptr - self.buffer.data_ptr()
        itemsize = 8 if dtype == torch.float64 else 4
        return self.buffer[off:off + count * itemsize].view(dtype)

    def core(self, k: int):
        import torch
        rl, n, rr = _c.c_int32(0), _c.c_int32(0), _c.c_int32(0)
        cp, lp, rp = _vp(), _vp(), _vp()
        _check(self.lib.ttq_tt_get(self.h, k, _c.byref(rl), _c.byref(n), _c.byref(rr), _c.byref(cp), _c.byref(lp),
                                   _c.byref(rp)), "ttq_tt_get")
        rl, n, rr = int(rl.value), int(n.value), int(rr.value)
        core = self._view(cp.value, rl * n * rr, torch.float64).view(rl, n, rr)
        left = self._view(lp.value, rl * (k - 1), torch.int32).view(rl, k - 1)
        right = self._view(rp.value, rr * (self.d - k), torch.int32).view(rr, self.d - k)
        return core, left, right

    def close(self):
        if getattr(self, "h", None):
            self.lib.ttq_tt_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _result_dict(res) -> Dict:
    return {"value": res.value, "value_lo": res.value_lo, "internal_conv": res.internal_conv,
            "n_eval": int(res.n_eval), "sweeps": res.sweeps, "max_rank": res.max_rank,
            "status": res.status, "status_name": STATUS_NAMES.get(res.status, str(res.status)),
            "ranks": [int(x) for x in res.ranks[:res.d + 1]]}


class Batch:
    """Many integrals advancing together: one launch per stage for all of them."""

    def __init__(self, problems: List[inputs.Problem], workspace=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise TTQError("no CUDA device: the TT-cross quadrature runs only on the GPU")
        self.lib = load()
        self.problems = list(problems)
        self.arrays = [_Arrays(p) for p in self.problems]
        self.structs = (TTQProblem * len(self.problems))(*[make_struct(p, a) for p, a in
                                                          zip(self.problems, self.arrays)])
        nbytes = _c.c_size_t(0)
        _check(self.lib.ttq_batch_workspace_bytes(self.structs, len(self.problems), _c.byref(nbytes)),
               "ttq_batch_workspace_bytes")
        self.nbytes = int(nbytes.value)
        if workspace is None:
            workspace = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        if stream is None:
            stream = torch.cuda.Stream()
            stream.wait_stream(torch.cuda.current_stream())
        self.stream = stream
        h = _vp()
        _check(self.lib.ttq_batch_create(self.structs, len(self.problems), _vp(workspace.data_ptr()), self.nbytes,
                                         _vp(self.stream.cuda_stream), _c.byref(h)), "ttq_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.ttq_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self) -> List[Dict]:
        res = (TTQResult * len(self.problems))()
        _check(self.lib.ttq_batch_run(self.h, res), "ttq_batch_run")
        return [_result_dict(r) for r in res]

    def autotune(self, sweeps: int = 3):
        chosen = (_c.c_int32 * 4)()
        _check(self.lib.ttq_batch_autotune(self.h, sweeps, chosen), "ttq_batch_autotune")
        return {"rook_ctas": chosen[0], "sample_ctas": chosen[1], "eval_ctas": chosen[2], "rook_rows": chosen[3]}

    def set_groups(self, groups: int):
        """Concurrent groups of the run graph (instances sorted by cost)."""
        _check(self.lib.ttq_batch_set_groups(self.h, groups), "ttq_batch_set_groups")

    def set_config(self, rook_ctas: int, sample_ctas: int, eval_ctas: int, rook_rows: int = 4):
        _check(self.lib.ttq_plan_set_config(self.h, rook_ctas, sample_ctas, eval_ctas), "ttq_plan_set_config")
        _check(self.lib.ttq_plan_set_rook_rows(self.h, rook_rows), "ttq_plan_set_rook_rows")

    def set_graphs(self, on: bool):
        _check(self.lib.ttq_plan_set_graphs(self.h, 1 if on else 0), "ttq_plan_set_graphs")

    def set_timing(self, on: bool):
        _check(self.lib.ttq_plan_set_timing(self.h, 1 if on else 0), "ttq_plan_set_timing")

    def kernel_times(self, reset: bool = False) -> Dict[str, Dict]:
        ms = (_c.c_double * len(KERNELS))()
        n = (_c.c_int64 * len(KERNELS))()
        fl = (_c.c_double * len(KERNELS))()
        _check(self.lib.ttq_plan_kernel_times(self.h, ms, n, fl, 1 if reset else 0), "ttq_plan_kernel_times")
        return {name: {"ms": ms[q], "launches": int(n[q]), "flops": fl[q]} for q, name in enumerate(KERNELS)}

    @property
    def launches(self) -> int:
        return int(self.lib.ttq_plan_launches(self.h))


class Server:
    """Continuous batching: requests join and leave the set in flight at sweep
    boundaries; admission by the plan footprint against a device pool."""

    def __init__(self, pool_bytes: int, max_slots: int = 512, stream=None, pool=None):
        import torch
        if not torch.cuda.is_available():
            raise TTQError("no CUDA device: the TT-cross quadrature runs only on the GPU")
        self.lib = load()
        if pool is None:
            pool = torch.empty(pool_bytes, dtype=torch.uint8, device="cuda")
        self.pool = pool
        if stream is None:
            stream = torch.cuda.Stream()
            stream.wait_stream(torch.cuda.current_stream())
        self.stream = stream
        h = _vp()
        _check(self.lib.ttq_server_create(_vp(pool.data_ptr()), pool_bytes, max_slots, _vp(stream.cuda_stream),
                                          _c.byref(h)), "ttq_server_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.ttq_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mode(self, batched: bool):
        """False (default): each request its own plan and graph, overlapping on
        the server's streams; True: requests advance together in batched sweeps."""
        _check(self.lib.ttq_server_set_mode(self.h, 1 if batched else 0), "ttq_server_set_mode")

    def submit(self, p: inputs.Problem) -> int:
        arrays = _Arrays(p)
        st = make_struct(p, arrays)
        rid = _c.c_uint64(0)
        _check(self.lib.ttq_server_submit(self.h, _c.byref(st), _c.byref(rid)), "ttq_server_submit")
        return int(rid.value)

    def step(self, sweeps: int = 1):
        a, q, c = _c.c_int(0), _c.c_int(0), _c.c_int64(0)
        _check(self.lib.ttq_server_step(self.h, sweeps, _c.byref(a), _c.byref(q), _c.byref(c)), "ttq_server_step")
        return a.value, q.value, int(c.value)

    def poll(self, rid: int):
        res = TTQResult()
        rc = self.lib.ttq_server_poll(self.h, rid, _c.byref(res))
        if rc == 4:
            return None
        _check(rc, "ttq_server_poll")
        return _result_dict(res)

    def drain(self, max_n: int = 4096):
        ids = (_c.c_uint64 * max_n)()
        res = (TTQResult * max_n)()
        n = _c.c_int(0)
        _check(self.lib.ttq_server_drain(self.h, ids, res, max_n, _c.byref(n)), "ttq_server_drain")
        return {int(ids[q]): _result_dict(res[q]) for q in range(n.value)}

    def stats(self):
        st = (_c.c_int64 * 6)()
        _check(self.lib.ttq_server_stats(self.h, st), "ttq_server_stats")
        return dict(zip(("in_flight", "queued", "admitted", "retired", "sweeps", "free_bytes"), list(st)))


def integrate(p: inputs.Problem) -> Dict:
    """Convenience: one plan, one full run."""
    plan = Plan(p)
    try:
        return plan.run()
    finally:
        plan.close()
