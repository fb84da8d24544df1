"""ctypes binding of libtdb (include/tdb.h): argument marshalling only.

Every computation runs in libtdb's CUDA kernels.  PyTorch provides device
memory (the workspace and snapshots) and the stream.  Loading fails loudly when
libtdb.so has not been built; there is no CPU fallback.

Snapshot convention: a logical N_1 x ... x N_p tensor is a C-contiguous torch
tensor of shape (N_p, ..., N_1) (column-major, mode 1 fastest), float64 in
"fp64" mode and float32 otherwise.
"""

from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdb.so")
MAX_MODES = 4
MAX_RANK = 32

PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2}
ERROR_MODE = {"exact": 0, "every_k": 1, "mlp": 2, "none": 3}
INTEGRATOR = {"euler": 0, "heun": 1, "rk2_central": 2}
ACTIONS = {0: "none", 1: "reinit", 2: "increase", 3: "decrease", 4: "revert", 5: "cap"}

TDB_OK = 0
TDB_WARN_RANK_CAP = 9


class tdb_config(C.Structure):
    _fields_ = [
        ("ndim", C.c_int),
        ("dims", C.c_int64 * MAX_MODES),
        ("rank", C.c_int * MAX_MODES),
        ("rank_max", C.c_int * MAX_MODES),
        ("weights", C.POINTER(C.c_double) * MAX_MODES),
        ("eps_th", C.c_double),
        ("gamma_th", C.c_double),
        ("slope_window", C.c_int),
        ("precision", C.c_int),
        ("error_mode", C.c_int),
        ("error_every", C.c_int),
        ("reorth", C.c_int),
        ("integrator", C.c_int),
    ]


class tdb_profile(C.Structure):
    _fields_ = [("steps", C.c_int64), ("ms_project", C.c_double), ("ms_project_main", C.c_double),
                ("ms_update", C.c_double), ("ms_error", C.c_double), ("ms_control", C.c_double),
                ("launches_main", C.c_int64), ("update_phases", C.c_int64),
                ("us_update_phase", C.c_double * 12), ("us_project_span", C.c_double), ("spans", C.c_int64)]


class tdb_step_info(C.Structure):
    _fields_ = [
        ("step", C.c_int64),
        ("eps", C.c_double),
        ("eps_exact", C.c_int),
        ("eps_step", C.c_double),
        ("gamma", C.c_double * MAX_MODES),
        ("sigma_min", C.c_double * MAX_MODES),
        ("ranks", C.c_int * MAX_MODES),
        ("reinit", C.c_int),
        ("action", C.c_int),
        ("cr", C.c_double),
        ("dv_norm", C.c_double),
        ("ds_norm", C.c_double),
        ("eps_est", C.c_double),
        ("gate", C.c_int),
    ]


_lib = None

EXPORTS = [
    "tdb_workspace_bytes", "tdb_init", "tdb_init_from_factors", "tdb_push_snapshot", "tdb_reconstruct",
    "tdb_adapt_rank", "tdb_reinit", "tdb_get_factors", "tdb_get_projection", "tdb_get_counters", "tdb_save_state",
    "tdb_load_state", "tdb_last_error", "tdb_status_string", "tdb_destroy", "tdb_version",
    "tdb_set_profiling", "tdb_get_profile", "tdb_kernel_launches", "tdb_project_noalloc",
    "tdb_mlp_param_count", "tdb_mlp_forward", "tdb_mlp_loss_grad", "tdb_mlp_adam_step", "tdb_estimator_fit",
    "tdb_estimator_params", "tdb_estimator_trace", "tdb_set_input_slots", "tdb_push_slot",
    "tdb_batch_create", "tdb_batch_push", "tdb_batch_last_error", "tdb_batch_destroy", "tdb_get_graph_counters",
    "tdb_selftest_recip", "tdb_selftest_timeout", "tdb_tc_tuning", "tdb_estimator_load_trace",
]


def load(path: str = LIB_PATH):
    """Load libtdb.so (build it first with paper_2201_06958_gb300.build_lib)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libtdb.so not found at {path}: build it with "
                          "`python -m paper_2201_06958_gb300.build_lib` (nvcc, sm_103a)")
    lib = C.CDLL(path)
    vp, sz, st = C.c_void_p, C.c_size_t, C.c_int
    lib.tdb_workspace_bytes.argtypes = [C.POINTER(tdb_config)]
    lib.tdb_workspace_bytes.restype = sz
    lib.tdb_init.argtypes = [C.POINTER(vp), C.POINTER(tdb_config), vp, sz, vp, vp]
    lib.tdb_init.restype = st
    lib.tdb_init_from_factors.argtypes = [C.POINTER(vp), C.POINTER(tdb_config), vp, sz, C.POINTER(C.c_double),
                                          C.POINTER(C.POINTER(C.c_double)), C.POINTER(C.c_int), vp, vp]
    lib.tdb_init_from_factors.restype = st
    lib.tdb_push_snapshot.argtypes = [vp, vp, C.POINTER(tdb_step_info)]
    lib.tdb_push_snapshot.restype = st
    lib.tdb_reconstruct.argtypes = [vp, vp]
    lib.tdb_reconstruct.restype = st
    lib.tdb_adapt_rank.argtypes = [vp, vp, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    lib.tdb_adapt_rank.restype = st
    lib.tdb_reinit.argtypes = [vp, vp]
    lib.tdb_reinit.restype = st
    lib.tdb_get_factors.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.POINTER(C.c_double)), C.POINTER(C.c_int)]
    lib.tdb_get_factors.restype = st
    lib.tdb_get_projection.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.POINTER(C.c_double))]
    lib.tdb_get_projection.restype = st
    lib.tdb_get_counters.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.tdb_get_counters.restype = st
    lib.tdb_save_state.argtypes = [vp, vp, C.POINTER(sz)]
    lib.tdb_save_state.restype = st
    lib.tdb_load_state.argtypes = [vp, vp, sz, vp]
    lib.tdb_load_state.restype = st
    lib.tdb_last_error.argtypes = [vp]
    lib.tdb_last_error.restype = C.c_char_p
    lib.tdb_status_string.argtypes = [st]
    lib.tdb_status_string.restype = C.c_char_p
    lib.tdb_destroy.argtypes = [vp]
    lib.tdb_destroy.restype = None
    lib.tdb_version.argtypes = []
    lib.tdb_version.restype = C.c_char_p
    lib.tdb_set_input_slots.argtypes = [vp, vp, vp]
    lib.tdb_set_input_slots.restype = st
    lib.tdb_push_slot.argtypes = [vp, C.c_int, C.POINTER(tdb_step_info)]
    lib.tdb_push_slot.restype = st
    lib.tdb_batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int, C.c_int, vp]
    lib.tdb_batch_create.restype = st
    lib.tdb_batch_push.argtypes = [vp, C.c_int, vp]
    lib.tdb_batch_push.restype = st
    lib.tdb_batch_last_error.argtypes = [vp]
    lib.tdb_batch_last_error.restype = C.c_char_p
    lib.tdb_batch_destroy.argtypes = [vp]
    lib.tdb_batch_destroy.restype = None
    lib.tdb_get_graph_counters.argtypes = [vp, vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.tdb_get_graph_counters.restype = st
    lib.tdb_set_profiling.argtypes = [vp, C.c_int]
    lib.tdb_set_profiling.restype = st
    lib.tdb_get_profile.argtypes = [vp, vp]
    lib.tdb_get_profile.restype = st
    lib.tdb_kernel_launches.argtypes = []
    lib.tdb_kernel_launches.restype = C.c_int64
    lib.tdb_project_noalloc.argtypes = [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int), vp, vp,
                                        C.POINTER(vp), C.POINTER(vp), vp, C.POINTER(vp), vp, vp]
    lib.tdb_project_noalloc.restype = st
    lib.tdb_estimator_load_trace.argtypes = [vp, vp, vp, C.c_int, C.c_int]
    lib.tdb_estimator_load_trace.restype = st
    lib.tdb_tc_tuning.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_int), C.POINTER(C.c_float)]
    lib.tdb_tc_tuning.restype = st
    lib.tdb_selftest_recip.argtypes = [vp, vp, vp, C.c_int64, vp]
    lib.tdb_selftest_recip.restype = st
    lib.tdb_selftest_timeout.argtypes = [C.c_int, C.c_int64, vp, vp]
    lib.tdb_selftest_timeout.restype = st
    lib.tdb_mlp_param_count.argtypes = []
    lib.tdb_mlp_param_count.restype = C.c_int
    lib.tdb_mlp_forward.argtypes = [vp, vp, C.c_int, vp, vp]
    lib.tdb_mlp_forward.restype = st
    lib.tdb_mlp_loss_grad.argtypes = [vp, vp, vp, C.c_int, vp, sz, vp, vp, vp]
    lib.tdb_mlp_loss_grad.restype = st
    lib.tdb_mlp_adam_step.argtypes = [vp, vp, vp, vp, C.c_int, C.c_float, vp]
    lib.tdb_mlp_adam_step.restype = st
    lib.tdb_estimator_fit.argtypes = [vp, C.c_int, C.c_float, C.c_uint64, C.c_double, C.POINTER(C.c_double)]
    lib.tdb_estimator_fit.restype = st
    lib.tdb_estimator_params.argtypes = [vp, vp, vp, C.c_double]
    lib.tdb_estimator_params.restype = st
    lib.tdb_estimator_trace.argtypes = [vp, vp, vp, C.POINTER(C.c_int)]
    lib.tdb_estimator_trace.restype = st
    _lib = lib
    return lib


class TDBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{load().tdb_status_string(status).decode()}: {msg}")
        self.status = status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_config(dims: Sequence[int], rank: Sequence[int], rank_max: Optional[Sequence[int]] = None,
                weights: Optional[Sequence[Optional[np.ndarray]]] = None, eps_th: float = 0.0,
                gamma_th: float = 99.999, slope_window: int = 10, precision: str = "fp32",
                error_mode: str = "exact", error_every: int = 1, reorth: bool = True,
                integrator: str = "euler"):
    """Build a tdb_config; returns (config, keepalive) - keep the second alive while the config is used."""
    p = len(dims)
    cfg = tdb_config()
    cfg.ndim = p
    keep = []
    for n in range(p):
        cfg.dims[n] = int(dims[n])
        cfg.rank[n] = int(rank[n])
        cfg.rank_max[n] = int(rank_max[n]) if rank_max is not None else 0
        if weights is not None and weights[n] is not None:
            w = np.ascontiguousarray(weights[n], dtype=np.float64)
            keep.append(w)
            cfg.weights[n] = _dptr(w)
    cfg.eps_th = float(eps_th)
    cfg.gamma_th = float(gamma_th)
    cfg.slope_window = int(slope_window)
    cfg.precision = PRECISION[precision]
    cfg.error_mode = ERROR_MODE[error_mode]
    cfg.error_every = int(error_every)
    cfg.reorth = 1 if reorth else 0
    cfg.integrator = INTEGRATOR[integrator]
    return cfg, keep


class TDB:
    """One compressor context.  ``device`` defaults to cuda:0; the stream is the
    current torch stream of that device at construction."""

    def __init__(self, dims, rank, rank_max=None, weights=None, eps_th=0.0, gamma_th=99.999, slope_window=10,
                 precision="fp32", error_mode="exact", error_every=1, reorth=True, integrator="euler",
                 device=None, stream=None):
        self.lib = load()
        self.dims = [int(d) for d in dims]
        self.p = len(self.dims)
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.device = torch.device(device or "cuda:0")
        self.cfg, self._keep = make_config(dims, rank, rank_max, weights, eps_th, gamma_th, slope_window,
                                           precision, error_mode, error_every, reorth, integrator)
        nbytes = self.lib.tdb_workspace_bytes(C.byref(self.cfg))
        if nbytes == 0:
            raise TDBError(1, "invalid configuration")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = C.c_void_p()
        self._prev = None

    @property
    def storage_shape(self):
        return tuple(reversed(self.dims))

    def _check(self, status: int, ctx=True):
        if status not in (TDB_OK, TDB_WARN_RANK_CAP):
            msg = self.lib.tdb_last_error(self.ctx if ctx else None).decode()
            raise TDBError(status, msg)
        return status

    def _snap(self, V: torch.Tensor) -> torch.Tensor:
        if V.dtype != self.dtype or V.device != self.device or not V.is_contiguous() or tuple(V.shape) != self.storage_shape:
            raise ValueError(f"snapshot must be a contiguous {self.dtype} tensor of shape {self.storage_shape} on "
                             f"{self.device}")
        return V

    def init(self, V0: torch.Tensor):
        V0 = self._snap(V0)
        st = self.lib.tdb_init(C.byref(self.ctx), C.byref(self.cfg), C.c_void_p(self.workspace.data_ptr()),
                               self.workspace.numel(), C.c_void_p(V0.data_ptr()), C.c_void_p(self.stream.cuda_stream))
        self._check(st, ctx=False)
        self._prev = V0
        return self

    def init_from_factors(self, core: np.ndarray, U: Sequence[np.ndarray], V0: torch.Tensor):
        """core: logical (r_1, ..., r_p) float64; U[n]: (N_n, r_n) float64."""
        V0 = self._snap(V0)
        core_f = np.asfortranarray(core, dtype=np.float64).ravel(order="F")
        Us = [np.asfortranarray(u, dtype=np.float64).ravel(order="F") for u in U]
        ranks = (C.c_int * self.p)(*[int(s) for s in core.shape])
        uptr = (C.POINTER(C.c_double) * self.p)(*[_dptr(u) for u in Us])
        st = self.lib.tdb_init_from_factors(C.byref(self.ctx), C.byref(self.cfg),
                                            C.c_void_p(self.workspace.data_ptr()), self.workspace.numel(),
                                            _dptr(core_f), uptr, ranks, C.c_void_p(V0.data_ptr()),
                                            C.c_void_p(self.stream.cuda_stream))
        self._check(st, ctx=False)
        self._prev = V0
        return self

    def push(self, V: torch.Tensor) -> dict:
        V = self._snap(V)
        info = tdb_step_info()
        st = self.lib.tdb_push_snapshot(self.ctx, C.c_void_p(V.data_ptr()), C.byref(info))
        self._check(st)
        self._prev2, self._prev = self._prev, V      # borrowed by the library until the next pushes
        return {
            "step": info.step, "eps": info.eps, "eps_exact": bool(info.eps_exact), "eps_step": info.eps_step,
            "gamma": list(info.gamma)[: self.p], "sigma_min": list(info.sigma_min)[: self.p],
            "ranks": list(info.ranks)[: self.p], "reinit": info.reinit, "action": ACTIONS.get(info.action, "?"),
            "cr": info.cr, "dv_norm": info.dv_norm, "ds_norm": info.ds_norm, "eps_est": info.eps_est,
            "gate": info.gate, "status": st,
        }

    def push_raw(self, ptr: int, info: Optional[tdb_step_info] = None) -> int:
        """Push a snapshot given by device address (no checks); returns the status."""
        return self.lib.tdb_push_snapshot(self.ctx, C.c_void_p(ptr), C.byref(info) if info is not None else None)

    def set_input_slots(self, slot0: Optional[torch.Tensor], slot1: Optional[torch.Tensor]):
        """Two snapshot buffers owned by the caller; steps then read V_{k+1} from one and
        V_k from the other (``push_slot``).  None, None removes them."""
        if slot0 is None and slot1 is None:
            self._check(self.lib.tdb_set_input_slots(self.ctx, None, None))
            self._slots = None
            return self
        a, b = self._snap(slot0), self._snap(slot1)
        self._check(self.lib.tdb_set_input_slots(self.ctx, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr())))
        self._slots = (a, b)
        return self

    def push_slot(self, parity: int) -> dict:
        """One step with V_{k+1} in slot ``parity`` (recorded once, then replayed as a graph)."""
        info = tdb_step_info()
        st = self.lib.tdb_push_slot(self.ctx, int(parity), C.byref(info))
        self._check(st)
        self._prev = self._slots[parity]
        return self._info_dict(info, st)

    def _info_dict(self, info, st):
        return {
            "step": info.step, "eps": info.eps, "eps_exact": bool(info.eps_exact), "eps_step": info.eps_step,
            "gamma": list(info.gamma)[: self.p], "sigma_min": list(info.sigma_min)[: self.p],
            "ranks": list(info.ranks)[: self.p], "reinit": info.reinit, "action": ACTIONS.get(info.action, "?"),
            "cr": info.cr, "dv_norm": info.dv_norm, "ds_norm": info.ds_norm, "eps_est": info.eps_est,
            "gate": info.gate, "status": st,
        }

    def reconstruct(self, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.storage_shape, dtype=self.dtype, device=self.device)
        self._check(self.lib.tdb_reconstruct(self.ctx, C.c_void_p(self._snap(out).data_ptr())))
        return out

    def reinit(self, V: torch.Tensor):
        """Truncated HOSVD of V at the current ranks (tdb_reinit); V becomes the previous snapshot."""
        V = self._snap(V)
        self._check(self.lib.tdb_reinit(self.ctx, C.c_void_p(V.data_ptr())))
        self._prev = V
        return self

    def adapt_rank(self, V: torch.Tensor):
        V = self._snap(V)
        ranks = (C.c_int * self.p)()
        eps = C.c_double()
        st = self.lib.tdb_adapt_rank(self.ctx, C.c_void_p(V.data_ptr()), ranks, C.byref(eps))
        self._check(st)
        self._prev = V
        return list(ranks), eps.value

    def ranks(self) -> List[int]:
        r = (C.c_int * self.p)()
        self._check(self.lib.tdb_get_factors(self.ctx, None, None, r))
        return list(r)

    def factors(self):
        """(core (r_1..r_p) float64, [U_n (N_n x r_n)]) as numpy arrays in logical index order."""
        r = self.ranks()
        core = np.empty(int(np.prod(r)), dtype=np.float64)
        Us = [np.empty(self.dims[n] * r[n], dtype=np.float64) for n in range(self.p)]
        uptr = (C.POINTER(C.c_double) * self.p)(*[_dptr(u) for u in Us])
        self._check(self.lib.tdb_get_factors(self.ctx, _dptr(core), uptr, None))
        return (core.reshape(r, order="F"),
                [u.reshape(self.dims[n], r[n], order="F") for n, u in enumerate(Us)])

    def projection(self):
        """(dS, [Y_n tensors]) of the last step, logical index order; Y_n has mode n of size N_n."""
        r = self.ranks()
        dS = np.empty(int(np.prod(r)), dtype=np.float64)
        shapes = []
        for n in range(self.p):
            sh = list(r)
            sh[n] = self.dims[n]
            shapes.append(sh)
        Ys = [np.empty(int(np.prod(sh)), dtype=np.float64) for sh in shapes]
        yptr = (C.POINTER(C.c_double) * self.p)(*[_dptr(y) for y in Ys])
        self._check(self.lib.tdb_get_projection(self.ctx, _dptr(dS), yptr))
        return dS.reshape(r, order="F"), [y.reshape(sh, order="F") for y, sh in zip(Ys, shapes)]

    def set_profiling(self, enable: bool):
        """Start (and zero) or stop the per-phase device timers (tdb_set_profiling)."""
        self._check(self.lib.tdb_set_profiling(self.ctx, 1 if enable else 0))

    def profile(self) -> dict:
        """Accumulated device milliseconds per phase of tdb_push_snapshot (tdb_get_profile)."""
        pr = tdb_profile()
        self._check(self.lib.tdb_get_profile(self.ctx, C.byref(pr)))
        return {"steps": pr.steps, "ms_project": pr.ms_project, "ms_project_main": pr.ms_project_main,
                "ms_update": pr.ms_update, "ms_error": pr.ms_error, "ms_control": pr.ms_control,
                "us_update_phase": [pr.us_update_phase[i] for i in range(pr.update_phases)],
                "us_project_span": pr.us_project_span, "spans": pr.spans}

    def counters(self):
        s, r, e = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self.lib.tdb_get_counters(self.ctx, C.byref(s), C.byref(r), C.byref(e)))
        g, gr = C.c_int64(), C.c_int64()
        self._check(self.lib.tdb_get_graph_counters(self.ctx, None, C.byref(g), C.byref(gr)))
        return {"steps": s.value, "reinits": r.value, "exact_evals": e.value, "graph_replays": g.value,
                "graph_records": gr.value}

    def tuning(self) -> dict:
        """The tensor-core projection's launch shape (tdb_tc_tuning): CTAs per tile position,
        the finish's split target, and the candidates the tuner timed (us per launch)."""
        ctas, fin, nc = C.c_int(), C.c_int(), C.c_int()
        cand, cus = (C.c_int * 4)(), (C.c_float * 4)()
        fc, fus = (C.c_int * 3)(), (C.c_float * 3)()
        self._check(self.lib.tdb_tc_tuning(self.ctx, C.byref(ctas), C.byref(fin), C.byref(nc), cand, cus, fc, fus))
        return {"ctas_per_position": ctas.value, "finish_split_target": fin.value, "timed": nc.value > 0,
                "candidates": {int(cand[i]): float(cus[i]) for i in range(nc.value)},
                "finish_candidates": {int(fc[i]): float(fus[i]) for i in range(3) if nc.value > 0}}

    def save_state(self) -> bytes:
        n = C.c_size_t(0)
        self._check(self.lib.tdb_save_state(self.ctx, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(self.lib.tdb_save_state(self.ctx, buf, C.byref(n)))
        return bytes(buf.raw[: n.value])

    def load_state(self, blob: bytes, V_prev: torch.Tensor):
        V_prev = self._snap(V_prev)
        buf = C.create_string_buffer(blob, len(blob))
        self._check(self.lib.tdb_load_state(self.ctx, buf, len(blob), C.c_void_p(V_prev.data_ptr())))
        self._prev = V_prev

    def estimator_fit(self, iters: int = 2000, lr: float = 3e-3, seed: int = 1, gate: float = 0.5) -> float:
        loss = C.c_double()
        self._check(self.lib.tdb_estimator_fit(self.ctx, iters, lr, seed, gate, C.byref(loss)))
        return loss.value

    def estimator_params(self, set_params: Optional[np.ndarray] = None, gate: float = 0.0) -> np.ndarray:
        n = self.lib.tdb_mlp_param_count() + 18
        out = np.empty(n, dtype=np.float32)
        inp = None if set_params is None else np.ascontiguousarray(set_params, dtype=np.float32)
        self._check(self.lib.tdb_estimator_params(
            self.ctx, out.ctypes.data_as(C.c_void_p), None if inp is None else inp.ctypes.data_as(C.c_void_p), gate))
        return out

    def estimator_trace(self):
        n = C.c_int(0)
        self._check(self.lib.tdb_estimator_trace(self.ctx, None, None, C.byref(n)))
        X = np.empty((n.value, 8), dtype=np.float32)
        t = np.empty(n.value, dtype=np.float32)
        self._check(self.lib.tdb_estimator_trace(self.ctx, X.ctypes.data_as(C.c_void_p), t.ctypes.data_as(C.c_void_p),
                                                 C.byref(n)))
        return X, t

    def estimator_load_trace(self, X: np.ndarray, t: np.ndarray, append: bool = False):
        """Install training rows (n x 8 features, n targets) recorded elsewhere."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        self._check(self.lib.tdb_estimator_load_trace(self.ctx, X.ctypes.data_as(C.c_void_p),
                                                      t.ctypes.data_as(C.c_void_p), int(t.size), int(append)))
        return self

    def close(self):
        if self.ctx:
            self.lib.tdb_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent contexts stepped together: every member's step recorded into one
    graph over ``nstreams`` streams, one synchronisation per batch step.  Members must
    be initialised and have input slots; they stay owned by the caller."""

    def __init__(self, members: Sequence[TDB], nstreams: int = 8, stream=None):
        self.lib = load()
        self.members = list(members)
        arr = (C.c_void_p * len(self.members))(*[m.ctx.value for m in self.members])
        self.stream = stream or torch.cuda.current_stream(self.members[0].device)
        self.b = C.c_void_p()
        st = self.lib.tdb_batch_create(C.byref(self.b), arr, len(self.members), int(nstreams),
                                       C.c_void_p(self.stream.cuda_stream))
        if st != TDB_OK:
            raise TDBError(st, "batch create")
        self._infos = (tdb_step_info * len(self.members))()

    def push(self, parity: int) -> List[dict]:
        st = self.lib.tdb_batch_push(self.b, int(parity), C.cast(self._infos, C.c_void_p))
        if st not in (TDB_OK, TDB_WARN_RANK_CAP):
            raise TDBError(st, self.lib.tdb_batch_last_error(self.b).decode())
        out = []
        for m, info in zip(self.members, self._infos):
            m._prev = m._slots[parity]
            out.append(m._info_dict(info, st))
        return out

    def counters(self):
        g, gr = C.c_int64(), C.c_int64()
        st = self.lib.tdb_get_graph_counters(None, self.b, C.byref(g), C.byref(gr))
        if st != TDB_OK:
            raise TDBError(st, "graph counters")
        return {"graph_replays": g.value, "graph_records": gr.value}

    def close(self):
        if self.b:
            self.lib.tdb_batch_destroy(self.b)
            self.b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def project_noalloc(dims, ranks, V_next: torch.Tensor, V_prev: torch.Tensor, A, w, dS: torch.Tensor,
                    Y, dv2: torch.Tensor, stream=None) -> int:
    """tdb_project_noalloc (include/tdb.h): the fused difference + projection into
    caller-owned device outputs, with no device allocation inside the library.
    A[n]: float32 (N_n, r_n) device tensors of W_n U_n in column-major order;
    w[n]: float64 device tensors; dS, Y[n], dv2: float32 / float64 device outputs.
    Returns the tdb_status code."""
    lib = load()
    p = len(dims)
    cdims = (C.c_int64 * p)(*[int(d) for d in dims])
    cr = (C.c_int * p)(*[int(r) for r in ranks])
    aptr = (C.c_void_p * p)(*[a.data_ptr() for a in A])
    wptr = (C.c_void_p * p)(*[x.data_ptr() for x in w])
    yptr = (C.c_void_p * p)(*[y.data_ptr() for y in Y])
    s = stream if stream is not None else torch.cuda.current_stream(V_next.device)
    return lib.tdb_project_noalloc(p, cdims, cr, C.c_void_p(V_next.data_ptr()), C.c_void_p(V_prev.data_ptr()),
                                   aptr, wptr, C.c_void_p(dS.data_ptr()), yptr, C.c_void_p(dv2.data_ptr()),
                                   C.c_void_p(s.cuda_stream))


def selftest_recip(x: torch.Tensor):
    """tdb_selftest_recip on a float64 device tensor: (1/x, 1/sqrt(x)) from the library's
    double reciprocal helpers."""
    lib = load()
    x = x.contiguous()
    rcp, rs = torch.empty_like(x), torch.empty_like(x)
    st = lib.tdb_selftest_recip(C.c_void_p(x.data_ptr()), C.c_void_p(rcp.data_ptr()), C.c_void_p(rs.data_ptr()),
                                x.numel(), C.c_void_p(torch.cuda.current_stream(x.device).cuda_stream))
    if st != 0:
        raise TDBError(st, "tdb_selftest_recip")
    return rcp, rs


def selftest_timeout(which: int, limit_cycles: int, device="cuda") -> int:
    """tdb_selftest_timeout: run one bounded device wait until it runs out; returns the
    status (TDB_ERR_TIMEOUT = 7 expected)."""
    lib = load()
    scratch = torch.zeros(4, dtype=torch.int32, device=device)
    return lib.tdb_selftest_timeout(int(which), int(limit_cycles), C.c_void_p(scratch.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream(scratch.device).cuda_stream))


def mlp_forward(params: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
    """tdb_mlp_forward on device tensors (float32)."""
    lib = load()
    y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    st = lib.tdb_mlp_forward(C.c_void_p(params.data_ptr()), C.c_void_p(X.data_ptr()), X.shape[0],
                             C.c_void_p(y.data_ptr()), C.c_void_p(torch.cuda.current_stream(X.device).cuda_stream))
    if st != 0:
        raise TDBError(st, "tdb_mlp_forward")
    return y


def mlp_loss_grad(params: torch.Tensor, X: torch.Tensor, t: torch.Tensor):
    """tdb_mlp_loss_grad on device tensors (float32); returns (loss tensor, grad tensor)."""
    lib = load()
    npar = lib.tdb_mlp_param_count()
    scratch = torch.empty(1024 * (npar + 1), dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    grad = torch.empty(npar, dtype=torch.float32, device=X.device)
    st = lib.tdb_mlp_loss_grad(C.c_void_p(params.data_ptr()), C.c_void_p(X.data_ptr()), C.c_void_p(t.data_ptr()),
                               X.shape[0], C.c_void_p(scratch.data_ptr()), scratch.numel(),
                               C.c_void_p(loss.data_ptr()), C.c_void_p(grad.data_ptr()),
                               C.c_void_p(torch.cuda.current_stream(X.device).cuda_stream))
    if st != 0:
        raise TDBError(st, "tdb_mlp_loss_grad")
    return loss, grad


def mlp_adam_step(params: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: int, lr: float):
    lib = load()
    st = lib.tdb_mlp_adam_step(C.c_void_p(params.data_ptr()), C.c_void_p(grad.data_ptr()), C.c_void_p(m.data_ptr()),
                               C.c_void_p(v.data_ptr()), step, lr,
                               C.c_void_p(torch.cuda.current_stream(params.device).cuda_stream))
    if st != 0:
        raise TDBError(st, "tdb_mlp_adam_step")
