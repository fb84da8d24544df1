"""Grouped modes on the GPU: the reactive flow as the TDB-2 (DBO) scheme of Sec. 3.2, one
two-dimensional spatial mode (32 x 16 points) and the species mode, against the oracle.

FP32 and BF16: the bounds of the three-mode reactive tests.  FP64: the rank controller's
actions, ranks and errors step by step, as for the three-mode decision test.
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_06958_gb300 import synth as S

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


@pytest.fixture(scope="module")
def tdbmod():
    from paper_2201_06958_gb300 import build_lib, tdb
    build_lib.build()
    return tdb


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@cuda
@pytest.mark.parametrize("precision,eps_tol,rec_tol", [("fp32", 1e-3, 1e-5), ("bf16", 0.02, 5e-4)])
def test_dbo_reactive_tracks_oracle(tdbmod, precision, eps_tol, rec_tol):
    """40 Euler steps at ranks (8, 8) from the oracle's HOSVD state; the step record's CR is
    the TDB-2 storage ratio of Sec. 3.2."""
    wl = S.make_workload("reactive_dbo")
    w = wl.weights
    snaps = [wl.snapshot(k, device="cuda") for k in range(41)]
    V0 = S.to_logical(snaps[0])
    T, U, _ = O.hosvd(V0, w, [8, 8])
    c = tdbmod.TDB(wl.dims, [8, 8], weights=w, precision=precision, error_mode="exact")
    c.init_from_factors(T, U, snaps[0])
    To, Uo, Vp = T, U, V0
    worst = 0.0
    for k in range(1, 41):
        info = c.push(snaps[k])
        Vk = S.to_logical(snaps[k])
        To, Uo, _, _ = O.step_euler(To, Uo, w, Vp, Vk)
        Vp = Vk
        eo = O.error_exact(Vk, To, Uo, w)
        worst = max(worst, abs(info["eps"] - eo) / eo)
    Tg, Ug = c.factors()
    r = rel(O.reconstruct(Tg, Ug), O.reconstruct(To, Uo))
    assert r <= rec_tol, (r, worst)
    assert worst <= eps_tol, (r, worst)
    assert abs(info["cr"] - 32 * 16 * 12 / O.storage_tdb2(8, 32, 16, 12)) <= 1e-12 * info["cr"]


@cuda
def test_dbo_rank_control_matches_oracle(tdbmod):
    """Sec. 2.5 on the grouped stream (FP64, 150 steps): both ranks move together (the
    two-mode bound r_1 <= r_2 <= r_1), and every step's action, ranks and error equal
    the oracle controller's."""
    wl = S.make_workload("reactive_dbo")
    w = wl.weights
    snaps = [wl.snapshot(k, device="cuda", dtype=torch.float64) for k in range(151)]
    logical = [S.to_logical(x) for x in snaps]
    eps_th, gamma_th, K = 5e-5, 99.99, 5
    ctrl = O.ControllerConfig(eps_th, gamma_th, K, [12, 12])
    _, recs = O.compress_stream(logical, w, [0, 0], ctrl)
    c = tdbmod.TDB(wl.dims, [0, 0], rank_max=[12, 12], weights=w, eps_th=eps_th, gamma_th=gamma_th,
                   slope_window=K, precision="fp64", error_mode="exact")
    c.init(snaps[0])
    seen = set()
    for k in range(1, 151):
        info = c.push(snaps[k])
        rec = recs[k - 1]
        assert info["action"] == rec.action, (k, info["action"], rec.action)
        assert info["ranks"] == rec.ranks, (k, info["ranks"], rec.ranks)
        assert info["reinit"] == rec.reinit, k
        assert abs(info["eps"] - rec.eps) <= 1e-8 * rec.eps, (k, info["eps"], rec.eps)
        assert info["ranks"][0] == info["ranks"][1]
        seen.add(info["action"])
    assert {"increase", "reinit"} <= seen, seen


@cuda
def test_dbo_bf16_adaptive_stream(tdbmod):
    """The grouped stream with the BF16 projection and the float HOSVD (its 512-point mode
    has a Gram of rank <= 12): 120 adaptive steps, the error after control below eps_th at
    every step, both ranks equal, and the reported error that of the returned factors."""
    wl = S.make_workload("reactive_dbo")
    w = wl.weights
    snaps = [wl.snapshot(k, device="cuda") for k in range(121)]
    c = tdbmod.TDB(wl.dims, [0, 0], rank_max=[12, 12], weights=w, eps_th=5e-5, gamma_th=99.99, slope_window=5,
                   precision="bf16", error_mode="exact")
    c.init(snaps[0])
    for k in range(1, 121):
        info = c.push(snaps[k])
        assert info["ranks"][0] == info["ranks"][1], (k, info)
        assert info["eps"] <= 5e-5 or info["action"] == "cap", (k, info)
    Tg, Ug = c.factors()
    e = O.error_exact(S.to_logical(snaps[120]), Tg, Ug, w)
    assert abs(info["eps"] - e) <= 0.02 * e, (info["eps"], e)
