"""The midpoint RK2 scheme with central differences of the data (TDB_RK2_CENTRAL) on the
GPU against the oracle's step_rk2_central.

Stage 1 takes (V_{k+1} - V_{k-1}) / 4 over half a step (or (V_{k+1} - V_k) / 2 on the
first step), stage 2 takes V_{k+1} - V_k at the midpoint state over the whole step
(Sec. 3.1's central second-order approximation of the data derivative with a
second-order RK scheme).  FP64: 1e-10 relative on T x U, sigma^(n) and epsilon, as for
the Euler and Heun steps (plus the rounding floor of epsilon where it is tiny against
||V||_W).  BF16: the bounds of the corresponding Euler test (two projections per step).
Input slots hold two snapshots and refuse the scheme.
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
def test_rk2_central_fp64_analytic_matches_oracle(tdbmod):
    """32^3 exact-rank-4 field, dt = 4e-3, 50 steps in FP64 from the oracle's HOSVD state:
    T x U and sigma^(n) within 1e-10 of the oracle's run every 10 steps, epsilon every
    step, bases W-orthonormal, and the error far below Euler's at the same dt."""
    wl = S.make_workload("analytic", n=32, dt=4e-3, steps=50)
    w = wl.weights
    V0 = wl.logical(0)
    T, U, _ = O.hosvd(V0, w, [4, 4, 4])
    c = tdbmod.TDB(wl.dims, [4, 4, 4], weights=w, precision="fp64", error_mode="exact", integrator="rk2_central")
    snaps = [wl.snapshot(k, device="cuda") for k in range(wl.steps + 1)]
    c.init_from_factors(T, U, snaps[0])
    To, Uo, Te, Ue = T, U, T, U
    Vpp, Vp = None, V0
    worst = {"rec": 0.0, "sig": 0.0, "eps": 0.0}
    for k in range(1, wl.steps + 1):
        info = c.push(snaps[k])
        Vk = S.to_logical(snaps[k])
        To, Uo = O.step_rk2_central(To, Uo, w, Vpp, Vp, Vk)
        Te, Ue, _, _ = O.step_euler(Te, Ue, w, Vp, Vk)
        Vpp, Vp = Vp, Vk
        eo = O.error_exact(Vk, To, Uo, w)
        tol = 1e-10 * eo + 1e-13 * np.sqrt(O.weighted_norm2(Vk, w))
        worst["eps"] = max(worst["eps"], abs(info["eps"] - eo) / tol)
        if k % 10 == 0:
            Tg, Ug = c.factors()
            worst["rec"] = max(worst["rec"], rel(O.reconstruct(Tg, Ug), O.reconstruct(To, Uo)))
            for a, b in zip(O.core_singular_values(Tg), O.core_singular_values(To)):
                worst["sig"] = max(worst["sig"], rel(a, b))
            for n in range(3):
                assert np.abs(Ug[n].T @ (w[n][:, None] * Ug[n]) - np.eye(4)).max() <= 1e-12
    assert worst["rec"] <= 1e-10, worst
    assert worst["sig"] <= 1e-10, worst
    assert worst["eps"] <= 1.0, worst
    assert info["eps"] < O.error_exact(Vp, Te, Ue, w) / 10.0


@cuda
@pytest.mark.parametrize("precision,eps_bound,rec_bound", [("fp32", 1e-3, 1e-5), ("bf16", 2e-2, 5e-4)])
def test_rk2_central_reactive_tracks_oracle(tdbmod, precision, eps_bound, rec_bound):
    """The reactive stream, ranks (11, 11, 7), 40 steps from the oracle's HOSVD state:
    epsilon within the stated relative bound every step and T x U at the end."""
    wl = S.make_workload("reactive")
    w = wl.weights
    snaps = [wl.snapshot(k, device="cuda") for k in range(41)]
    V0 = S.to_logical(snaps[0])
    T, U, _ = O.hosvd(V0, w, [11, 11, 7])
    c = tdbmod.TDB(wl.dims, [11, 11, 7], weights=w, precision=precision, error_mode="exact",
                   integrator="rk2_central")
    c.init_from_factors(T, U, snaps[0])
    To, Uo, Vpp, Vp = T, U, None, V0
    worst = 0.0
    for k in range(1, 41):
        info = c.push(snaps[k])
        Vk = S.to_logical(snaps[k])
        To, Uo = O.step_rk2_central(To, Uo, w, Vpp, Vp, Vk)
        Vpp, Vp = Vp, Vk
        eo = O.error_exact(Vk, To, Uo, w)
        worst = max(worst, abs(info["eps"] - eo) / eo)
    Tg, Ug = c.factors()
    r = rel(O.reconstruct(Tg, Ug), O.reconstruct(To, Uo))
    assert worst <= eps_bound, worst
    assert r <= rec_bound, r


@cuda
def test_rk2_central_refused_by_input_slots(tdbmod):
    wl = S.make_workload("reactive", nx=64, ny=48, ns=6)
    snaps = [wl.snapshot(k, device="cuda") for k in range(2)]
    c = tdbmod.TDB(wl.dims, [5, 5, 4], weights=wl.weights, precision="bf16", error_mode="exact",
                   integrator="rk2_central").init(snaps[0])
    slots = [torch.empty_like(snaps[0]), snaps[0]]
    c.set_input_slots(slots[0], slots[1])
    slots[0].copy_(snaps[1])
    with pytest.raises(tdbmod.TDBError) as ei:
        c.push_slot(0)
    assert ei.value.status == 11          # TDB_ERR_UNSUPPORTED
