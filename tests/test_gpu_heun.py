"""Heun's second-order scheme (TDB_HEUN) on the GPU against the oracle's step_heun.

Both stages use the snapshot difference; the first stage's predicted state is not
re-orthonormalised, the step's result is (Sec. 3.1 compares this scheme with Euler).
FP64: 1e-10 relative on T x U, sigma^(n) and epsilon, as for the Euler step (plus the
rounding floor of epsilon where it is tiny against ||V||_W).  FP32 and
BF16: the bounds of the corresponding Euler tests (the second stage repeats the same
arithmetic once more).
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
def test_heun_fp64_analytic_matches_oracle(tdbmod):
    """32^3 exact-rank-4 field, dt = 4e-3, 50 Heun steps in FP64 from the oracle's HOSVD
    state: T x U and sigma^(n) within 1e-10 of the oracle's Heun run, bases W-orthonormal,
    and the error far below the Euler run's at the same dt.  Epsilon is only ~6e-6 of
    ||V||_W here, so besides 1e-10 relative it is allowed the FP64 rounding of the
    difference V - T x U, whose entries are of the size of V: 1e-13 ||V||_W."""
    wl = S.make_workload("analytic", n=32, dt=4e-3, steps=50)
    w = wl.weights
    V0 = wl.logical(0)
    T, U, _ = O.hosvd(V0, w, [4, 4, 4])
    c = tdbmod.TDB(wl.dims, [4, 4, 4], weights=w, precision="fp64", error_mode="exact", integrator="heun")
    snaps = [wl.snapshot(k, device="cuda") for k in range(wl.steps + 1)]
    c.init_from_factors(T, U, snaps[0])
    To, Uo, Te, Ue, Vp = T, U, T, U, V0
    worst = {"rec": 0.0, "sig": 0.0, "eps": 0.0}
    for k in range(1, wl.steps + 1):
        info = c.push(snaps[k])
        Vk = S.to_logical(snaps[k])
        To, Uo = O.step_heun(To, Uo, w, Vp, Vk)
        Te, Ue, _, _ = O.step_euler(Te, Ue, w, Vp, Vk)
        Vp = Vk
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
    assert info["eps"] < O.error_exact(Vp, Te, Ue, w) / 20.0


@cuda
def test_heun_fp64_four_modes_matches_oracle(tdbmod):
    """Four modes with ragged sizes, a random walk of the data around a rank-(4,3,2,2)
    tensor, 12 Heun steps in FP64: T x U within 1e-10 of the oracle every step."""
    rng = np.random.default_rng(411)
    dims, ranks = (37, 24, 6, 5), (4, 3, 2, 2)
    w = []
    for N in dims:
        x = rng.uniform(0.5, 1.5, N)
        w.append(x / x.sum())
    U = []
    for N, r, wn in zip(dims, ranks, w):
        Q, _ = np.linalg.qr(rng.standard_normal((N, r)))
        U.append(Q / np.sqrt(wn)[:, None])
    T = rng.standard_normal(ranks)
    V = [O.reconstruct(T, U)]
    for _ in range(12):
        V.append(V[-1] + 2e-3 * rng.standard_normal(dims))
    c = tdbmod.TDB(dims, ranks, weights=w, precision="fp64", error_mode="exact", integrator="heun")
    g = [S.from_logical(v, device="cuda") for v in V]
    c.init_from_factors(T, U, g[0])
    To, Uo = T, U
    for k in range(1, len(V)):
        info = c.push(g[k])
        To, Uo = O.step_heun(To, Uo, w, V[k - 1], V[k])
        Tg, Ug = c.factors()
        assert rel(O.reconstruct(Tg, Ug), O.reconstruct(To, Uo)) <= 1e-10, k
        eo = O.error_exact(V[k], To, Uo, w)
        assert abs(info["eps"] - eo) <= 1e-10 * eo, k


@cuda
@pytest.mark.parametrize("precision,eps_tol,rec_tol", [("fp32", 1e-3, 1e-5), ("bf16", 0.02, 5e-4)])
def test_heun_reactive_tracks_oracle(tdbmod, precision, eps_tol, rec_tol):
    """40 Heun steps of the 512 x 256 x 12 reactive stream in the plain FP32 path and
    with the fused BF16 projection (two passes per snapshot), against the oracle's
    Heun run on the same float32 snapshots."""
    wl = S.make_workload("reactive")
    w = wl.weights
    snaps = [wl.snapshot(k, device="cuda") for k in range(41)]
    V0 = S.to_logical(snaps[0])
    T, U, _ = O.hosvd(V0, w, [11, 11, 7])
    c = tdbmod.TDB(wl.dims, [11, 11, 7], weights=w, precision=precision, error_mode="exact", integrator="heun")
    c.init_from_factors(T, U, snaps[0])
    To, Uo, Vp = T, U, V0
    worst = 0.0
    for k in range(1, 41):
        info = c.push(snaps[k])
        Vk = S.to_logical(snaps[k])
        To, Uo = O.step_heun(To, Uo, w, Vp, Vk)
        Vp = Vk
        eo = O.error_exact(Vk, To, Uo, w)
        worst = max(worst, abs(info["eps"] - eo) / eo)
    Tg, Ug = c.factors()
    r = rel(O.reconstruct(Tg, Ug), O.reconstruct(To, Uo))
    assert r <= rec_tol, (r, worst)
    assert worst <= eps_tol, (r, worst)


@cuda
def test_heun_slot_graph_equals_pointer_pushes(tdbmod):
    """Recorded Heun steps (two projections and two fused updates per replay) give the
    step records and factors of plain pushes bit for bit, across control actions."""
    wl = S.make_workload("reactive")
    steps = 40
    snaps = [wl.snapshot(k, device="cuda") for k in range(steps + 1)]
    kw = dict(rank_max=wl.rank_max, weights=wl.weights, eps_th=8e-5, gamma_th=99.9, slope_window=5,
              precision="bf16", error_mode="exact", integrator="heun")
    A = tdbmod.TDB(wl.dims, wl.rank, **kw).init(snaps[0])
    B = tdbmod.TDB(wl.dims, wl.rank, **kw)
    slots = [torch.empty_like(snaps[0]), torch.empty_like(snaps[0])]
    slots[1].copy_(snaps[0])
    B.init(slots[1]).set_input_slots(slots[0], slots[1])
    for k in range(1, steps + 1):
        parity = (k - 1) % 2
        slots[parity].copy_(snaps[k])
        ib = B.push_slot(parity)
        ia = A.push(snaps[k])
        for key in ("eps", "eps_step", "ranks", "reinit", "action", "dv_norm"):
            assert ia[key] == ib[key], (k, key, ia[key], ib[key])
    Ta, Ua = A.factors()
    Tb, Ub = B.factors()
    assert np.array_equal(Ta, Tb)
    assert all(np.array_equal(x, y) for x, y in zip(Ua, Ub))
