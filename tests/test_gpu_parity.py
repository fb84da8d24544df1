"""GPU path (libtdb through its C ABI) against the FP64 oracle, element by element.

FP64 mode: 1e-10 relative on the reconstruction T x U, the core singular values
and the error, per step; the projections dS, Y_n to 1e-12.  FP32 mode (unfused
CUDA-core kernels): bounds stated per test, derived from float rounding
(~6e-8 per operation, accumulated over the contraction lengths).
"""

import math

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


def rand_case(rng, dims, ranks, dtype=np.float64):
    w = []
    for N in dims:
        x = rng.uniform(0.5, 1.5, N)
        w.append(x / x.sum())
    U = []
    for N, r, wn in zip(dims, ranks, w):
        Q, _ = np.linalg.qr(rng.standard_normal((N, r)))
        U.append(Q / np.sqrt(wn)[:, None])
    T = rng.standard_normal(ranks)
    for n in range(len(dims)):
        T = O.mode_product(T, np.diag(np.linspace(1.0, 0.3, ranks[n])), n)
    return w, U, T


@cuda
@pytest.mark.parametrize("dims,ranks", [((37, 29, 23), (3, 4, 2)), ((64, 33, 5, 7), (4, 3, 2, 3)),
                                        ((131, 97), (5, 5)), ((128, 64, 16), (8, 8, 4))])
def test_projection_fp64_elementwise(tdbmod, dims, ranks):
    """a1 + a2: dS and every Y_n after one step, element by element (Eqs. 2.15, 2.16)."""
    rng = np.random.default_rng(100)
    w, U, T = rand_case(rng, dims, ranks)
    V0 = O.reconstruct(T, U) + 0.01 * rng.standard_normal(dims)
    V1 = V0 + 1e-3 * rng.standard_normal(dims)
    c = tdbmod.TDB(dims, ranks, weights=w, precision="fp64", error_mode="exact")
    g0 = S.from_logical(V0, device="cuda")
    g1 = S.from_logical(V1, device="cuda")
    c.init_from_factors(T, U, g0)
    c.push(g1)
    dS, Y = c.projection()
    dSo, Yo = O.project(V1 - V0, U, w)
    np.testing.assert_allclose(dS, dSo, rtol=1e-12, atol=1e-14 * np.abs(dSo).max())
    for n in range(len(dims)):
        sh = list(ranks)
        sh[n] = dims[n]
        Yt = O.fold(Yo[n], n, sh)
        np.testing.assert_allclose(Y[n], Yt, rtol=1e-11, atol=1e-13 * np.abs(Yt).max())


@cuda
def test_analytic_fp64_200_steps_matches_oracle(tdbmod):
    """The 64^3 exact-rank-4 field, 200 Euler steps in FP64 from the oracle's HOSVD
    state: T x U, sigma^(n) and epsilon match the oracle to 1e-10 relative every step."""
    wl = S.make_workload("analytic")
    w = wl.weights
    V0 = wl.logical(0)
    T, U, _ = O.hosvd(V0, w, [4, 4, 4])
    c = tdbmod.TDB(wl.dims, [4, 4, 4], weights=w, precision="fp64", error_mode="exact")
    snaps = [wl.snapshot(k, device="cuda") for k in range(wl.steps + 1)]
    c.init_from_factors(T, U, snaps[0])
    To, Uo, Vp = T, U, V0
    worst = {"rec": 0.0, "sig": 0.0, "eps": 0.0}
    for k in range(1, wl.steps + 1):
        info = c.push(snaps[k])
        Vk = S.to_logical(snaps[k])
        To, Uo, _, _ = O.step_euler(To, Uo, w, Vp, Vk)
        Vp = Vk
        eo = O.error_exact(Vk, To, Uo, w)
        worst["eps"] = max(worst["eps"], abs(info["eps"] - eo) / eo)
        if k % 20 == 0 or k == wl.steps:
            Tg, Ug = c.factors()
            worst["rec"] = max(worst["rec"], rel(O.reconstruct(Tg, Ug), O.reconstruct(To, Uo)))
            sg = O.core_singular_values(Tg)
            so = O.core_singular_values(To)
            worst["sig"] = max(worst["sig"], max(rel(a, b) for a, b in zip(sg, so)))
            for n in range(3):
                assert np.abs(Ug[n].T @ (w[n][:, None] * Ug[n]) - np.eye(4)).max() <= 1e-12
    assert worst["rec"] <= 1e-10, worst
    assert worst["sig"] <= 1e-10, worst
    assert worst["eps"] <= 1e-10, worst


@cuda
@pytest.mark.parametrize("dims,ranks", [((40, 30, 20), (5, 4, 3)), ((130, 24, 12), (6, 5, 4))])
def test_hosvd_init_fp64(tdbmod, dims, ranks):
    """GPU HOSVD (Jacobi, one CTA for N <= 96, cooperative multi-CTA above) against the
    oracle: the same projectors U U^T W, core singular values and reconstruction."""
    rng = np.random.default_rng(101)
    w, U, T = rand_case(rng, dims, [min(d, 8) for d in dims])
    V = O.reconstruct(T, U) + 1e-4 * rng.standard_normal(dims)
    c = tdbmod.TDB(dims, ranks, weights=w, precision="fp64", error_mode="exact")
    c.init(S.from_logical(V, device="cuda"))
    Tg, Ug = c.factors()
    To, Uo, spec = O.hosvd(V, w, ranks)
    for n in range(3):
        Pg = Ug[n] @ (Ug[n].T * w[n][None, :])
        Po = Uo[n] @ (Uo[n].T * w[n][None, :])
        assert np.abs(Pg - Po).max() <= 1e-9
    assert rel(O.reconstruct(Tg, Ug), O.reconstruct(To, Uo)) <= 1e-10
    for a, b in zip(O.core_singular_values(Tg), O.core_singular_values(To)):
        assert rel(a, b) <= 1e-10


@cuda
def test_reactive_fp32_tracks_oracle(tdbmod):
    """The 512 x 256 x 12 reactive stream in the plain FP32 path, 60 steps from the
    oracle's HOSVD state: reconstruction within 1e-5 relative and epsilon within 1e-3
    relative of the FP64 oracle run on the same float32 snapshots."""
    wl = S.make_workload("reactive")
    w = wl.weights
    snaps = [wl.snapshot(k, device="cuda") for k in range(61)]
    V0 = S.to_logical(snaps[0])
    T, U, _ = O.hosvd(V0, w, [11, 11, 7])
    c = tdbmod.TDB(wl.dims, [11, 11, 7], weights=w, precision="fp32", error_mode="exact")
    c.init_from_factors(T, U, snaps[0])
    To, Uo, Vp = T, U, V0
    worst_eps, worst_rec = 0.0, 0.0
    for k in range(1, 61):
        info = c.push(snaps[k])
        Vk = S.to_logical(snaps[k])
        To, Uo, _, _ = O.step_euler(To, Uo, w, Vp, Vk)
        Vp = Vk
        eo = O.error_exact(Vk, To, Uo, w)
        worst_eps = max(worst_eps, abs(info["eps"] - eo) / eo)
    Tg, Ug = c.factors()
    worst_rec = rel(O.reconstruct(Tg, Ug), O.reconstruct(To, Uo))
    assert worst_rec <= 1e-5, (worst_rec, worst_eps)
    assert worst_eps <= 1e-3, (worst_rec, worst_eps)


@cuda
def test_rank_control_decisions_match_oracle(tdbmod):
    """Sec. 2.5 on a small reactive stream with a tight threshold: the same actions,
    ranks and re-initialisation counts as the oracle controller, step by step (FP64)."""
    wl = S.make_workload("reactive", nx=48, ny=40, ns=6)
    w = wl.weights
    K = 5
    snaps = [wl.snapshot(k, device="cuda", dtype=torch.float64) for k in range(0, 121)]
    logical = [S.to_logical(x) for x in snaps]
    eps_th, gamma_th = 8e-5, 99.9       # exercises increase, reinit and revert within 120 steps
    ctrl = O.ControllerConfig(eps_th, gamma_th, K, [8, 8, 6])
    st, recs = O.compress_stream(logical, w, [0, 0, 0], ctrl)
    c = tdbmod.TDB(wl.dims, [0, 0, 0], rank_max=[8, 8, 6], weights=w, eps_th=eps_th, gamma_th=gamma_th,
                   slope_window=K, precision="fp64", error_mode="exact")
    c.init(snaps[0])
    acts = []
    for k in range(1, 121):
        info = c.push(snaps[k])
        rec = recs[k - 1]
        acts.append((info["action"], rec.action))
        assert info["ranks"] == rec.ranks, (k, info, rec)
        assert info["action"] == rec.action, (k, info["action"], rec.action)
        assert info["reinit"] == rec.reinit, k
        assert abs(info["eps"] - rec.eps) <= 1e-8 * rec.eps, (k, info["eps"], rec.eps)
    seen = {a for a, _ in acts}
    assert {"increase", "reinit", "revert"} <= seen, seen


@cuda
def test_runge_adaptive_ranks_match_oracle(tdbmod):
    """The Runge function of Sec. 3.1 (48^3, t in [0, 2]) through the FP64 path with rank
    adaptivity: every step's action and ranks equal the oracle controller's, ε within
    1e-8 relative, and the ranks rise before t = 1 and fall after."""
    wl = S.make_workload("runge", n=48)
    w = wl.weights
    snaps = [wl.snapshot(k, device="cuda") for k in range(0, wl.steps + 1)]
    logical = [S.to_logical(x) for x in snaps]
    ctrl = O.ControllerConfig(wl.eps_th, wl.gamma_th, 10, wl.rank_max)
    _, recs = O.compress_stream(logical, w, [0, 0, 0], ctrl)
    c = tdbmod.TDB(wl.dims, [0, 0, 0], rank_max=wl.rank_max, weights=w, eps_th=wl.eps_th, gamma_th=wl.gamma_th,
                   slope_window=10, precision="fp64", error_mode="exact")
    c.init(snaps[0])
    totals = []
    for k in range(1, wl.steps + 1):
        info = c.push(snaps[k])
        rec = recs[k - 1]
        assert info["action"] == rec.action, (k, info["action"], rec.action)
        assert info["ranks"] == rec.ranks, (k, info["ranks"], rec.ranks)
        assert abs(info["eps"] - rec.eps) <= 1e-8 * rec.eps, (k, info["eps"], rec.eps)
        totals.append(sum(info["ranks"]))
    assert max(totals) > totals[0] and totals[-1] < max(totals)


@cuda
def test_reinit_is_the_oracle_hosvd(tdbmod):
    """tdb_reinit re-initialises from a snapshot by the truncated HOSVD at the current
    ranks (Sec. 2.3 end): after two steps, the state equals the oracle's HOSVD of that
    snapshot to 1e-10 (FP64), with W-orthonormal bases, and a following push runs."""
    rng = np.random.default_rng(41)
    dims, ranks = (37, 29, 23), (3, 4, 2)
    w, U, T = rand_case(rng, dims, ranks)
    Vs = [O.reconstruct(T, U) + 1e-3 * k * rng.standard_normal(dims) for k in range(4)]
    dev = [S.from_logical(v, dtype=torch.float64, device="cuda") for v in Vs]
    c = tdbmod.TDB(dims, ranks, weights=w, precision="fp64", error_mode="exact").init(dev[0])
    c.push(dev[1])
    c.push(dev[2])
    c.reinit(dev[3])
    Tg, Ug = c.factors()
    To, Uo, _ = O.hosvd(Vs[3], w, list(ranks))
    assert rel(O.reconstruct(Tg, Ug), O.reconstruct(To, Uo)) <= 1e-10
    for n in range(3):
        assert np.abs(Ug[n].T @ (w[n][:, None] * Ug[n]) - np.eye(ranks[n])).max() <= 1e-12
    info = c.push(dev[2])
    assert info["ranks"] == list(ranks)


@cuda
def test_save_load_resume_is_bit_identical(tdbmod):
    wl = S.make_workload("reactive", nx=64, ny=48, ns=6)
    snaps = [wl.snapshot(k, device="cuda") for k in range(0, 13)]
    a = tdbmod.TDB(wl.dims, [5, 5, 4], weights=wl.weights, precision="fp32").init(snaps[0])
    for k in range(1, 7):
        a.push(snaps[k])
    blob = a.save_state()
    b = tdbmod.TDB(wl.dims, [5, 5, 4], weights=wl.weights, precision="fp32").init(snaps[0])
    b.load_state(blob, snaps[6])
    for k in range(7, 13):
        ia, ib = a.push(snaps[k]), b.push(snaps[k])
        assert ia["eps"] == ib["eps"]
    Ta, Ua = a.factors()
    Tb, Ub = b.factors()
    assert np.array_equal(Ta, Tb) and all(np.array_equal(x, y) for x, y in zip(Ua, Ub))


@cuda
def test_reconstruct_matches_oracle_and_error_statuses(tdbmod):
    rng = np.random.default_rng(102)
    dims, ranks = (50, 41, 9), (4, 3, 2)
    w, U, T = rand_case(rng, dims, ranks)
    V0 = O.reconstruct(T, U)
    c = tdbmod.TDB(dims, ranks, weights=w, precision="fp64")
    g0 = S.from_logical(V0, device="cuda")
    c.init_from_factors(T, U, g0)
    out = c.reconstruct()
    torch.cuda.synchronize()
    assert rel(S.to_logical(out), V0) <= 1e-13
    bad = g0.clone()
    bad.view(-1)[17] = float("nan")
    with pytest.raises(tdbmod.TDBError) as ei:
        c.push(bad)
    assert ei.value.status == 5          # TDB_ERR_NONFINITE
    # p = 2 needs r_1 = r_2 (each rank bounded by the other, Sec. 2.2)
    with pytest.raises(tdbmod.TDBError) as ei:
        tdbmod.TDB((20, 10), (3, 2), precision="fp64").init_from_factors(
            np.ones((3, 2)), [np.ones((20, 3)), np.ones((10, 2))], torch.zeros(10, 20, dtype=torch.float64, device="cuda"))
    assert ei.value.status == 3
    # rank above the product bound
    with pytest.raises(tdbmod.TDBError) as ei:
        tdbmod.TDB(dims, (4, 3, 2), weights=w, precision="fp64").init_from_factors(
            np.ones((7, 1, 1)), [np.ones((50, 7)), np.ones((41, 1)), np.ones((9, 1))], g0)
    assert ei.value.status == 3          # TDB_ERR_RANK
