"""TDB-2 at the size of Sec. 3.2 on the GPU: the reactive flow with its 251 x 76 grid taken
as one 19,076-point spatial mode beside the 23-species mode, against the oracle.

The long mode takes its HOSVD from the short side (the 23 x 23 Gram of the species index,
then B z / sqrt(lambda)); the update kernel sums its 597 row tiles' partials of P_n and of
the Cholesky-QR Gram with the whole grid; the BF16 projection adds its 150 tiles along
the mode in tile order.  FP64: 1e-10 relative on T x U and epsilon over fixed-rank Euler
steps, and the rank controller's actions, ranks and errors step by step over 150 steps.
FP32 and BF16: the bounds of the three-mode reactive tests.
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


@pytest.fixture(scope="module")
def wl():
    return S.make_workload("reactive_tdb2")


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@cuda
def test_tdb2_fp64_euler_matches_oracle(tdbmod, wl):
    """30 Euler steps at ranks (8, 8) from the oracle's HOSVD state: T x U within 1e-10 of
    the oracle's every 10 steps, epsilon every step, and U_1^T W U_1 = I to 1e-12."""
    w = wl.weights
    snaps = [wl.snapshot(k, device="cuda", dtype=torch.float64) for k in range(31)]
    V0 = S.to_logical(snaps[0])
    T, U, _ = O.hosvd(V0, w, [8, 8])
    c = tdbmod.TDB(wl.dims, [8, 8], weights=w, precision="fp64", error_mode="exact")
    c.init_from_factors(T, U, snaps[0])
    To, Uo, Vp = T, U, V0
    worst_eps, worst_rec = 0.0, 0.0
    for k in range(1, 31):
        info = c.push(snaps[k])
        Vk = S.to_logical(snaps[k])
        To, Uo, _, _ = O.step_euler(To, Uo, w, Vp, Vk)
        Vp = Vk
        eo = O.error_exact(Vk, To, Uo, w)
        worst_eps = max(worst_eps, abs(info["eps"] - eo) / eo)
        if k % 10 == 0:
            Tg, Ug = c.factors()
            worst_rec = max(worst_rec, rel(O.reconstruct(Tg, Ug), O.reconstruct(To, Uo)))
            assert np.abs(Ug[0].T @ (w[0][:, None] * Ug[0]) - np.eye(8)).max() <= 1e-12
    assert worst_rec <= 1e-10, worst_rec
    assert worst_eps <= 1e-10, worst_eps


@cuda
def test_tdb2_fp64_rank_control_matches_oracle(tdbmod, wl):
    """Sec. 2.5 on the paper-size grouped stream (FP64, 150 steps, HOSVD start from the
    short side): every step's action, ranks, re-initialisation and error equal the oracle
    controller's, whose long-mode spectrum is a thin SVD."""
    w = wl.weights
    snaps = [wl.snapshot(k, device="cuda", dtype=torch.float64) for k in range(151)]
    logical = [S.to_logical(x) for x in snaps]
    eps_th, gamma_th, K = 2e-5, 99.999, 5
    ctrl = O.ControllerConfig(eps_th, gamma_th, K, [23, 23])
    _, recs = O.compress_stream(logical, w, [0, 0], ctrl)
    c = tdbmod.TDB(wl.dims, [0, 0], rank_max=[23, 23], weights=w, eps_th=eps_th, gamma_th=gamma_th,
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
        seen.add(info["action"])
    assert {"increase", "reinit"} <= seen, seen


@cuda
def test_tdb2_fp32_hosvd_from_short_side(tdbmod, wl):
    """The float HOSVD (weighted data in float, the 23 x 23 Gram solved in double): the
    gamma_th = 99.999 % ranks equal the oracle's, and T x U is the oracle's truncated HOSVD
    to float accuracy."""
    w = wl.weights
    snap = wl.snapshot(0, device="cuda")
    V0 = S.to_logical(snap)
    spec = O.hosvd_spectrum(V0, w)
    ranks = O.clamp_product_bound([min(23, O.rank_from_spectrum(lam, 99.999)) for lam, _ in spec])
    c = tdbmod.TDB(wl.dims, [0, 0], rank_max=[23, 23], weights=w, eps_th=1e-4, gamma_th=99.999,
                   precision="fp32", error_mode="exact")
    c.init(snap)
    got = c.ranks()
    assert got == ranks, (got, ranks)
    T, U, _ = O.hosvd(V0, w, got, spectrum=spec)
    Tg, Ug = c.factors()
    assert rel(O.reconstruct(Tg, Ug), O.reconstruct(T, U)) <= 1e-5


@cuda
@pytest.mark.parametrize("precision,eps_tol,rec_tol", [("fp32", 1e-3, 1e-5), ("bf16", 0.02, 5e-4)])
def test_tdb2_reduced_precision_tracks_oracle(tdbmod, wl, precision, eps_tol, rec_tol):
    """40 Euler steps at ranks (8, 8) from the oracle's HOSVD state in FP32 and in BF16
    (150 tensor-core tiles along the spatial mode)."""
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
