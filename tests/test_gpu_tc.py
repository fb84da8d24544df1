"""The fused BF16 tensor-core projection (tcgen05 + TMA) against the FP64 oracle.

Bound used for every entry of dS and Y_n: the two BF16 roundings of a product
term (|delta| <= 2^-9 each) give |error| <= 2^-8 * sum |A||dV| over the BF16
contraction; the FP32 accumulation and the FP32 contractions of the remaining
modes add far less.  The tests allow 2^-7 * (|dV| contracted with |A_m| in every
mode) elementwise, computed by the oracle's mode products on absolute values.
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


def case(rng, dims, ranks):
    w = []
    for N in dims:
        x = rng.uniform(0.5, 1.5, N)
        w.append(x / x.sum())
    U = []
    for N, r, wn in zip(dims, ranks, w):
        Q, _ = np.linalg.qr(rng.standard_normal((N, r)))
        U.append(Q / np.sqrt(wn)[:, None])
    T = rng.standard_normal(ranks)
    return w, U, T


def abs_bound(dV, U, w, keep):
    A = [np.abs(w[n][:, None] * U[n]) for n in range(len(U))]
    X = np.abs(dV)
    for m in range(dV.ndim):
        if m != keep:
            X = O.mode_product(X, A[m].T, m)
    return X


@cuda
@pytest.mark.parametrize("dims,ranks", [
    ((512, 256, 12), (16, 16, 12)),      # the reactive-flow shape: 4 x 2 tiles per slice
    ((200, 136, 7), (12, 10, 5)),        # ragged tiles in modes 1 and 2
    ((192, 129, 12, 3), (30, 30, 8, 3)), # four modes, ragged mode 2, padded rank 32
    ((256, 100), (20, 20)),              # two modes (DBO)
    ((64, 64, 64), (4, 4, 4)),           # one tile per slice
    # more tile-slices than SMs: the persistent path (several tiles per CTA, the whole
    # operand images resident, the TMEM double buffer and the stages reused across tiles)
    ((256, 128, 512), (20, 20, 20)),     # the stochastic shape at rank 20: 1024 tiles, 8 stages
    ((256, 128, 320), (16, 16, 12)),     # 640 tiles, 16 stages
    ((192, 129, 192, 3), (30, 30, 30, 3)),  # the channel shape at its rank caps: 2304 tiles
    ((101, 67, 9), (7, 6, 4)),           # N_1 not a multiple of 4: zero-padded copies of both snapshots
])
def test_bf16_projection_within_rounding_bound(tdbmod, dims, ranks):
    rng = np.random.default_rng(200)
    w, U, T = case(rng, dims, ranks)
    V0 = rng.standard_normal(dims).astype(np.float32).astype(np.float64)
    V1 = (V0 + 1e-2 * rng.standard_normal(dims)).astype(np.float32).astype(np.float64)
    c = tdbmod.TDB(dims, ranks, weights=w, precision="bf16", error_mode="none")
    g0 = S.from_logical(V0, dtype=torch.float32, device="cuda")
    g1 = S.from_logical(V1, dtype=torch.float32, device="cuda")
    c.init_from_factors(T, U, g0)
    c.push(g1)
    dS, Y = c.projection()
    dV = V1 - V0
    dSo, Yo = O.project(dV, U, w)
    # dS: every mode contracted
    B = abs_bound(dV, U, w, keep=-1)
    assert np.all(np.abs(dS - dSo) <= 2.0 ** -7 * B + 1e-30), np.max(np.abs(dS - dSo) / B)
    for n in range(len(dims)):
        sh = list(ranks)
        sh[n] = dims[n]
        Yt = O.fold(Yo[n], n, sh)
        Bn = abs_bound(dV, U, w, keep=n)
        ratio = np.max(np.abs(Y[n] - Yt) / (Bn + 1e-300))
        assert ratio <= 2.0 ** -7, (n, ratio)
        # and the relative Frobenius error is at BF16 level
        assert np.linalg.norm(Y[n] - Yt) <= 4e-3 * np.linalg.norm(Yt), n


@cuda
def test_bf16_stream_tracks_oracle_reactive(tdbmod):
    """60 steps of the reactive stream with the fused BF16 projection: the error
    trace stays within 2 % of the FP64 oracle's and the reconstruction within
    5e-4 relative (BF16 operands, FP32 accumulation, FP64 small algebra)."""
    wl = S.make_workload("reactive")
    w = wl.weights
    snaps = [wl.snapshot(k, device="cuda") for k in range(61)]
    V0 = S.to_logical(snaps[0])
    T, U, _ = O.hosvd(V0, w, [11, 11, 7])
    c = tdbmod.TDB(wl.dims, [11, 11, 7], weights=w, precision="bf16", error_mode="exact")
    c.init_from_factors(T, U, snaps[0])
    To, Uo, Vp = T, U, V0
    worst = 0.0
    for k in range(1, 61):
        info = c.push(snaps[k])
        Vk = S.to_logical(snaps[k])
        To, Uo, _, _ = O.step_euler(To, Uo, w, Vp, Vk)
        Vp = Vk
        eo = O.error_exact(Vk, To, Uo, w)
        worst = max(worst, abs(info["eps"] - eo) / eo)
    Tg, Ug = c.factors()
    Rg, Ro = O.reconstruct(Tg, Ug), O.reconstruct(To, Uo)
    rel = np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro)
    assert worst <= 0.02, worst
    assert rel <= 5e-4, rel


@cuda
def test_bf16_dv_norm_matches(tdbmod):
    """||dV||_W accumulated inside the fused kernel (FP32 products, FP64 per-CTA sums)."""
    rng = np.random.default_rng(201)
    dims, ranks = (136, 200, 9), (6, 5, 4)
    w, U, T = case(rng, dims, ranks)
    V0 = rng.standard_normal(dims).astype(np.float32).astype(np.float64)
    V1 = (V0 + rng.standard_normal(dims)).astype(np.float32).astype(np.float64)
    c = tdbmod.TDB(dims, ranks, weights=w, precision="bf16", error_mode="none")
    c.init_from_factors(T, U, S.from_logical(V0, dtype=torch.float32, device="cuda"))
    info = c.push(S.from_logical(V1, dtype=torch.float32, device="cuda"))
    ref = np.sqrt(O.weighted_norm2(V1 - V0, w))
    assert abs(info["dv_norm"] - ref) <= 1e-5 * ref


@cuda
def test_launch_shape_tuner(tdbmod):
    """The projection's tuner times its candidate grids on the first step and keeps the
    fastest; a second context of the same shape takes the choice from the process-wide
    cache without timing; both produce the same projection (the shape changes only the
    work split, not the arithmetic of an element beyond the order of the slice sums)."""
    rng = np.random.default_rng(202)
    dims, ranks = (128, 96, 300), (8, 6, 5)
    w, U, T = case(rng, dims, ranks)
    V0 = rng.standard_normal(dims).astype(np.float32).astype(np.float64)
    V1 = (V0 + 1e-2 * rng.standard_normal(dims)).astype(np.float32).astype(np.float64)
    g0 = S.from_logical(V0, dtype=torch.float32, device="cuda")
    g1 = S.from_logical(V1, dtype=torch.float32, device="cuda")
    out = []
    for i in range(2):
        c = tdbmod.TDB(dims, ranks, weights=w, precision="bf16", error_mode="none")
        c.init_from_factors(T, U, g0)
        c.push(g1)
        t = c.tuning()
        out.append((t, c.projection()))
        c.close()
    t0, t1 = out[0][0], out[1][0]
    assert t0["timed"] and len(t0["candidates"]) >= 2
    assert t0["ctas_per_position"] in t0["candidates"]
    assert t0["ctas_per_position"] == min(t0["candidates"], key=t0["candidates"].get)
    assert t0["finish_split_target"] in t0["finish_candidates"]
    assert not t1["timed"] and t1["ctas_per_position"] == t0["ctas_per_position"]
    dSo, Yo = O.project(V1 - V0, U, w)
    B = abs_bound(V1 - V0, U, w, keep=-1)
    for _, (dS, Y) in out:
        assert np.all(np.abs(dS - dSo) <= 2.0 ** -7 * B + 1e-30)
