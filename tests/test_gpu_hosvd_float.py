"""Truncated HOSVD of the float compute types (weighted data, 64 x 64 Gram tiles
with float-float accumulation, cooperative subspace iteration with Rayleigh-Ritz)
against the FP64 oracle on the same float32 snapshot.

Bounds: the Gram is accumulated from float products in float chunks of 32 columns,
so its entries carry ~1e-7 relative rounding; eigen-projectors move by that over
the eigen-gap (the cases below keep gaps of O(10 %) of the top eigenvalue), hence
1e-4 on the projectors, 1e-5 on the reconstruction and 1e-4 on the core singular
values, and the eigenvalues within 1e-6 of the largest.
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


def case(rng, dims, inner):
    w = []
    for N in dims:
        x = rng.uniform(0.5, 1.5, N)
        w.append(x / x.sum())
    U = []
    for N, r, wn in zip(dims, inner, w):
        Q, _ = np.linalg.qr(rng.standard_normal((N, r)))
        U.append(Q / np.sqrt(wn)[:, None])
    T = rng.standard_normal(inner)
    for n in range(len(dims)):
        T = O.mode_product(T, np.diag(np.linspace(1.0, 0.3, inner[n])), n)
    return w, U, T


@cuda
@pytest.mark.parametrize("dims,ranks", [
    ((200, 130, 12), (6, 5, 4)),     # modes 1 and 2 through the subspace iteration, ragged row blocks
    ((512, 64, 12), (12, 10, 6)),    # the reactive mode-1 size; mode 2 (N = 64) also through the subspace iteration
    ((40, 36, 12), (5, 5, 4)),       # every mode through the single-CTA Jacobi (N <= 48)
])
def test_float_hosvd_init_matches_oracle(tdbmod, dims, ranks):
    rng = np.random.default_rng(301)
    inner = [min(d, r + 4) for d, r in zip(dims, ranks)]
    w, U, T = case(rng, dims, inner)
    V = O.reconstruct(T, U) + 1e-4 * rng.standard_normal(dims)
    V = V.astype(np.float32).astype(np.float64)
    c = tdbmod.TDB(dims, ranks, weights=w, precision="fp32", error_mode="exact")
    c.init(S.from_logical(V, dtype=torch.float32, device="cuda"))
    Tg, Ug = c.factors()
    To, Uo, spec = O.hosvd(V, w, ranks)
    for n in range(3):
        Pg = Ug[n] @ (Ug[n].T * w[n][None, :])
        Po = Uo[n] @ (Uo[n].T * w[n][None, :])
        assert np.abs(Pg - Po).max() <= 1e-4, (n, np.abs(Pg - Po).max())
        # the bases are W-orthonormal to double rounding after the Cholesky-QR
        assert np.abs(Ug[n].T @ (w[n][:, None] * Ug[n]) - np.eye(ranks[n])).max() <= 1e-12
    assert rel(O.reconstruct(Tg, Ug), O.reconstruct(To, Uo)) <= 1e-5
    for a, b in zip(O.core_singular_values(Tg), O.core_singular_values(To)):
        assert rel(a, b) <= 1e-4


@cuda
def test_float_reinit_matches_oracle(tdbmod):
    """A re-initialisation (Sec. 2.5) in the float path, in the middle of a stream.
    The state it leaves is the truncated HOSVD of that snapshot at the new ranks:
    projectors within
    max(1e-4, 20 u lambda_1 / gap) of the oracle's (u = 2^-24; the float Gram moves
    the r-dimensional eigenspace by its rounding over the gap lambda_r - lambda_{r+1}),
    the reconstruction within max(1e-5, sum_n b_n sqrt(2 lambda_r / sum lambda)): a
    rotation of the kept subspace by an angle b_n near the cut moves the energy of the
    directions r and r + 1, about 2 lambda_r of the total."""
    wl = S.make_workload("reactive")
    w = wl.weights
    c = tdbmod.TDB(wl.dims, wl.rank, rank_max=wl.rank_max, weights=w, eps_th=8e-5, gamma_th=99.9,
                   slope_window=5, precision="fp32", error_mode="exact")
    c.init(wl.snapshot(0, device="cuda"))
    snap, info = None, None
    for k in range(1, 81):
        snap = wl.snapshot(k, device="cuda")
        info = c.push(snap)
        if info["reinit"] > 0 and info["action"] in ("reinit", "increase"):
            break
    else:
        pytest.fail("no re-initialisation within 80 steps")
    V = S.to_logical(snap)
    ranks = info["ranks"]
    spec = O.hosvd_spectrum(V, w)
    To, Uo, _ = O.hosvd(V, w, ranks, spectrum=spec)
    Tg, Ug = c.factors()
    rec_bound = 0.0
    for n in range(3):
        lam = spec[n][0]
        r = ranks[n]
        gap = lam[r - 1] - (lam[r] if r < len(lam) else 0.0)
        bound = max(1e-4, 20 * 2.0 ** -24 * lam[0] / max(gap, 1e-300))
        rec_bound += bound * np.sqrt(2 * lam[r - 1] / lam.sum())
        Pg = Ug[n] @ (Ug[n].T * w[n][None, :])
        Po = Uo[n] @ (Uo[n].T * w[n][None, :])
        assert np.abs(Pg - Po).max() <= bound, (n, r, np.abs(Pg - Po).max(), bound)
    d = rel(O.reconstruct(Tg, Ug), O.reconstruct(To, Uo))
    assert d <= max(1e-5, rec_bound), (d, rec_bound)
