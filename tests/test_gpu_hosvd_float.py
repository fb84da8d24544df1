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
    ((512, 64, 12), (12, 10, 6)),    # the reactive mode-1 size; mode 2 through the single-CTA Jacobi
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
