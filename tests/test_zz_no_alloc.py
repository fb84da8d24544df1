"""The allocation-free projection entry point against the ordinary one and the oracle.

Some callers cannot allocate device memory (a simulation that gives the whole GPU
to its own pool allocator, or code that may not call cudaMalloc once running).
tdb_project_noalloc computes the fused snapshot difference and projection with its
scratch in a static device array.  Each case makes two calls in a row, checks them
against a context's own projection of the same step (1e-6) and, element by element,
against the FP64 oracle's projection within the BF16 rounding bound (2^-7 times the
difference contracted with |W U| in every mode; see test_gpu_tc.py).  The cases
cover both ways the projection finishes: few slices (three modes, N_3 <= 64) and the
slab reduction with mode products (three modes with many slices, four modes), with
more tiles than the GPU has SMs.  This file runs last (pytest collects files in name
order) so that a failure here comes after every other test has run."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_06958_gb300 import synth as S

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def _col_major(a: np.ndarray, dtype) -> torch.Tensor:
    """(N, r) numpy -> device tensor holding the column-major (N x r) layout."""
    return torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda", dtype)


def _abs_bound(dV, U, w, keep):
    A = [np.abs(w[n][:, None] * U[n]) for n in range(len(U))]
    X = np.abs(dV)
    for m in range(dV.ndim):
        if m != keep:
            X = O.mode_product(X, A[m].T, m)
    return X


@cuda
@pytest.mark.parametrize("name,kw,ranks", [
    ("reactive", {}, [11, 11, 7]),                                  # 96 tiles, few slices
    ("stochastic", {"ns": 160}, [12, 12, 8]),                       # 320 tiles, slab branch
    ("channel", {"nx": 128, "nz": 32}, [10, 10, 8, 3]),             # 192 tiles, four modes
])
def test_noalloc_matches_push_projection_two_calls(name, kw, ranks):
    from paper_2201_06958_gb300 import build_lib, tdb
    build_lib.build()
    wl = S.make_workload(name, **kw)
    w = wl.weights
    dims = wl.dims
    p = len(dims)
    snaps = [wl.snapshot(k, device="cuda") for k in range(3)]
    T, U, _ = O.hosvd(S.to_logical(snaps[0]), w, ranks)
    ctx = tdb.TDB(dims, ranks, weights=w, precision="bf16", error_mode="none")
    ctx.init_from_factors(T, U, snaps[0])
    w_dev = [torch.from_numpy(x).to("cuda", torch.float64) for x in w]
    for k in (1, 2):
        # weighted bases of the state the step starts from, as the library forms them
        _, Uk = ctx.factors()
        A = [_col_major((w[n][:, None] * Uk[n]).astype(np.float32), torch.float32) for n in range(p)]
        ctx.push(snaps[k])
        dS_ref, Y_ref = ctx.projection()
        dS = torch.empty(int(np.prod(ranks)), dtype=torch.float32, device="cuda")
        Y = []
        for n in range(p):
            sh = list(ranks)
            sh[n] = dims[n]
            Y.append(torch.empty(int(np.prod(sh)), dtype=torch.float32, device="cuda"))
        dv2 = torch.empty(1, dtype=torch.float64, device="cuda")
        st = tdb.project_noalloc(dims, ranks, snaps[k], snaps[k - 1], A, w_dev, dS, Y, dv2)
        assert st == 0, st
        torch.cuda.synchronize()
        got = dS.cpu().numpy().astype(np.float64).reshape(ranks, order="F")
        np.testing.assert_allclose(got, dS_ref, rtol=1e-6, atol=1e-6 * np.abs(dS_ref).max())
        Yg = []
        for n in range(p):
            yr = Y_ref[n]
            yg = Y[n].cpu().numpy().astype(np.float64).reshape(yr.shape, order="F")
            np.testing.assert_allclose(yg, yr, rtol=1e-6, atol=1e-6 * np.abs(yr).max())
            Yg.append(yg)
        # independent of the library's own path: the FP64 oracle on the same snapshots
        # and the bases the call was given (their float values)
        dV = S.to_logical(snaps[k]) - S.to_logical(snaps[k - 1])
        Uf = [(A[n].T.cpu().numpy().astype(np.float64)) / w[n][:, None] for n in range(p)]
        dSo, Yo = O.project(dV, Uf, w)
        B = _abs_bound(dV, Uf, w, keep=-1)
        assert np.all(np.abs(got - dSo) <= 2.0 ** -7 * B + 1e-30), np.max(np.abs(got - dSo) / B)
        for n in range(p):
            sh = list(ranks)
            sh[n] = dims[n]
            Yt = O.fold(Yo[n], n, sh)
            ratio = np.max(np.abs(Yg[n] - Yt) / (_abs_bound(dV, Uf, w, keep=n) + 1e-300))
            assert ratio <= 2.0 ** -7, (n, ratio)
        ref_dv = np.sqrt(O.weighted_norm2(dV, w))
        assert abs(np.sqrt(dv2.item()) - ref_dv) <= 1e-5 * ref_dv


@cuda
def test_noalloc_refuses_sizes_beyond_its_scratch():
    from paper_2201_06958_gb300 import build_lib, tdb
    build_lib.build()
    dims, ranks = [512, 256, 256], [16, 16, 8]        # the mode-1 partial sums alone exceed 16 MiB
    z = torch.zeros(1, dtype=torch.float32, device="cuda")
    zd = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = tdb.project_noalloc(dims, ranks, z, z, [z, z, z], [zd, zd, zd], z, [z, z, z], zd)
    assert st == 10      # TDB_ERR_WORKSPACE, refused before any launch
