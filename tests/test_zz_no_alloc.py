"""The allocation-free projection entry point against the ordinary one.

Some callers cannot allocate device memory (a simulation that gives the whole GPU
to its own pool allocator, or code that may not call cudaMalloc once running).
tdb_project_noalloc computes the fused snapshot difference and projection with its
scratch in a static device array.  This file runs last (pytest collects files in
name order) so that a failure here comes after every other test has run."""

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


@cuda
def test_noalloc_matches_push_projection_two_calls():
    from paper_2201_06958_gb300 import build_lib, tdb
    build_lib.build()
    wl = S.make_workload("reactive")
    w = wl.weights
    dims, ranks = wl.dims, [11, 11, 7]
    snaps = [wl.snapshot(k, device="cuda") for k in range(3)]
    T, U, _ = O.hosvd(S.to_logical(snaps[0]), w, ranks)
    ctx = tdb.TDB(dims, ranks, weights=w, precision="bf16", error_mode="none")
    ctx.init_from_factors(T, U, snaps[0])
    w_dev = [torch.from_numpy(x).to("cuda", torch.float64) for x in w]
    for k in (1, 2):
        # weighted bases of the state the step starts from, as the library forms them
        _, Uk = ctx.factors()
        A = [_col_major((w[n][:, None] * Uk[n]).astype(np.float32), torch.float32) for n in range(3)]
        ctx.push(snaps[k])
        dS_ref, Y_ref = ctx.projection()
        dS = torch.empty(int(np.prod(ranks)), dtype=torch.float32, device="cuda")
        Y = []
        for n in range(3):
            sh = list(ranks)
            sh[n] = dims[n]
            Y.append(torch.empty(int(np.prod(sh)), dtype=torch.float32, device="cuda"))
        dv2 = torch.empty(1, dtype=torch.float64, device="cuda")
        st = tdb.project_noalloc(dims, ranks, snaps[k], snaps[k - 1], A, w_dev, dS, Y, dv2)
        assert st == 0, st
        torch.cuda.synchronize()
        got = dS.cpu().numpy().astype(np.float64).reshape(ranks, order="F")
        np.testing.assert_allclose(got, dS_ref, rtol=1e-6, atol=1e-6 * np.abs(dS_ref).max())
        for n in range(3):
            yr = Y_ref[n]
            yg = Y[n].cpu().numpy().astype(np.float64).reshape(yr.shape, order="F")
            np.testing.assert_allclose(yg, yr, rtol=1e-6, atol=1e-6 * np.abs(yr).max())
        ref_dv = np.sqrt(O.weighted_norm2(S.to_logical(snaps[k]) - S.to_logical(snaps[k - 1]), w))
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
