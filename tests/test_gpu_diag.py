"""The library's own device arithmetic and failure handling, through the C-ABI.

* The double reciprocal and reciprocal square root of the small-matrix kernels
  (Newton-Raphson from a float seed) against 1/x and 1/sqrt(x) taken in extended
  precision on the host, over the whole exponent range: within 2 ulp.
* The bounded device waits: the fused update's grid barrier and the projection
  kernel's mbarrier wait, each made to wait for an arrival that never comes, return
  TDB_ERR_TIMEOUT after their limit; the CUDA context stays usable and a compressor
  runs normally afterwards.
"""

import numpy as np
import pytest
import torch

from paper_2201_06958_gb300 import synth as S

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


@pytest.fixture(scope="module")
def tdbmod():
    from paper_2201_06958_gb300 import build_lib, tdb
    build_lib.build()
    return tdb


def ulp_error(got: np.ndarray, ref_ld: np.ndarray) -> np.ndarray:
    ref = ref_ld.astype(np.float64)
    ulp = np.spacing(np.abs(ref))
    return np.abs((got.astype(np.longdouble) - ref_ld) / ulp.astype(np.longdouble)).astype(np.float64)


@cuda
def test_double_reciprocal_helpers_within_2_ulp(tdbmod):
    rng = np.random.default_rng(5)
    # mantissas in [1, 2) at every binary exponent of normal doubles (both signs for 1/x),
    # plus powers of two and values next to them
    e = np.arange(-1020, 1021)
    m = rng.uniform(1.0, 2.0, size=(e.size, 16))
    x = (m * np.ldexp(1.0, e)[:, None]).ravel()
    edges = np.ldexp(1.0, e)
    x = np.concatenate([x, edges, np.nextafter(edges, 0), np.nextafter(edges, np.inf), -x[::7]])
    xt = torch.from_numpy(x).cuda()
    rcp, rs = tdbmod.selftest_recip(xt)
    rcp, rs = rcp.cpu().numpy(), rs.cpu().numpy()
    xl = x.astype(np.longdouble)
    err_r = ulp_error(rcp, np.longdouble(1) / xl)
    pos = x > 0
    err_s = ulp_error(rs[pos], np.longdouble(1) / np.sqrt(xl[pos]))
    print(f"drcp max {err_r.max():.3f} ulp, drsqrt max {err_s.max():.3f} ulp over {x.size} values")
    assert np.all(np.isfinite(rcp)) and np.all(np.isfinite(rs[pos]))
    assert err_r.max() <= 2.0, err_r.max()
    assert err_s.max() <= 2.0, err_s.max()


@cuda
@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_runs_out_and_context_stays_usable(tdbmod, which):
    st = tdbmod.selftest_timeout(which, 2_000_000)       # ~1 ms of SM clock
    assert st == 7, st                                    # TDB_ERR_TIMEOUT
    torch.cuda.synchronize()
    # the context still works: a BF16 compressor steps normally afterwards
    wl = S.make_workload("reactive", nx=128, ny=64, ns=6)
    snaps = [wl.snapshot(k, device="cuda") for k in range(4)]
    c = tdbmod.TDB(wl.dims, [6, 6, 4], weights=wl.weights, precision="bf16", error_mode="exact").init(snaps[0])
    for k in range(1, 4):
        info = c.push(snaps[k])
        assert info["status"] == 0 and np.isfinite(info["eps"])
    c.close()
