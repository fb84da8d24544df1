"""The learned error estimator: GPU kernels against the FP64 reference
(oracle/mlp_oracle.py), and what the fitted estimator gains on a stream."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_06958_gb300 import synth as S

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")
M = O.mlp_oracle
F, H = 8, 64


@pytest.fixture(scope="module")
def tdbmod():
    from paper_2201_06958_gb300 import build_lib, tdb
    build_lib.build()
    return tdb


def _params(rng):
    return (M.init_params(F, H, rng) + 0.05 * rng.standard_normal(M.n_params(F, H))).astype(np.float32)


@cuda
@pytest.mark.parametrize("n", [1, 33, 1000])
def test_gradient_and_forward_match_reference(tdbmod, n):
    rng = np.random.default_rng(300 + n)
    th = _params(rng)
    X = rng.standard_normal((n, F)).astype(np.float32)
    t = rng.standard_normal(n).astype(np.float32)
    d = lambda a: torch.from_numpy(a).cuda()
    loss, grad = tdbmod.mlp_loss_grad(d(th), d(X), d(t))
    y = tdbmod.mlp_forward(d(th), d(X))
    torch.cuda.synchronize()
    L_ref, g_ref = M.loss_and_grad(th.astype(np.float64), X.astype(np.float64), t.astype(np.float64), F, H)
    y_ref = M.forward(th.astype(np.float64), X.astype(np.float64), F, H)
    assert abs(loss.item() - L_ref) <= 1e-4 * max(L_ref, 1e-6)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    np.testing.assert_allclose(y.cpu().numpy(), y_ref, rtol=1e-4, atol=1e-5)


@cuda
def test_adam_step_matches_reference(tdbmod):
    rng = np.random.default_rng(310)
    npar = M.n_params(F, H)
    th = rng.standard_normal(npar).astype(np.float32)
    g = rng.standard_normal(npar).astype(np.float32)
    m = (0.1 * rng.standard_normal(npar)).astype(np.float32)
    v = np.abs(0.1 * rng.standard_normal(npar)).astype(np.float32)
    dth, dg, dm, dv = (torch.from_numpy(a.copy()).cuda() for a in (th, g, m, v))
    tdbmod.mlp_adam_step(dth, dg, dm, dv, 7, 1e-3)
    torch.cuda.synchronize()
    th_r, m_r, v_r = M.adam_update(th.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                                   v.astype(np.float64), 7, 1e-3)
    np.testing.assert_allclose(dth.cpu().numpy(), th_r, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(dm.cpu().numpy(), m_r, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(dv.cpu().numpy(), v_r, rtol=1e-5, atol=1e-9)


@cuda
def test_estimator_gain_on_reactive_stream(tdbmod):
    """Reactive stream, BF16 projection.  Context A records exact errors for 150 steps,
    fits the estimator on the GPU and then gates the exact error; context B evaluates it
    every step.  A takes the same Sec. 2.5 decisions at the same steps, evaluates the
    error exactly on a small fraction of the gated steps, and never skips a step whose
    exact error (from B) exceeds eps_th.  The gate (0.9 eps_th) leaves room for the
    estimator's error: on this stream the exact error stays between half the threshold
    (after each HOSVD) and the threshold.  Estimates are chained through skipped steps,
    so a per-step bias of a few 1e-3 in log10 compounds; re-anchoring on an exact
    evaluation at least every 20 steps (error_every) bounds that drift to under 10 %."""
    wl = S.make_workload("reactive")
    w = wl.weights
    steps = 450
    snaps = [wl.snapshot(k, device="cuda") for k in range(steps + 1)]
    kw = dict(rank_max=wl.rank_max, weights=w, eps_th=wl.eps_th, gamma_th=wl.gamma_th, precision="bf16",
              error_every=20)
    A = tdbmod.TDB(wl.dims, wl.rank, error_mode="mlp", **kw).init(snaps[0])
    B = tdbmod.TDB(wl.dims, wl.rank, error_mode="exact", **kw).init(snaps[0])
    skipped_true = []
    acts_a, acts_b = [], []
    reasons = {1: 0, 2: 0, 4: 0}
    for k in range(1, steps + 1):
        ia = A.push(snaps[k])
        ib = B.push(snaps[k])
        acts_a.append((ia["action"], tuple(ia["ranks"])))
        acts_b.append((ib["action"], tuple(ib["ranks"])))
        if k == 150:
            loss = A.estimator_fit(iters=2000, lr=3e-3, seed=7, gate=0.9)
            assert loss < 0.1, loss
        if k > 150 and not ia["eps_exact"]:
            skipped_true.append((ib["eps_step"], ia["eps"]))
        if k > 150:
            for bit in reasons:
                reasons[bit] += bool(ia["gate"] & bit)
    assert acts_a == acts_b
    gated = steps - 150
    exact_after = A.counters()["exact_evals"] - 150
    assert exact_after <= 0.5 * gated, (exact_after, reasons)
    true_at_skips = np.array([a for a, _ in skipped_true])
    est_at_skips = np.array([b for _, b in skipped_true])
    assert np.all(true_at_skips <= wl.eps_th)
    ratio = est_at_skips / true_at_skips
    assert np.all((ratio > 0.8) & (ratio < 1.25)), (ratio.min(), ratio.max())
    assert any(a != "none" for a, _ in acts_b[150:]), "the gated phase should include a control action"


@cuda
def test_estimator_gain_in_device_time_stochastic(tdbmod):
    """What the learned estimator buys, in device time (CUDA events per phase), on the
    stochastic stream (256 x 128 x 512, BF16 projection), where the exact error is a full
    pass over a 67 MB snapshot.  A records exact errors for 150 steps and fits the
    estimator; then A gates the exact error while B evaluates it every step, for 100 more
    steps.  A takes B's decisions at every step, evaluates the error exactly on at most a
    third of the gated steps, and spends less device time than B on the error phase and on
    the whole step."""
    wl = S.make_workload("stochastic")
    w = wl.weights
    steps, fit_at = 250, 150
    snaps = [wl.snapshot(k, device="cuda") for k in range(steps + 1)]
    kw = dict(rank_max=wl.rank_max, weights=w, eps_th=wl.eps_th, gamma_th=wl.gamma_th, precision="bf16",
              error_every=20)
    A = tdbmod.TDB(wl.dims, wl.rank, error_mode="mlp", **kw).init(snaps[0])
    B = tdbmod.TDB(wl.dims, wl.rank, error_mode="exact", **kw).init(snaps[0])
    for k in range(1, steps + 1):
        ia = A.push(snaps[k])
        ib = B.push(snaps[k])
        assert (ia["action"], ia["ranks"]) == (ib["action"], ib["ranks"]), k
        if k == fit_at:
            loss = A.estimator_fit(iters=2000, lr=3e-3, seed=7, gate=0.9)
            assert loss < 0.1, loss
            A.set_profiling(True)
            B.set_profiling(True)
    gated = steps - fit_at
    exact_after = A.counters()["exact_evals"] - fit_at
    assert exact_after <= gated / 3, exact_after
    pa, pb = A.profile(), B.profile()
    assert pa["steps"] == pb["steps"] == gated, (pa["steps"], pb["steps"])
    tot = lambda pr: pr["ms_project"] + pr["ms_update"] + pr["ms_error"]
    assert pa["ms_error"] < pb["ms_error"], (pa, pb)
    assert tot(pa) < tot(pb), (pa, pb)


@cuda
def test_trace_keeps_the_last_rows_in_order(tdbmod):
    """The recorded (features, target) rows form a window of the last 8192, oldest first,
    through loads, appends and a reset; dropping old rows keeps the order of the rest."""
    wl = S.make_workload("reactive", nx=64, ny=32, ns=4)
    c = tdbmod.TDB(wl.dims, [4, 4, 2], weights=wl.weights, precision="fp32", error_mode="exact")
    c.init(wl.snapshot(0, device="cuda"))
    F, cap = 8, 8192

    def rows(lo, hi):
        k = np.arange(lo, hi, dtype=np.float32)
        return np.repeat(k[:, None], F, axis=1) + np.arange(F, dtype=np.float32) / 16, k * 0.5

    X, t = rows(0, 20000)
    c.estimator_load_trace(X, t)
    gx, gt = c.estimator_trace()
    assert gx.shape == (cap, F) and np.array_equal(gt, t[-cap:]) and np.array_equal(gx, X[-cap:])
    for lo in range(20000, 20000 + 3 * cap, 977):           # appends past several compactions
        X2, t2 = rows(lo, lo + 977)
        c.estimator_load_trace(X2, t2, append=True)
        X, t = np.concatenate([X, X2]), np.concatenate([t, t2])
        gx, gt = c.estimator_trace()
        assert np.array_equal(gt, t[-cap:]) and np.array_equal(gx, X[-cap:])
    X3, t3 = rows(5, 105)
    c.estimator_load_trace(X3, t3)                          # a reset
    gx, gt = c.estimator_trace()
    assert np.array_equal(gt, t3) and np.array_equal(gx, X3)
    c.close()
