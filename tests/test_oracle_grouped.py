"""Grouped (multi-dimensional) modes: the TDB-2 / DBO scheme of Sec. 3.2 on CPU.

Grouping consecutive modes is a reshape of the storage tensor with product quadrature
weights; for two modes the truncated HOSVD is the truncated SVD of the weighted matrix
(Eckart-Young), so the TDB-2 error is the optimal one of its rank and no larger than the
TDB-1 error of a decomposition whose grouped unfolding has that rank.
"""

import math

import numpy as np
import torch

import oracle as O
from paper_2201_06958_gb300 import synth as S


def _pair(seed=1006, nx=24, ny=10, ns=7):
    t1 = S._reactive(seed, nx=nx, ny=ny, ns=ns)
    t2 = S.group_modes(t1, [[0, 1], [2]], rank_max=[ns, ns])
    return t1, t2


def test_grouping_is_a_reshape_with_product_weights():
    """Same data, same weighted norm (nx != ny, so a transposed weight product fails),
    and the grouped weight of (i_1, i_2) is w_1(i_1) w_2(i_2) at i_1 + N_1 i_2."""
    t1, t2 = _pair()
    assert t2.dims == [24 * 10, 7]
    a = t1.snapshot(3).reshape(-1)
    b = t2.snapshot(3).reshape(-1)
    assert torch.equal(a, b)
    V1, V2 = t1.logical(3), t2.logical(3)
    n1, n2 = O.weighted_norm2(V1, t1.weights), O.weighted_norm2(V2, t2.weights)
    assert abs(n1 - n2) <= 1e-14 * n1
    i1, i2 = 5, 7
    assert t2.weights[0][i1 + 24 * i2] == t1.weights[0][i1] * t1.weights[1][i2]
    # the product rule of two unit-sum trapezoid rules is a unit-sum rule on the grouped grid (C6)
    assert abs(t2.weights[0].sum() - 1.0) <= 1e-14 and np.array_equal(t2.weights[1], t1.weights[2])
    with np.testing.assert_raises(ValueError):
        S.group_modes(t1, [[0, 2], [1]])


def test_tdb2_hosvd_is_the_weighted_svd():
    """p = 2: the oracle's HOSVD error at ranks (r, r) equals the discarded singular values
    of W_1^(1/2) V W_2^(1/2) (a library SVD), and the TDB-1 HOSVD error at (r1, r2, r3) is
    never below the TDB-2 error at min(r1 r2, r3)."""
    t1, t2 = _pair()
    V1, V2 = t1.logical(0), t2.logical(0)
    s = np.linalg.svd(np.sqrt(t2.weights[0])[:, None] * V2 * np.sqrt(t2.weights[1])[None, :], compute_uv=False)
    for r in (1, 3, 5):
        T, U, _ = O.hosvd(V2, t2.weights, [r, r])
        e = O.error_exact(V2, T, U, t2.weights)
        ref = math.sqrt(float(np.sum(s[r:] ** 2)))
        assert abs(e - ref) <= 1e-9 * ref + 1e-15, (r, e, ref)
    for rr in ((2, 2, 3), (3, 2, 4), (4, 4, 5), (2, 3, 7)):
        T, U, _ = O.hosvd(V1, t1.weights, list(rr))
        e1 = O.error_exact(V1, T, U, t1.weights)
        r = min(rr[0] * rr[1], rr[2])
        T, U, _ = O.hosvd(V2, t2.weights, [r, r])
        e2 = O.error_exact(V2, T, U, t2.weights)
        assert e2 <= e1 * (1 + 1e-12), (rr, e1, e2)


def test_tdb2_storage_is_the_two_mode_compression_ratio():
    """The TDB-2 storage of Sec. 3.2, r N_1 N_2 + r n_s + r^2, is the general
    sum r_n N_n + prod r_n of Sec. 2.6 for the grouped dimensions."""
    for r, N1, N2, ns in ((4, 251, 76, 23), (12, 32, 16, 12), (1, 2, 3, 4)):
        cr = O.compression_ratio([N1 * N2, ns], [r, r])
        assert math.isclose(cr, N1 * N2 * ns / O.storage_tdb2(r, N1, N2, ns), rel_tol=1e-15)


def test_grouped_euler_step_keeps_exact_rank_data_exact():
    """A grouped mode is an ordinary mode to the method: on data whose grouped unfolding
    has rank r and fixed column space, the two-mode Euler step reproduces every
    snapshot (the fixed-subspace case of Sec. 2.2 in the grouped variables)."""
    rng = np.random.default_rng(5)
    t1, t2 = _pair()
    w = t2.weights
    N1, N2, r = t2.dims[0], t2.dims[1], 3
    Q1, _ = np.linalg.qr(rng.standard_normal((N1, r)))
    Q2, _ = np.linalg.qr(rng.standard_normal((N2, r)))
    U = [Q1 / np.sqrt(w[0])[:, None], Q2 / np.sqrt(w[1])[:, None]]
    V = [O.reconstruct(np.diag([3.0, 2.0, 1.0]) + 0.1 * k * rng.standard_normal((r, r)), U) for k in range(6)]
    T = O.multi_mode_product(V[0], [(w[n][:, None] * U[n]).T for n in range(2)])
    Uc = [u.copy() for u in U]
    for k in range(1, 6):
        T, Uc, _, _ = O.step_euler(T, Uc, w, V[k - 1], V[k])
        e = O.error_exact(V[k], T, Uc, w)
        assert e <= 1e-12 * math.sqrt(O.weighted_norm2(V[k], w)), (k, e)


def _grouped_analytic_rk4(n, steps, dt):
    wl = S.group_modes(S.make_workload("analytic", n=n, dt=dt, steps=steps), [[0, 1], [2]], rank_max=[4, 4])
    w = wl.weights
    T, U, _ = O.hosvd(wl.logical(0), w, [4, 4])
    vdot = lambda t: S.to_logical(wl.snapshot_dot(t))
    for k in range(1, steps + 1):
        T, U = O.step_rk4(T, U, w, (k - 1) * dt, dt, vdot)
    V = wl.logical(steps)
    return O.error_exact(V, T, U, w) / math.sqrt(O.weighted_norm2(V, w))


def test_grouped_analytic_field_is_exact_rank_and_recovered_at_order_4():
    """The analytic field sum_j a_j f_j(x_1) g_j(x_2) h_j(x_3) grouped as ((x_1, x_2), x_3) is
    sum_j a_j (f_j g_j) h_j: rank 4 in both modes (the fifth weighted Gram eigenvalue is
    rounding), so the two-mode equations keep e = 0 and RK4 with the exact derivative
    converges at order 4 in the grouped variables, as in three modes."""
    wl = S.group_modes(S.make_workload("analytic", n=16), [[0, 1], [2]])
    spec = O.hosvd_spectrum(wl.logical(3), wl.weights)
    for n in range(2):
        lam = spec[n][0] / spec[n][0][0]
        assert lam[3] > 1e-3 and lam[4] < 1e-13, lam[:6]
    e1 = _grouped_analytic_rk4(16, 50, 4e-3)
    e2 = _grouped_analytic_rk4(16, 100, 2e-3)
    assert 12.0 < e1 / e2 < 20.0, (e1, e2)
    assert e2 < 1e-9


def test_grouped_controller_moves_both_ranks_together():
    """Two modes: r_1 <= r_2 and r_2 <= r_1 (the product bound of Sec. 2.2), so every
    rank the controller sets on the grouped reactive stream has r_1 = r_2, through an
    increase and a revert."""
    wl = S.make_workload("reactive_dbo")
    snaps = [S.to_logical(wl.snapshot(k, dtype=torch.float64)) for k in range(41)]
    ctrl = O.ControllerConfig(5e-5, 99.99, 5, [12, 12])
    _, recs = O.compress_stream(snaps, wl.weights, [0, 0], ctrl)
    assert all(r.ranks[0] == r.ranks[1] for r in recs)
    assert {"increase", "revert"} <= {r.action for r in recs}


def test_long_mode_spectrum_by_thin_svd_equals_gram_eigendecomposition():
    """A mode longer than the product of the others (60 > 4 x 3) takes its HOSVD spectrum
    from the thin SVD of the weighted unfolding: the same leading eigenvalues and
    eigenvectors (as projectors) as the eigen-decomposition of its N_n x N_n Gram, and a
    zero tail beyond the 12 returned values."""
    rng = np.random.default_rng(61)
    dims = (60, 4, 3)
    w = [rng.uniform(0.5, 1.5, N) for N in dims]
    w = [x / x.sum() for x in w]
    V = rng.standard_normal(dims)
    lam, Q = O.hosvd_spectrum(V, w)[0]
    assert lam.shape == (12,) and Q.shape == (60, 12)
    B = np.sqrt(w[0])[:, None] * O.unfold(V * np.sqrt(w[1])[None, :, None] * np.sqrt(w[2])[None, None, :], 0)
    ev, EV = np.linalg.eigh(B @ B.T)
    order = np.argsort(ev)[::-1]
    ev, EV = ev[order], EV[:, order]
    assert np.allclose(lam, ev[:12], rtol=1e-12, atol=1e-14 * ev[0])
    assert np.abs(ev[12:]).max() <= 1e-12 * ev[0]
    for k in (3, 7, 12):
        assert np.abs(Q[:, :k] @ Q[:, :k].T - EV[:, :k] @ EV[:, :k].T).max() <= 1e-10
