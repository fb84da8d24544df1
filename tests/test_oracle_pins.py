"""Pins of the FP64 oracle against things other than itself: brute force on tiny
inputs, closed forms, exact special cases, convergence orders, invariants and
library routines used only here.  No GPU needed."""

import itertools
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_06958_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_orth_w(rng, N, r, w):
    """Random U with U^T W U = I (built from a plain QR of W^{1/2}-scaled noise)."""
    Q, _ = np.linalg.qr(rng.standard_normal((N, r)))
    return Q / np.sqrt(w)[:, None]


def _rand_weights(rng, N):
    w = rng.uniform(0.5, 1.5, N)
    return w / w.sum()


# ---------------------------------------------------------------------------
# Projection (Eqs. 2.15, 2.16): brute force with literal loops
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,ranks", [((5, 4, 3), (2, 2, 2)), ((6, 5, 4, 3), (2, 3, 2, 2)), ((7, 5), (3, 2))])
def test_projection_bruteforce(dims, ranks):
    rng = np.random.default_rng(1)
    p = len(dims)
    w = [_rand_weights(rng, N) for N in dims]
    U = [_rand_orth_w(rng, N, r, wn) for N, r, wn in zip(dims, ranks, w)]
    dV = rng.standard_normal(dims)
    dS, Y = O.project(dV, U, w)

    # dS[a...] = sum_i prod_n w_n(i_n) U_n(i_n, a_n) dV[i]   (literal loops)
    ref = np.zeros(ranks)
    for a in itertools.product(*[range(r) for r in ranks]):
        s = 0.0
        for i in itertools.product(*[range(N) for N in dims]):
            f = dV[i]
            for n in range(p):
                f *= w[n][i[n]] * U[n][i[n], a[n]]
            s += f
        ref[a] = s
    np.testing.assert_allclose(dS, ref, rtol=1e-12, atol=1e-14)

    # Y_n[i_n, col(a_{-n})] with the paper's column index: first remaining mode fastest (Sec. 2.2)
    for n in range(p):
        others = [m for m in range(p) if m != n]
        Yref = np.zeros((dims[n], int(np.prod([ranks[m] for m in others]))))
        for i_n in range(dims[n]):
            for a in itertools.product(*[range(ranks[m]) for m in others]):
                col, stride = 0, 1
                for m, am in zip(others, a):
                    col += am * stride
                    stride *= ranks[m]
                s = 0.0
                for irest in itertools.product(*[range(dims[m]) for m in others]):
                    idx = [0] * p
                    idx[n] = i_n
                    f = 1.0
                    for m, im, am in zip(others, irest, a):
                        idx[m] = im
                        f *= w[m][im] * U[m][im, am]
                    s += f * dV[tuple(idx)]
                Yref[i_n, col] = s
        np.testing.assert_allclose(Y[n], Yref, rtol=1e-12, atol=1e-14)


def test_projection_consistency_and_column_order():
    """dS = Y_n x_n A_n^T for every n; Y_(n) T_(n)^T is the same in the cyclic
    column order of Sec. 2.1 and the Kolda-Bader order of Sec. 2.2."""
    rng = np.random.default_rng(2)
    dims, ranks = (9, 7, 6, 5), (3, 2, 4, 2)
    w = [_rand_weights(rng, N) for N in dims]
    U = [_rand_orth_w(rng, N, r, wn) for N, r, wn in zip(dims, ranks, w)]
    dV = rng.standard_normal(dims)
    T = rng.standard_normal(ranks)
    dS, Y = O.project(dV, U, w)
    A = O.weighted_bases(U, w)
    for n in range(4):
        shape = list(ranks)
        shape[n] = dims[n]
        Yt = O.fold(Y[n], n, shape)
        np.testing.assert_allclose(O.mode_product(Yt, A[n].T, n), dS, rtol=1e-12, atol=1e-13)
        # cyclic order: columns r_{n+1} ... r_p r_1 ... r_{n-1}, first listed fastest
        perm = [n] + list(range(n + 1, 4)) + list(range(0, n))
        Yc = np.reshape(np.transpose(Yt, perm), (dims[n], -1), order="F")
        Tc = np.reshape(np.transpose(T, perm), (ranks[n], -1), order="F")
        np.testing.assert_allclose(Yc @ Tc.T, Y[n] @ O.unfold(T, n).T, rtol=1e-12, atol=1e-12)


def test_p2_matrix_case_is_dbo_gemms():
    """p = 2 (DBO, Sec. 2.2): the projections are plain matrix products."""
    rng = np.random.default_rng(3)
    N1, N2, r1, r2 = 11, 8, 3, 4
    w = [_rand_weights(rng, N1), _rand_weights(rng, N2)]
    U = [_rand_orth_w(rng, N1, r1, w[0]), _rand_orth_w(rng, N2, r2, w[1])]
    dV = rng.standard_normal((N1, N2))
    dS, Y = O.project(dV, U, w)
    W1, W2 = np.diag(w[0]), np.diag(w[1])
    np.testing.assert_allclose(dS, U[0].T @ W1 @ dV @ W2 @ U[1], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Y[0], dV @ W2 @ U[1], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(Y[1], dV.T @ W1 @ U[0], rtol=1e-12, atol=1e-14)
    # and the basis update is the DBO one: (I - U U^T W) Y (T T^T)^{-1} T etc.
    T = rng.standard_normal((r1, r2))
    dU1 = O.basis_rhs(Y[0], T, U[0], w[0], 0)
    ref = (np.eye(N1) - U[0] @ U[0].T @ W1) @ (dV @ W2 @ U[1]) @ T.T @ np.linalg.inv(T @ T.T)
    np.testing.assert_allclose(dU1, ref, rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------------------
# The evolution equations: exact cases and convergence orders
# ---------------------------------------------------------------------------

def test_fixed_subspace_is_exact():
    """Data V_k = T_k x U with fixed U and full-rank T_k: the complement projection
    of Y_n vanishes, dU = 0, and Euler with the data difference reproduces every
    snapshot (Eqs. 2.15, 2.16)."""
    rng = np.random.default_rng(4)
    dims, ranks = (12, 10, 8), (3, 4, 2)
    w = [_rand_weights(rng, N) for N in dims]
    U = [_rand_orth_w(rng, N, r, wn) for N, r, wn in zip(dims, ranks, w)]
    T0 = rng.standard_normal(ranks)
    T1 = rng.standard_normal(ranks)

    def V(k):
        t = 0.01 * k
        return O.reconstruct(T0 * math.cos(t) + T1 * math.sin(3 * t) + 0.1 * t * T0 * T1, U)

    T = O.multi_mode_product(V(0), [a.T for a in O.weighted_bases(U, w)])
    Uc = [u.copy() for u in U]
    worst = 0.0
    for k in range(1, 201):
        T, Uc, _, _ = O.step_euler(T, Uc, w, V(k - 1), V(k))
        Vk = V(k)
        worst = max(worst, O.error_exact(Vk, T, Uc, w) / math.sqrt(O.weighted_norm2(Vk, w)))
    assert worst <= 1e-13


def _analytic_run(n, steps, dt, scheme):
    wl = S.make_workload("analytic", n=n, dt=dt, steps=steps)
    w = wl.weights
    V0 = wl.logical(0)
    T, U, _ = O.hosvd(V0, w, [4, 4, 4])
    vdot = lambda t: S.to_logical(wl.snapshot_dot(t))
    Vp, Vpp = V0, None
    orth = 0.0
    for k in range(1, steps + 1):
        if scheme == "rk4":
            T, U = O.step_rk4(T, U, w, (k - 1) * dt, dt, vdot)
        elif scheme == "heun":
            Vk = wl.logical(k)
            T, U = O.step_heun(T, U, w, Vp, Vk)
            Vp = Vk
        elif scheme == "rk2c":
            Vk = wl.logical(k)
            T, U = O.step_rk2_central(T, U, w, Vpp, Vp, Vk)
            Vpp, Vp = Vp, Vk
        else:
            Vk = wl.logical(k)
            T, U, _, _ = O.step_euler(T, U, w, Vp, Vk)
            Vp = Vk
        for n in range(3):
            orth = max(orth, np.abs(U[n].T @ (w[n][:, None] * U[n]) - np.eye(4)).max())
    V = wl.logical(steps)
    return O.error_exact(V, T, U, w) / math.sqrt(O.weighted_norm2(V, w)), orth


def test_exact_recovery_rk4_order4():
    """Multilinear rank <= r: the continuous equations keep e = 0 (Eq. 2.5 with 2.15,
    2.16), so RK4 with the exact derivative converges at order 4."""
    e1, _ = _analytic_run(32, 50, 4e-3, "rk4")
    e2, orth = _analytic_run(32, 100, 2e-3, "rk4")
    assert 12.0 < e1 / e2 < 20.0
    assert e2 < 1e-9
    assert orth <= 1e-12


def test_exact_recovery_analytic_64_to_1e10():
    """The 64^3, dt = 1e-3, 200-step analytic field is recovered to 1e-10 relative."""
    e, orth = _analytic_run(64, 200, 1e-3, "rk4")
    assert e <= 1e-10
    assert orth <= 1e-12


def test_euler_difference_first_order():
    """Explicit Euler with the first-order data difference converges at order 1
    (Sec. 3.1 compares these schemes); it does not reach 1e-10 on moving subspaces."""
    e1, _ = _analytic_run(32, 25, 8e-3, "ee")
    e2, orth = _analytic_run(32, 50, 4e-3, "ee")
    assert 1.6 < e1 / e2 < 2.4
    assert e2 > 1e-6
    assert orth <= 1e-12


def test_heun_difference_at_least_second_order():
    """Heun's scheme with the data difference on both stages is at least second order
    (Sec. 3.1 compares Runge-Kutta schemes with Euler): halving dt divides the error by
    more than 4 (about 8 on this exact-rank field), and it beats Euler at the same dt by
    more than an order of magnitude.  Evaluating stage 2 at the old state (Euler again)
    or dropping a stage fails the ratio."""
    e1, _ = _analytic_run(32, 25, 8e-3, "heun")
    e2, orth = _analytic_run(32, 50, 4e-3, "heun")
    ee2, _ = _analytic_run(32, 50, 4e-3, "ee")
    assert 3.5 < e1 / e2 < 12.0
    assert e2 < ee2 / 20.0
    assert orth <= 1e-12


def test_rotation_covariance():
    """Starting from (U_n Q_n, T x_n Q_n^T) gives the same T x U trajectory: the
    method does not depend on the basis inside the subspace (Sec. 2.4)."""
    rng = np.random.default_rng(5)
    wl = S.make_workload("reactive", nx=24, ny=20, ns=6)
    w = wl.weights
    V = [wl.logical(k) for k in range(0, 21)]
    T, U, _ = O.hosvd(V[0], w, [4, 4, 3])
    Q = [np.linalg.qr(rng.standard_normal((r, r)))[0] for r in (4, 4, 3)]
    T2 = O.multi_mode_product(T, [q.T for q in Q])
    U2 = [u @ q for u, q in zip(U, Q)]
    for k in range(1, 21):
        T, U, _, _ = O.step_euler(T, U, w, V[k - 1], V[k])
        T2, U2, _, _ = O.step_euler(T2, U2, w, V[k - 1], V[k])
        R1, R2 = O.reconstruct(T, U), O.reconstruct(T2, U2)
        assert np.abs(R1 - R2).max() <= 1e-12 * np.abs(R1).max()


# ---------------------------------------------------------------------------
# HOSVD, singular values, gamma and the error (Secs. 2.4, 2.5)
# ---------------------------------------------------------------------------

def test_hosvd_against_library_svd():
    rng = np.random.default_rng(6)
    dims = (9, 7, 5)
    w = [_rand_weights(rng, N) for N in dims]
    V = rng.standard_normal(dims)
    ranks = (4, 3, 2)
    T, U, spec = O.hosvd(V, w, ranks)
    Vw = O.multi_mode_product(V, [np.diag(np.sqrt(x)) for x in w])
    for n in range(3):
        Ls, s, _ = np.linalg.svd(O.unfold(Vw, n), full_matrices=False)
        np.testing.assert_allclose(np.sqrt(np.maximum(spec[n][0][: len(s)], 0)), s, rtol=1e-10)
        # same subspace: projectors agree
        Q = np.sqrt(w[n])[:, None] * U[n]
        np.testing.assert_allclose(Q @ Q.T, Ls[:, : ranks[n]] @ Ls[:, : ranks[n]].T, atol=1e-10)
        np.testing.assert_allclose(U[n].T @ (w[n][:, None] * U[n]), np.eye(ranks[n]), atol=1e-12)


def test_core_singular_values_follow_hosvd_at_init():
    """At full rank in the other modes, sigma^(n) of the HOSVD core equals the
    leading mode-n singular values of the data (Sec. 2.4)."""
    rng = np.random.default_rng(7)
    dims = (8, 6, 5)
    w = [_rand_weights(rng, N) for N in dims]
    V = rng.standard_normal(dims)
    for n in range(3):
        ranks = list(dims)
        ranks[n] = 3
        T, U, spec = O.hosvd(V, w, ranks)
        sig = O.core_singular_values(T)[n]
        np.testing.assert_allclose(sig, np.sqrt(spec[n][0][:3]), rtol=1e-12)


def test_gamma_forms_agree_for_matrices():
    """For p = 2 at the truncated SVD, eps^2 is the discarded energy, so the two
    forms of Eq. 2.21 coincide."""
    rng = np.random.default_rng(8)
    N1, N2, r = 12, 9, 4
    w = [_rand_weights(rng, N1), _rand_weights(rng, N2)]
    V = rng.standard_normal((N1, N2)) @ np.diag(np.exp(-np.arange(N2)))
    T, U, spec = O.hosvd(V, w, [r, r])
    eps = O.error_exact(V, T, U, w)
    sig = O.core_singular_values(T)
    lam = spec[0][0]
    g1 = np.sum(lam[:r]) / np.sum(lam) * 100
    assert abs(O.gamma_percent(sig[0], eps) - g1) < 1e-10
    assert abs(O.gamma_percent(sig[1], eps) - g1) < 1e-10


def test_error_pythagorean_identity():
    """eps^2 = ||V||^2 - ||P V||^2 + ||P V - T||^2 with P V = V x_n A_n^T, because the
    U_n are W-orthonormal (Eq. 2.6, Eq. 2.20)."""
    rng = np.random.default_rng(9)
    dims, ranks = (10, 9, 7), (3, 4, 3)
    w = [_rand_weights(rng, N) for N in dims]
    U = [_rand_orth_w(rng, N, r, wn) for N, r, wn in zip(dims, ranks, w)]
    V = rng.standard_normal(dims)
    T = rng.standard_normal(ranks)
    PV = O.multi_mode_product(V, [a.T for a in O.weighted_bases(U, w)])
    lhs = O.error_exact(V, T, U, w) ** 2
    rhs = O.weighted_norm2(V, w) - np.sum(PV ** 2) + np.sum((PV - T) ** 2)
    assert abs(lhs - rhs) <= 1e-10 * lhs


def test_rank_selection_rules():
    lam = np.array([50.0, 30.0, 15.0, 4.0, 0.9, 0.1])    # total 100
    assert O.rank_from_spectrum(lam, 80.0) == 2
    assert O.rank_from_spectrum(lam, 95.0) == 3
    assert O.rank_from_spectrum(lam, 99.0) == 4
    assert O.rank_from_spectrum(lam, 99.95) == 6
    sig = np.sqrt(np.array([50.0, 30.0, 15.0, 4.0]))
    # denominator 99 + eps^2 = 100 -> same thresholds as above
    assert O.rank_from_core(sig, 1.0, 95.0) == 3
    assert O.rank_from_core(sig, 1.0, 99.5) == 4
    assert O.clamp_product_bound([5, 1, 2]) == [2, 1, 2]
    assert O.rank_caps([10, 3, 2], [8, 8, 8]) == [6, 3, 2]


# ---------------------------------------------------------------------------
# Compression ratios (Sec. 2.6, Sec. 3.2) and the paper's printed numbers
# ---------------------------------------------------------------------------

def test_compression_ratio_closed_forms():
    # CR at the channel case's initial multirank (Sec. 3.4): 150^3 / (150 (54+57+36) + 54*57*36)
    assert abs(O.compression_ratio([150, 150, 150], [54, 57, 36]) - 3375000 / 132858) < 1e-12
    # S_TDB-1 equals the CR denominator for three modes (Sec. 3.2 vs Sec. 2.6)
    assert O.storage_tdb1(5, 6, 7, 251, 76, 23) == 5 * 251 + 6 * 76 + 7 * 23 + 5 * 6 * 7
    assert abs(O.compression_ratio([251, 76, 23], [5, 6, 7]) - 251 * 76 * 23 / O.storage_tdb1(5, 6, 7, 251, 76, 23)) < 1e-12
    # TDB-2 with a 2-D spatial basis is the two-mode CR
    assert abs(O.compression_ratio([251 * 76, 23], [7, 7]) - 251 * 76 * 23 / O.storage_tdb2(7, 251, 76, 23)) < 1e-12


def test_weighted_cr_is_total_size_ratio():
    """CR-bar (Eq. 2.22) over a piecewise-constant rank history equals total raw
    size over total compressed size for snapshots uniform in time."""
    rng = np.random.default_rng(10)
    dims = [40, 30, 20]
    times = [0.0]
    crs, raw, comp = [], 0.0, 0.0
    for _ in range(7):
        r = list(rng.integers(2, 9, size=3))
        nsteps = int(rng.integers(3, 50))
        times.append(times[-1] + nsteps)
        cr = O.compression_ratio(dims, r)
        crs.append(cr)
        raw += nsteps * np.prod(dims)
        comp += nsteps * (sum(a * b for a, b in zip(r, dims)) + np.prod(r))
    assert abs(O.weighted_compression_ratio(times, crs) - raw / comp) < 1e-9 * (raw / comp)


def test_printed_compression_numbers_consistent():
    """The paper's CR-bar values agree with its printed sizes within the rounding
    of the printed sizes (CR-bar is a size ratio, Eq. 2.22)."""
    with open(os.path.join(GOLDEN, "printed_compression.json")) as f:
        rows = json.load(f)["rows"]
    for row in rows:
        raw, comp, crbar, ulp = row["raw_gb"], row["compressed_gb"], row["crbar"], row["compressed_rounding_gb"]
        lo, hi = raw / (comp + ulp / 2), raw / (comp - ulp / 2)
        assert lo <= crbar <= hi, row


# ---------------------------------------------------------------------------
# Rank control (Sec. 2.5) on constructed data with a known spectrum
# ---------------------------------------------------------------------------

def _lowrank_tensor(rng, dims, energies):
    """Sum of rank-one terms with W-orthonormal factors and the given energies."""
    w = [np.full(N, 1.0 / N) for N in dims]
    k = len(energies)
    F = [_rand_orth_w(rng, N, k, wn) for N, wn in zip(dims, w)]
    core = np.zeros((k,) * len(dims))
    for j, e in enumerate(energies):
        core[(j,) * len(dims)] = math.sqrt(e)
    return O.reconstruct(core, F), w


def test_controller_reinit_then_increase():
    rng = np.random.default_rng(11)
    energies = [1.0, 0.3, 0.1, 1e-3, 1e-5, 1e-8]
    V, w = _lowrank_tensor(rng, (10, 9, 8), energies)
    ctrl = O.Controller(O.ControllerConfig(eps_th=2e-3, gamma_th=99.9999, slope_window=3,
                                           rank_max=[6, 6, 6]), V.shape, w)
    T, U, _ = O.hosvd(V, w, [2, 2, 2])
    eps = O.error_exact(V, T, U, w)
    assert eps > 2e-3
    st, e1, n_re, action = ctrl.act(V, O.TDBState(T, U), eps)
    # gamma_th = 99.9999 % of total energy asks for 5 modes (kept energy reaches 1 - 1e-8/1.40101)
    assert action == "increase" and st.ranks == [5, 5, 5] and e1 <= 2e-3 and n_re == 2


def test_controller_cap_and_increment_rule():
    rng = np.random.default_rng(12)
    energies = [1.0, 0.5, 0.2, 0.1]
    V, w = _lowrank_tensor(rng, (7, 6, 5), energies)
    ctrl = O.Controller(O.ControllerConfig(eps_th=1e-12, gamma_th=50.0, slope_window=3,
                                           rank_max=[2, 3, 2]), V.shape, w)
    T, U, _ = O.hosvd(V, w, [1, 1, 1])
    st, e1, n_re, action = ctrl.act(V, O.TDBState(T, U), 1.0)
    # gamma 50 % needs 1 mode; the increment rule then raises mode by mode up to the caps
    # (1,1,1) -> (2,2,1) [mode 1 follows for the product bound] -> (2,2,2) -> (2,3,2) -> cap
    assert action == "cap" and st.ranks == [2, 3, 2] and e1 > 1e-12 and n_re == 4


def test_controller_decrease_and_revert():
    rng = np.random.default_rng(13)
    energies = [1.0, 0.2, 1e-9]
    V, w = _lowrank_tensor(rng, (8, 7, 6), energies)
    T, U, _ = O.hosvd(V, w, [3, 3, 3])
    eps0 = O.error_exact(V, T, U, w)
    cfgd = O.ControllerConfig(eps_th=1e-3, gamma_th=99.99, slope_window=2, rank_max=[3, 3, 3])
    ctrl = O.Controller(cfgd, V.shape, w)
    st = O.TDBState(T, U)
    # falling error over K = 2 steps, and the third mode carries < 0.01 % of the energy
    actions = [ctrl.act(V, st, e)[3] for e in (3e-4, 2e-4)]
    assert actions == ["none", "none"]
    st2, e2, n_re, action = ctrl.act(V, st, 1e-4)
    assert action == "decrease" and st2.ranks == [2, 2, 2] and n_re == 1 and e2 <= 1e-3
    # same situation with a threshold the reduced reconstruction cannot meet: revert
    ctrl = O.Controller(O.ControllerConfig(eps_th=1e-6, gamma_th=99.99, slope_window=2,
                                           rank_max=[3, 3, 3]), V.shape, w)
    for e in (3e-7, 2e-7):
        ctrl.act(V, st, e)
    st3, e3, n_re, action = ctrl.act(V, st, 1e-7)
    assert action == "revert" and st3.ranks == [3, 3, 3] and e3 == 1e-7
    # rising error: no reduction
    ctrl = O.Controller(cfgd, V.shape, w)
    for e in (1e-4, 2e-4):
        ctrl.act(V, st, e)
    assert ctrl.act(V, st, 3e-4)[3] == "none"
    assert eps0 < 1e-3


def test_rank_from_core_counts_the_error_in_the_denominator():
    """Eq. 2.21, second form: gamma(r) = sum_{i<=r} sigma_i^2 / (sum_i sigma_i^2 + eps^2).
    With sigma^2 = (1/2, 1/4, 1/4) and gamma_th = 60 %, eps = 0 needs r = 2 (3/4 >= 0.6);
    eps^2 = 1 makes the target 1.2, which no r reaches, so the rule keeps every mode."""
    sig = np.sqrt(np.array([0.5, 0.25, 0.25]))
    assert O.rank_from_core(sig, 0.0, 60.0) == 2
    assert O.rank_from_core(sig, 1.0, 60.0) == 3
    # eps^2 = 1/4: target 0.75, reached at r = 2 exactly
    assert O.rank_from_core(sig, 0.5, 60.0) == 2
    assert O.rank_from_core(sig, 0.5, 61.0) == 3


def test_controller_raise_ties_go_to_the_lowest_mode():
    """Equal discarded HOSVD energy in every mode: the increment rule raises mode 1 (the
    lowest index), and the product bound needs no other mode to follow.  Fractions within
    1e-9 relative + 1e-12 count as equal (rounding of equal spectra)."""
    lam = np.array([1.0, 0.5, 0.25, 0.125])
    w = [np.full(4, 0.25)] * 3
    ctrl = O.Controller(O.ControllerConfig(eps_th=1.0, gamma_th=99.0, slope_window=3, rank_max=[4, 4, 4]),
                        (4, 4, 4), w)
    assert ctrl._raise_one([2, 2, 2], [lam, lam, lam]) == [3, 2, 2]
    # unequal: the mode that discards most is raised
    assert ctrl._raise_one([2, 2, 2], [lam, lam, np.array([1.0, 0.5, 0.5, 0.5])]) == [2, 2, 3]
    # equal up to rounding (a symmetric field's modes): still a tie, the lowest mode is raised;
    # a difference well above rounding decides
    lam_up = lam * np.array([1.0, 1.0, 1.0 + 1e-13, 1.0 + 1e-13])
    assert ctrl._raise_one([2, 2, 2], [lam, lam_up, lam]) == [3, 2, 2]
    lam_more = lam * np.array([1.0, 1.0, 1.0 + 1e-4, 1.0 + 1e-4])
    assert ctrl._raise_one([2, 2, 2], [lam, lam_more, lam]) == [2, 3, 2]
    # small discarded fractions (1.3e-7) whose rounding-level absolute difference (7e-16) is
    # 5e-9 of them: still a tie; a difference of 1e-10 absolute decides
    tail = np.array([1.0, 0.5, 1e-7, 1e-7])
    assert ctrl._raise_one([2, 2, 2], [tail, tail + np.array([0, 0, 1e-15, 0]), tail]) == [3, 2, 2]
    assert ctrl._raise_one([2, 2, 2], [tail, tail + np.array([0, 0, 1.5e-10, 0]), tail]) == [2, 3, 2]


def test_controller_slope_window_restarts_after_reinit():
    """Steps with a HOSVD re-initialisation are excluded from the error slope and the window
    restarts (Sec. 2.5): after a re-initialising act the history is empty, and it then
    holds exactly the errors of the following plain steps."""
    rng = np.random.default_rng(14)
    V, w = _lowrank_tensor(rng, (8, 7, 6), [1.0, 0.2, 1e-2])
    T, U, _ = O.hosvd(V, w, [2, 2, 2])
    ctrl = O.Controller(O.ControllerConfig(eps_th=1e-3, gamma_th=99.0, slope_window=3, rank_max=[3, 3, 3]),
                        V.shape, w)
    st = O.TDBState(T, U)
    for e in (5e-4, 4e-4):
        ctrl.act(V, st, e)
    assert ctrl.history == [5e-4, 4e-4]
    st2, _, n_re, action = ctrl.act(V, st, 0.5)     # above eps_th: re-initialise
    assert n_re >= 1 and action in ("reinit", "increase")
    assert ctrl.history == []
    ctrl.act(V, st2, 3e-4)
    assert ctrl.history == [3e-4]


def test_hosvd_sign_convention():
    """Each HOSVD vector's entry of largest magnitude is positive (the sign convention that
    makes the oracle's bases unique up to rotation within equal eigenvalues)."""
    rng = np.random.default_rng(15)
    dims = (9, 7, 6)
    w = [_rand_weights(rng, N) for N in dims]
    V = rng.standard_normal(dims)
    for lam, Q in O.hosvd_spectrum(V, w):
        for j in range(Q.shape[1]):
            i = int(np.argmax(np.abs(Q[:, j])))
            assert Q[i, j] > 0


def test_runge_field_and_derivative_closed_form():
    """The Runge workload is Eq. 3.1's function itself: values at grid points and the
    analytic time derivative against a central difference."""
    wl = S.make_workload("runge", n=9)
    x = np.linspace(-math.pi, math.pi, 9)
    t = 0.37
    a = 1.0 - 0.5 * math.exp(-0.5 * (t - 1.0) ** 2)
    V = S.to_logical(wl._field(t, torch.device("cpu")))
    for (i, j, k) in [(0, 0, 0), (4, 4, 4), (1, 7, 3), (8, 2, 5)]:
        assert V[i, j, k] == pytest.approx(1.0 / (a * a + x[i] ** 2 + x[j] ** 2 + x[k] ** 2), rel=1e-14)
    h = 1e-5
    fd = (S.to_logical(wl._field(t + h, torch.device("cpu"))) - S.to_logical(wl._field(t - h, torch.device("cpu")))) / (2 * h)
    dV = S.to_logical(wl.snapshot_dot(t))
    assert np.abs(fd - dV).max() <= 1e-8 * np.abs(dV).max()


def test_runge_ranks_rise_towards_t1_and_fall_after():
    """Sec. 3.1: with a(t) = 1 - 0.5 exp(-0.5 (t-1)^2) the rank that keeps the error
    below the threshold must grow from t = 0 to t = 1 and shrink after.  The oracle's
    controller on the function over t in [0, 2] (48^3 grid; the spectrum does not
    depend on the grid at this resolution) adds modes before t = 1, removes them after,
    and keeps every step's error at or below eps_th."""
    wl = S.make_workload("runge", n=48)
    snaps = [S.to_logical(wl.snapshot(k)) for k in range(0, wl.steps + 1)]
    ctrl = O.ControllerConfig(wl.eps_th, wl.gamma_th, 10, wl.rank_max)
    _, recs = O.compress_stream(snaps, wl.weights, [0, 0, 0], ctrl)
    total = [sum(r.ranks) for r in recs]
    t_of = lambda i: (i + 1) * wl.dt
    up = [i for i in range(1, len(recs)) if total[i] > total[i - 1]]
    down = [i for i in range(1, len(recs)) if total[i] < total[i - 1]]
    assert up and down, (up, down)
    assert all(t_of(i) <= 1.0 for i in up) and all(t_of(i) > 1.0 for i in down), (up, down)
    assert max(total) > total[0] and total[-1] < max(total)
    assert all(r.eps <= wl.eps_th for r in recs)


# ---------------------------------------------------------------------------
# The estimator network's reference (textbook back-propagation and Adam)
# ---------------------------------------------------------------------------

def test_mlp_gradient_matches_finite_differences():
    M = O.mlp_oracle
    rng = np.random.default_rng(14)
    F, H, B = 7, 64, 33
    theta = M.init_params(F, H, rng) + 0.01 * rng.standard_normal(M.n_params(F, H))
    X = rng.standard_normal((B, F))
    t = rng.standard_normal(B)
    L, g = M.loss_and_grad(theta, X, t, F, H)
    idx = rng.choice(theta.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (M.loss_and_grad(theta + e, X, t, F, H)[0] - M.loss_and_grad(theta - e, X, t, F, H)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i]))
    assert abs(L - np.mean((M.forward(theta, X, F, H) - t) ** 2)) < 1e-14


def test_mlp_adam_first_step_and_fit():
    M = O.mlp_oracle
    # first Adam step: bias correction makes m-hat = g and v-hat = g^2, so each
    # parameter moves by -lr g / (|g| + eps)
    g0 = np.array([2.0, -0.5, 1e-3])
    th, m, v = M.adam_update(np.zeros(3), g0, np.zeros(3), np.zeros(3), 1, 0.1)
    np.testing.assert_allclose(th, -0.1 * g0 / (np.abs(g0) + 1e-8), rtol=1e-12)
    # and training fits a smooth function
    rng = np.random.default_rng(15)
    F, H = 3, 64
    X = rng.uniform(-1, 1, size=(256, F))
    t = np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2]
    theta = M.init_params(F, H, rng)
    m = np.zeros_like(theta); v = np.zeros_like(theta)
    L0 = M.loss_and_grad(theta, X, t, F, H)[0]
    for s in range(1, 801):
        L, g = M.loss_and_grad(theta, X, t, F, H)
        theta, m, v = M.adam_update(theta, g, m, v, s, 3e-3)
    assert L < 0.02 * L0


# ---------------------------------------------------------------------------
# Coherent-structure rotation (Eq. 2.19)
# ---------------------------------------------------------------------------

def test_rotate_coherent_diagonalises_the_core_grams():
    """U~_n = U_n Psi_n (Eq. 2.19): recovering Psi_n = U_n^T W_n U~_n and rotating the core
    by Psi_n^T makes every T~_(n) T~_(n)^T diagonal with the squared core singular values
    (Eq. 2.18, computed separately by an eigensolver) in descending order, keeps
    U~_n^T W_n U~_n = I, and leaves T x U unchanged."""
    rng = np.random.default_rng(77)
    dims, ranks = (9, 8, 7), (4, 3, 3)
    w = [_rand_weights(rng, N) for N in dims]
    U = [_rand_orth_w(rng, N, r, wn) for N, r, wn in zip(dims, ranks, w)]
    T = rng.standard_normal(ranks)
    Ut = O.rotate_coherent(T, U)
    Psi = [U[n].T @ (w[n][:, None] * Ut[n]) for n in range(3)]
    Tt = T
    for n in range(3):
        Tt = O.mode_product(Tt, Psi[n].T, n)
    sig = O.core_singular_values(T)
    for n in range(3):
        G = O.unfold(Tt, n) @ O.unfold(Tt, n).T
        assert np.abs(G - np.diag(np.diag(G))).max() <= 1e-12 * np.abs(G).max()
        np.testing.assert_allclose(np.diag(G), sig[n] ** 2, rtol=1e-12)
        np.testing.assert_allclose(Ut[n].T @ (w[n][:, None] * Ut[n]), np.eye(ranks[n]), atol=1e-12)
    ref = O.reconstruct(T, U)
    assert np.abs(O.reconstruct(Tt, Ut) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_rk2_central_second_order():
    """The midpoint RK2 scheme with central differences of the data (Sec. 3.1) converges at
    order 2: halving dt divides the error by about 4, and it is more than ten times more
    accurate than Euler with the first-order difference at the same dt.  A wrong stage
    weight or a first-order derivative in either stage falls back to order 1."""
    e1, _ = _analytic_run(32, 25, 8e-3, "rk2c")
    e2, orth = _analytic_run(32, 50, 4e-3, "rk2c")
    ee2, _ = _analytic_run(32, 50, 4e-3, "ee")
    assert 3.2 < e1 / e2 < 5.0
    assert e2 < ee2 / 10.0
    assert orth <= 1e-12


def test_rk2_central_uses_the_exact_derivatives_of_quadratic_data():
    """For data quadratic in time, V(t) = A + B t + C t^2, both central differences are
    exact: (V(t+h) - V(t-h)) / 4 = (h/2) V'(t) and V(t+h) - V(t) = h V'(t + h/2).  The
    scheme's step then equals the midpoint RK2 step taken with the exact derivatives,
    and its first step (no V_{k-1}) uses (V(t+h) - V(t)) / 2 = (h/2) V'(t + h/2)."""
    rng = np.random.default_rng(31)
    dims, ranks = (9, 7, 5), (3, 3, 2)
    w = [rng.uniform(0.5, 1.5, N) for N in dims]
    w = [x / x.sum() for x in w]
    A, B, C = (rng.standard_normal(dims) for _ in range(3))
    V = lambda t: A + B * t + C * t * t
    Vd = lambda t: B + 2.0 * C * t
    T, U, _ = O.hosvd(V(0.3), w, list(ranks))
    t, h = 0.3, 0.05
    T1, U1 = O.step_rk2_central(T, U, w, V(t - h), V(t), V(t + h), reorth=False)
    k1T, k1U = O.tdb_rhs(T, U, w, 0.5 * h * Vd(t))
    Tm, Um = T + k1T, [U[n] + k1U[n] for n in range(3)]
    k2T, k2U = O.tdb_rhs(Tm, Um, w, h * Vd(t + 0.5 * h))
    assert np.abs(T1 - (T + k2T)).max() <= 1e-12 * np.abs(T).max()
    for n in range(3):
        assert np.abs(U1[n] - (U[n] + k2U[n])).max() <= 1e-12 * np.abs(U[n]).max()
    # the first step: stage 1 with (V(t+h) - V(t)) / 2
    T2, _ = O.step_rk2_central(T, U, w, None, V(t), V(t + h), reorth=False)
    k1T, k1U = O.tdb_rhs(T, U, w, 0.5 * h * Vd(t + 0.5 * h))
    Tm, Um = T + k1T, [U[n] + k1U[n] for n in range(3)]
    k2T, _ = O.tdb_rhs(Tm, Um, w, h * Vd(t + 0.5 * h))
    assert np.abs(T2 - (T + k2T)).max() <= 1e-12 * np.abs(T).max()
