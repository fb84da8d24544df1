"""Plain FP64 restatement of the TDB compressor, one function per passage.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline / reference legs; never by the product path.

Conventions
-----------
* A p-mode tensor is a numpy float64 array of logical shape (N_1, ..., N_p);
  X[i_1, ..., i_p] is the paper's entry with 0-based indices.
* Unfoldings follow Kolda and Bader (cited in Sec. 2.1): the mode-n unfolding
  X_(n) has rows i_n and its columns run over the remaining modes in ascending
  order with the first remaining mode fastest.  This is the index map the
  paper writes out for the pseudo-inverse in Sec. 2.2 (column i'_2 + (i'_3-1) r_2
  for mode 1).  Sec. 2.1 also names a cyclic column order; the products
  Y_(n) T_(n)^T and T_(n) T_(n)^T do not depend on the column order as long as
  both factors use the same one, and the tests check that.
* The n-mode product X x_n A (A of shape J x N_n) replaces mode n by J:
  (X x_n A)[.., j, ..] = sum_i A[j, i] X[.., i, ..]   (Sec. 2.1).
* Quadrature weights w_n are the diagonals of W^(n) (Eq. 2.17).  The weighted
  bases A_n = W^(n) U^(n) are what the discrete inner products contract with.

Parity status: every function here is pinned by a test in
tests/test_oracle_*.py except where its docstring says "parity unpinned".
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "unfold", "fold", "mode_product", "multi_mode_product", "weighted_bases",
    "project", "core_gram", "basis_rhs", "tdb_rhs", "step_euler", "step_heun", "step_rk2_central", "step_rk4",
    "cholqr", "reconstruct", "weighted_norm2", "error_exact",
    "hosvd_spectrum", "hosvd", "rank_from_spectrum", "rank_from_core",
    "core_singular_values", "gamma_percent", "rotate_coherent",
    "compression_ratio", "weighted_compression_ratio", "storage_tdb1",
    "storage_tdb2", "rank_caps", "clamp_product_bound", "Controller",
    "ControllerConfig", "StepRecord", "TDBState", "compress_stream",
]


# ---------------------------------------------------------------------------
# Tensor algebra (Sec. 2.1)
# ---------------------------------------------------------------------------

def unfold(X: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding X_(n) (Sec. 2.1), Kolda-Bader column order."""
    return np.reshape(np.moveaxis(X, n, 0), (X.shape[n], -1), order="F")


def fold(M: np.ndarray, n: int, shape: Sequence[int]) -> np.ndarray:
    """Inverse of :func:`unfold` for a tensor of logical ``shape``."""
    rest = [shape[m] for m in range(len(shape)) if m != n]
    X = np.reshape(M, [shape[n]] + rest, order="F")
    return np.moveaxis(X, 0, n)


def mode_product(X: np.ndarray, A: np.ndarray, n: int) -> np.ndarray:
    """n-mode product X x_n A with A of shape (J, N_n) (Sec. 2.1)."""
    return np.moveaxis(np.tensordot(A, X, axes=(1, n)), 0, n)


def multi_mode_product(X: np.ndarray, mats: Sequence[Optional[np.ndarray]]) -> np.ndarray:
    """X x_1 mats[0] x_2 mats[1] ... ; a ``None`` entry leaves that mode alone."""
    for n, A in enumerate(mats):
        if A is not None:
            X = mode_product(X, A, n)
    return X


def weighted_bases(U: Sequence[np.ndarray], w: Sequence[np.ndarray]) -> List[np.ndarray]:
    """A_n = W^(n) U^(n): the discrete inner product <u, v>_{x_n} = u^T W^(n) v (Eq. 2.17)."""
    return [w[n][:, None] * U[n] for n in range(len(U))]


# ---------------------------------------------------------------------------
# Projection of the data derivative (Eqs. 2.15 and 2.16, discrete form Sec. 2.3)
# ---------------------------------------------------------------------------

def project(dV: np.ndarray, U: Sequence[np.ndarray], w: Sequence[np.ndarray]):
    """Fused multi-mode projection of a data increment dV.

    dS  = dV x_1 A_1^T x_2 ... x_p A_p^T                    (Eq. 2.15, right side)
    Y_n = [dV x_{m != n} A_m^T]_(n)   (N_n x prod_{m!=n} r_m)  (Eq. 2.16, the
          inner product over every space except x_n)
    with A_n = W^(n) U^(n).  Returned as (dS, [Y_1, ..., Y_p]).
    """
    A = weighted_bases(U, w)
    p = dV.ndim
    dS = multi_mode_product(dV, [a.T for a in A])
    Y = []
    for n in range(p):
        Z = multi_mode_product(dV, [A[m].T if m != n else None for m in range(p)])
        Y.append(unfold(Z, n))
    return dS, Y


def core_gram(T: np.ndarray, n: int) -> np.ndarray:
    """G_n = T_(n) T_(n)^T, the r_n x r_n matrix inverted by the pseudo-inverse (Sec. 2.2, Sec. 2.6 item 2)."""
    Tn = unfold(T, n)
    return Tn @ Tn.T


def basis_rhs(Y_n: np.ndarray, T: np.ndarray, U_n: np.ndarray, w_n: np.ndarray, n: int) -> np.ndarray:
    """Right side of Eq. 2.16 for mode n, times the time step.

    X   = Y_(n) T_(n)^dagger,  T_(n)^dagger = T_(n)^T (T_(n) T_(n)^T)^{-1}  (Sec. 2.2)
    dU  = (I - U U^T W) X       (the complement projector of Sec. 2.2, weighted per Eq. 2.17)
    """
    Tn = unfold(T, n)
    G = Tn @ Tn.T
    M = Y_n @ Tn.T                       # N_n x r_n
    X = np.linalg.solve(G, M.T).T        # M G^{-1}; G is symmetric
    P = U_n.T @ (w_n[:, None] * X)       # U^T W X
    return X - U_n @ P


def tdb_rhs(T: np.ndarray, U: Sequence[np.ndarray], w: Sequence[np.ndarray], dV: np.ndarray):
    """(dT, [dU_n]) for a data increment dV, gauge phi = 0 (Eqs. 2.15, 2.16).

    With dV = V(t + dt) - V(t) this is dt times the continuous right side evaluated
    with the first-order forward difference of the data (Sec. 2.3); with
    dV = dt * dV/dt it is dt times the exact right side.
    """
    dS, Y = project(dV, U, w)
    dU = [basis_rhs(Y[n], T, U[n], w[n], n) for n in range(T.ndim)]
    return dS, dU


def cholqr(T: np.ndarray, U: Sequence[np.ndarray], w: Sequence[np.ndarray]):
    """Weighted Cholesky-QR re-orthonormalisation with core compensation.

    The paper does not re-orthonormalise; this is the reading used here (its
    Eq. 2.6 is the invariant being restored).  For each mode,
    C = U^T W U = R^T R,  U <- U R^{-1},  T <- T x_n R,
    so that T x_1 U_1 ... x_p U_p is unchanged.
    """
    U_out = []
    for n in range(T.ndim):
        C = U[n].T @ (w[n][:, None] * U[n])
        R = np.linalg.cholesky(C).T            # upper, C = R^T R
        U_out.append(np.linalg.solve(R.T, U[n].T).T)   # U R^{-1}
        T = mode_product(T, R, n)
    return T, U_out


def step_euler(T, U, w, V_k, V_k1, reorth: bool = True):
    """One explicit-Euler step with the first-order data difference (Sec. 2.3; Sec. 3.1
    names the Euler scheme).  dt cancels: T' = T + dS, U_n' = U_n + dU_n, all right
    sides taken at the state of step k.  Returns (T', U', dS, Y)."""
    dV = V_k1 - V_k
    dS, Y = project(dV, U, w)
    dU = [basis_rhs(Y[n], T, U[n], w[n], n) for n in range(T.ndim)]
    T1 = T + dS
    U1 = [U[n] + dU[n] for n in range(T.ndim)]
    if reorth:
        T1, U1 = cholqr(T1, U1, w)
    return T1, U1, dS, Y


def step_heun(T, U, w, V_k, V_k1, reorth: bool = True):
    """One step of Heun's second-order Runge-Kutta scheme on the same equations, with the
    data forcing taken from the piecewise-linear interpolant of the snapshots (both stages
    use the step's difference V_k1 - V_k; the paper's Sec. 3.1 compares this family of
    schemes with Euler).  Stage 1 is the Euler increment at the state of step k, stage 2
    the increment at the predicted state; the step takes their mean, then re-orthonormalises
    (reading C4; the predicted state is an intermediate of the scheme and is not).
    Returns (T', U')."""
    dV = V_k1 - V_k
    k1T, k1U = tdb_rhs(T, U, w, dV)
    Tp = T + k1T
    Up = [U[n] + k1U[n] for n in range(T.ndim)]
    k2T, k2U = tdb_rhs(Tp, Up, w, dV)
    T1 = T + 0.5 * (k1T + k2T)
    U1 = [U[n] + 0.5 * (k1U[n] + k2U[n]) for n in range(T.ndim)]
    if reorth:
        T1, U1 = cholqr(T1, U1, w)
    return T1, U1


def step_rk2_central(T, U, w, V_km1, V_k, V_k1, reorth: bool = True):
    """One step of the midpoint second-order Runge-Kutta scheme with second-order central
    differences of the data (Sec. 3.1 compares the central second-order approximation of
    the data derivative with the first-order one and with the exact derivative, and
    advances with a second-order RK scheme; Sec. 2.3 notes that higher-order differences
    keep several snapshots in memory).  Stage 1 takes the derivative at t_k,
    dt V'(t_k) ~ (V_{k+1} - V_{k-1}) / 2, over half a step to the midpoint state; stage 2
    takes the derivative at t_k + dt/2, dt V'(t_k + dt/2) ~ V_{k+1} - V_k (the central
    difference about the midpoint), at the midpoint state, over the whole step from the
    state of step k.  Without V_{k-1} (the first step) stage 1 uses (V_{k+1} - V_k) / 2.
    Re-orthonormalisation after the step (reading C4; the midpoint state is an
    intermediate of the scheme and is not).  Returns (T', U')."""
    dV1 = 0.25 * (V_k1 - V_km1) if V_km1 is not None else 0.5 * (V_k1 - V_k)
    k1T, k1U = tdb_rhs(T, U, w, dV1)
    Tm = T + k1T
    Um = [U[n] + k1U[n] for n in range(T.ndim)]
    k2T, k2U = tdb_rhs(Tm, Um, w, V_k1 - V_k)
    T1 = T + k2T
    U1 = [U[n] + k2U[n] for n in range(T.ndim)]
    if reorth:
        T1, U1 = cholqr(T1, U1, w)
    return T1, U1


def step_rk4(T, U, w, t: float, dt: float, vdot, reorth: bool = True):
    """Classical RK4 on the continuous equations (2.15, 2.16) with the exact data
    derivative ``vdot(t)`` (the paper's adaptivity study uses the exact derivative,
    Sec. 3.1).  Used only to pin the right-hand side: the error of an exact-rank
    field must fall as dt^4."""
    def rhs(Ts, Us, ts):
        return tdb_rhs(Ts, Us, w, vdot(ts))

    k1T, k1U = rhs(T, U, t)
    T2 = T + 0.5 * dt * k1T
    U2 = [U[n] + 0.5 * dt * k1U[n] for n in range(T.ndim)]
    k2T, k2U = rhs(T2, U2, t + 0.5 * dt)
    T3 = T + 0.5 * dt * k2T
    U3 = [U[n] + 0.5 * dt * k2U[n] for n in range(T.ndim)]
    k3T, k3U = rhs(T3, U3, t + 0.5 * dt)
    T4 = T + dt * k3T
    U4 = [U[n] + dt * k3U[n] for n in range(T.ndim)]
    k4T, k4U = rhs(T4, U4, t + dt)
    Tn = T + dt / 6.0 * (k1T + 2 * k2T + 2 * k3T + k4T)
    Un = [U[n] + dt / 6.0 * (k1U[n] + 2 * k2U[n] + 2 * k3U[n] + k4U[n]) for n in range(T.ndim)]
    if reorth:
        Tn, Un = cholqr(Tn, Un, w)
    return Tn, Un


# ---------------------------------------------------------------------------
# Reconstruction and error (Eqs. 2.5, 2.20)
# ---------------------------------------------------------------------------

def reconstruct(T: np.ndarray, U: Sequence[np.ndarray]) -> np.ndarray:
    """V^TDB = T x_1 U_1 x_2 ... x_p U_p (Eq. 2.5 without the error term)."""
    return multi_mode_product(T, list(U))


def weighted_norm2(X: np.ndarray, w: Sequence[np.ndarray]) -> float:
    """||X||^2 in the weighted inner product of Eq. 2.2 with the quadrature of Eq. 2.17."""
    Wt = np.ones(X.shape)
    for n in range(X.ndim):
        shape = [1] * X.ndim
        shape[n] = X.shape[n]
        Wt = Wt * w[n].reshape(shape)
    return float(np.sum(Wt * X * X))


def error_exact(V: np.ndarray, T: np.ndarray, U: Sequence[np.ndarray], w) -> float:
    """epsilon = ||V - V^TDB||_F in the weighted norm (Eq. 2.20 and the sentence after it)."""
    return math.sqrt(weighted_norm2(V - reconstruct(T, U), w))


# ---------------------------------------------------------------------------
# HOSVD initialisation and singular values (Sec. 2.3 end, Sec. 2.4, Sec. 2.5)
# ---------------------------------------------------------------------------

def _sign_fix(Q: np.ndarray) -> np.ndarray:
    """Each column's entry of largest magnitude made positive (first such entry on ties)."""
    Q = Q.copy()
    for j in range(Q.shape[1]):
        i = int(np.argmax(np.abs(Q[:, j])))
        if Q[i, j] < 0:
            Q[:, j] = -Q[:, j]
    return Q


def hosvd_spectrum(V: np.ndarray, w: Sequence[np.ndarray]):
    """Per-mode eigen-decomposition of the weighted mode-n Gram matrix.

    C_n = W_n^{1/2} V_(n) (W_{-n}) V_(n)^T W_n^{1/2}, whose eigenvalues are the
    squared mode-n singular values of the weighted data (Sec. 2.4; Sec. 2.6 gives
    the same correlation matrix for the HOSVD cost).  Returns a list of
    (lambda descending, Q) with Q orthonormal columns, sign fixed.

    A mode longer than the product M of the others (a grouped spatial mode, Sec. 3.2)
    has C_n = B B^T of rank at most M, with B the weighted unfolding (N_n x M): its
    nonzero eigenvalues are the squared singular values of B and their eigenvectors B's
    left singular vectors.  For such a mode the thin SVD of B gives them (a library
    routine as a step, the same definition without forming the N_n x N_n matrix), and
    the list holds M eigenvalues and M vectors; the rest of the spectrum is zero.
    """
    sw = [np.sqrt(wn) for wn in w]
    Vw = multi_mode_product(V, [np.diag(s) for s in sw])
    out = []
    for n in range(V.ndim):
        Vn = unfold(Vw, n)
        if Vn.shape[0] > Vn.shape[1]:
            Q, sv, _ = np.linalg.svd(Vn, full_matrices=False)
            out.append((sv * sv, _sign_fix(Q)))
            continue
        C = Vn @ Vn.T
        lam, Q = np.linalg.eigh(C)
        order = np.argsort(lam)[::-1]
        out.append((lam[order], _sign_fix(Q[:, order])))
    return out


def rank_caps(dims: Sequence[int], rank_max: Sequence[int]) -> List[int]:
    """Largest admissible rank per mode: r_n <= N_n, r_n <= prod_{m!=n} N_m and the user cap."""
    p = len(dims)
    caps = []
    for n in range(p):
        other = 1
        for m in range(p):
            if m != n:
                other *= dims[m]
        caps.append(int(min(dims[n], other, rank_max[n])))
    return caps


def clamp_product_bound(r: Sequence[int]) -> List[int]:
    """r_n <= prod_{m!=n} r_m, needed for T_(n) T_(n)^T to be invertible (Sec. 2.2, the
    under/over-determined remark).  Applied mode by mode until nothing changes."""
    r = list(r)
    changed = True
    while changed:
        changed = False
        for n in range(len(r)):
            other = 1
            for m in range(len(r)):
                if m != n:
                    other *= r[m]
            if r[n] > other:
                r[n] = other
                changed = True
    return r


def rank_from_spectrum(lam: np.ndarray, gamma_th: float) -> int:
    """Smallest r with sum_{i<=r} lambda_i / sum_i lambda_i >= gamma_th / 100 (Eq. 2.21,
    first form, on the HOSVD spectrum; Sec. 2.5 picks the initial ranks this way)."""
    lam = np.maximum(np.asarray(lam, dtype=np.float64), 0.0)
    total = float(np.sum(lam))
    if total <= 0.0:
        return 1
    target = gamma_th / 100.0 * total
    acc = 0.0
    for i, v in enumerate(lam):
        acc += float(v)
        if acc >= target:
            return i + 1
    return len(lam)


def hosvd(V: np.ndarray, w: Sequence[np.ndarray], ranks: Sequence[int], spectrum=None):
    """Truncated HOSVD used to initialise and re-initialise the TDB (Sec. 2.3 end, Sec. 2.5).

    U_n = W_n^{-1/2} Q_n[:, :r_n] so that U_n^T W_n U_n = I (Eq. 2.6);
    T = V x_1 A_1^T ... x_p A_p^T (the projection of Eq. 2.15 applied to V).
    """
    if spectrum is None:
        spectrum = hosvd_spectrum(V, w)
    U = []
    for n in range(V.ndim):
        lam, Q = spectrum[n]
        U.append(Q[:, : ranks[n]] / np.sqrt(w[n])[:, None])
    T = multi_mode_product(V, [a.T for a in weighted_bases(U, w)])
    return T, U, spectrum


def core_singular_values(T: np.ndarray) -> List[np.ndarray]:
    """sigma^(n): singular values of T_(n) (Eq. 2.18), descending, via eig of T_(n) T_(n)^T."""
    out = []
    for n in range(T.ndim):
        ev = np.linalg.eigvalsh(core_gram(T, n))[::-1]
        out.append(np.sqrt(np.maximum(ev, 0.0)))
    return out


def gamma_percent(sigma_n: np.ndarray, eps: float, r: Optional[int] = None) -> float:
    """gamma^(n)(r) = sum_{i<=r} sigma_i^2 / (sum_{i<=r_n} sigma_i^2 + eps^2) * 100 (Eq. 2.21, second form)."""
    s2 = np.asarray(sigma_n, dtype=np.float64) ** 2
    if r is None:
        r = len(s2)
    return float(np.sum(s2[:r]) / (np.sum(s2) + eps * eps) * 100.0)


def rank_from_core(sigma_n: np.ndarray, eps: float, gamma_th: float) -> int:
    """Smallest r with gamma^(n)(r) >= gamma_th, gamma from the core (Eq. 2.21, second form)."""
    s2 = np.asarray(sigma_n, dtype=np.float64) ** 2
    denom = float(np.sum(s2)) + eps * eps
    target = gamma_th / 100.0 * denom
    acc = 0.0
    for i, v in enumerate(s2):
        acc += float(v)
        if acc >= target:
            return i + 1
    return len(s2)


def rotate_coherent(T: np.ndarray, U: Sequence[np.ndarray]):
    """Energy-ranked bases U~_n = U_n Psi_n with Psi_n the left singular vectors of T_(n) (Eq. 2.19)."""
    out = []
    for n in range(T.ndim):
        Psi, _, _ = np.linalg.svd(unfold(T, n), full_matrices=False)
        out.append(U[n] @ Psi)
    return out


# ---------------------------------------------------------------------------
# Compression ratios and storage (Sec. 2.6, Sec. 3.2)
# ---------------------------------------------------------------------------

def compression_ratio(dims: Sequence[int], ranks: Sequence[int]) -> float:
    """CR = prod N_n / (sum r_n N_n + prod r_n) (Sec. 2.6)."""
    return float(np.prod([float(d) for d in dims]) /
                 (sum(float(r) * float(d) for r, d in zip(ranks, dims)) + float(np.prod([float(r) for r in ranks]))))


def weighted_compression_ratio(times: Sequence[float], crs: Sequence[float]) -> float:
    """CR-bar = (t_m - t_0) / sum_i (t_i - t_{i-1}) / CR_i (Eq. 2.22); ``times`` has m+1 entries."""
    total = times[-1] - times[0]
    denom = sum((times[i + 1] - times[i]) / crs[i] for i in range(len(crs)))
    return float(total / denom)


def storage_tdb1(r1, r2, r3, N1, N2, ns) -> int:
    """S_TDB-1 = r1 N1 + r2 N2 + r3 n_s + r1 r2 r3 (Sec. 3.2)."""
    return r1 * N1 + r2 * N2 + r3 * ns + r1 * r2 * r3


def storage_tdb2(r, N1, N2, ns) -> int:
    """S_TDB-2 = r N1 N2 + r n_s + r^2 (Sec. 3.2)."""
    return r * N1 * N2 + r * ns + r * r


# ---------------------------------------------------------------------------
# Adaptive rank control (Sec. 2.5)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class ControllerConfig:
    eps_th: float                 # epsilon_th; <= 0 turns adaptivity off
    gamma_th: float               # percent, e.g. 99.999
    slope_window: int = 10        # K: error slope taken over K steps
    rank_max: Optional[List[int]] = None


@dataclasses.dataclass
class TDBState:
    T: np.ndarray
    U: List[np.ndarray]

    @property
    def ranks(self) -> List[int]:
        return list(self.T.shape)


@dataclasses.dataclass
class StepRecord:
    step: int
    eps: float            # exact error after the step (and after any re-initialisation)
    eps_step: float       # exact error of the Euler step before control acted
    ranks: List[int]
    reinit: int           # number of HOSVD re-initialisations performed at this step
    action: str           # "none", "reinit", "increase", "decrease", "revert", "cap"
    gamma: List[float]
    cr: float


# Difference below which two modes' discarded HOSVD energy fractions (1 - kept/total) count
# as equal in the raise-one rule: rounding of equal spectra (the three modes of a symmetric
# field) reaches the fractions as an absolute error near the double unit, so the band is
# 1e-9 relative plus 1e-12 absolute.
TIE_REL = 1e-9
TIE_ABS = 1e-12


class Controller:
    """The add/remove-mode rule of Sec. 2.5, as read here.

    (i)   epsilon > epsilon_th: re-initialise by HOSVD of the current snapshot at the
          current ranks.
    (ii)  If the re-initialised error is still above epsilon_th, raise the ranks to
          those the HOSVD spectrum asks for at gamma_th (never lower), and if that
          changes nothing raise by one the mode with the largest discarded HOSVD
          energy (lowest mode on ties, within 1e-9 relative + 1e-12; other modes follow where the product bound
          r_n <= prod_{m != n} r_m requires it); re-initialise; repeat until epsilon <=
          epsilon_th or every rank is at its cap.
    (iii) Otherwise record epsilon in the slope window.  If some mode captures more
          energy than gamma_th needs (rank_from_core < r_n) and the average error
          slope over the last K steps since the last re-initialisation is negative,
          re-initialise by HOSVD with r_n <- min(r_n, r_n^gamma); if that
          reconstruction exceeds epsilon_th, keep the previous state (revert).
          Either way the window restarts.
    The window excludes steps with a HOSVD re-initialisation (Sec. 2.5) and
    restarts after each one.
    """

    def __init__(self, cfg: ControllerConfig, dims: Sequence[int], w: Sequence[np.ndarray]):
        self.cfg = cfg
        self.dims = list(dims)
        self.w = w
        rm = cfg.rank_max if cfg.rank_max is not None else list(dims)
        self.caps = rank_caps(self.dims, rm)
        self.history: List[float] = []

    def _discarded(self, lam_n: np.ndarray, r_n: int) -> float:
        tot = float(np.sum(np.maximum(lam_n, 0.0)))
        kept = float(np.sum(np.maximum(lam_n[:r_n], 0.0)))
        return 1.0 - kept / tot if tot > 0 else 0.0

    def _raise_one(self, r: List[int], lam) -> Optional[List[int]]:
        """Raise by one the mode below its cap with the largest discarded HOSVD energy
        (lowest mode on ties).  If that breaks r_n <= prod_{m != n} r_m, raise other
        modes the same way until it holds.  None when nothing can grow."""
        def pick(exclude):
            best, best_val = -1, -1.0
            for n in range(len(r)):
                if n in exclude or new[n] >= self.caps[n]:
                    continue
                d = self._discarded(lam[n], new[n])
                # a later mode wins only by more than rounding: fractions within the tie band
                # are equal (modes of a symmetric field), and ties go to the lowest mode
                if best < 0 or d > best_val * (1.0 + TIE_REL) + TIE_ABS:
                    best, best_val = n, d
            return best
        new = list(r)
        n0 = pick(())
        if n0 < 0:
            return None
        new[n0] += 1
        while clamp_product_bound(new) != new:
            m = pick((n0,))
            if m < 0:
                return None
            new[m] += 1
        return new

    def act(self, V: np.ndarray, state: TDBState, eps: float):
        """Apply the rule after a step whose exact error is ``eps``.  Returns
        (state, eps_after, n_reinit, action)."""
        cfg = self.cfg
        if cfg.eps_th <= 0:
            return state, eps, 0, "none"
        K = cfg.slope_window
        if eps > cfg.eps_th:
            r = state.ranks
            T, U, spec = hosvd(V, self.w, r)
            e1 = error_exact(V, T, U, self.w)
            n_re = 1
            action = "reinit"
            while e1 > cfg.eps_th:
                lam = [spec[n][0] for n in range(len(r))]
                new = [min(self.caps[n], max(r[n], rank_from_spectrum(lam[n], cfg.gamma_th)))
                       for n in range(len(r))]
                new = clamp_product_bound(new)
                if new == r:
                    new = self._raise_one(r, lam)
                    if new is None:
                        action = "cap"
                        break
                r = new
                T, U, spec = hosvd(V, self.w, r, spectrum=spec)
                e1 = error_exact(V, T, U, self.w)
                n_re += 1
                action = "increase"
            self.history = []
            return TDBState(T, U), e1, n_re, action

        self.history.append(eps)
        if len(self.history) > K + 1:
            self.history = self.history[-(K + 1):]
        sig = core_singular_values(state.T)
        r = state.ranks
        need = [rank_from_core(sig[n], eps, cfg.gamma_th) for n in range(len(r))]
        if len(self.history) == K + 1 and any(need[n] < r[n] for n in range(len(r))):
            slope = (self.history[-1] - self.history[0]) / K
            if slope < 0:
                self.history = []
                spec = hosvd_spectrum(V, self.w)
                new = [min(r[n], rank_from_spectrum(spec[n][0], cfg.gamma_th)) for n in range(len(r))]
                new = clamp_product_bound(new)
                if new == r:
                    return state, eps, 0, "none"
                T, U, _ = hosvd(V, self.w, new, spectrum=spec)
                e2 = error_exact(V, T, U, self.w)
                if e2 <= cfg.eps_th:
                    return TDBState(T, U), e2, 1, "decrease"
                return state, eps, 1, "revert"
        return state, eps, 0, "none"


def compress_stream(snapshots, w, init_ranks: Sequence[int], ctrl: Optional[ControllerConfig] = None,
                    reorth: bool = True, init_state: Optional[TDBState] = None,
                    exact_every: int = 1):
    """Run the compressor over a sequence of snapshots (Sec. 2.3 and Sec. 2.5).

    snapshots: iterable of arrays V_0, V_1, ...; the first initialises by HOSVD
    (or ``init_state``).  ``init_ranks`` entries of 0 pick the rank from gamma_th.
    Exact error is evaluated every ``exact_every`` steps; the controller acts only
    on those.  Returns (final state, list of StepRecord).
    """
    it = iter(snapshots)
    V0 = next(it)
    dims = list(V0.shape)
    if init_state is None:
        spec = hosvd_spectrum(V0, w)
        rm = ctrl.rank_max if (ctrl is not None and ctrl.rank_max is not None) else dims
        caps = rank_caps(dims, rm)
        r = []
        for n in range(V0.ndim):
            if init_ranks[n] > 0:
                r.append(min(init_ranks[n], caps[n]))
            else:
                r.append(min(caps[n], rank_from_spectrum(spec[n][0], ctrl.gamma_th)))
        r = clamp_product_bound(r)
        T, U, _ = hosvd(V0, w, r, spectrum=spec)
        state = TDBState(T, U)
    else:
        state = init_state
    controller = Controller(ctrl, dims, w) if ctrl is not None else None
    records: List[StepRecord] = []
    V_prev = V0
    for k, V in enumerate(it, start=1):
        T1, U1, _, _ = step_euler(state.T, state.U, w, V_prev, V, reorth=reorth)
        state = TDBState(T1, U1)
        eps = float("nan")
        eps_step = float("nan")
        n_re, action = 0, "none"
        if exact_every > 0 and k % exact_every == 0:
            eps = error_exact(V, state.T, state.U, w)
            eps_step = eps
            if controller is not None:
                state, eps, n_re, action = controller.act(V, state, eps)
        sig = core_singular_values(state.T)
        gam = [gamma_percent(s, eps if eps == eps else 0.0) for s in sig]
        records.append(StepRecord(k, eps, eps_step, state.ranks, n_re, action, gam,
                                  compression_ratio(dims, state.ranks)))
        V_prev = V
    return state, records
