"""Seeded synthetic snapshot streams shaped like the paper's four workloads.

This module holds field formulas and quadrature weights only; it contains none
of the compressor's arithmetic and is shared by the tests, the oracle runs and
the benchmark (it is the one module both sides may use).  The paper's datasets
(reactive-flow DNS, the 16 stochastic DNS runs, the DNSLab channel) are not
available, so each workload is a closed-form stand-in with the paper's shape,
weights and kind of structure:

* ``analytic``   - 64^3 sum of four separable sin/cos terms with moving phases and
                   amplitudes; multilinear rank exactly (4,4,4) (stands in for
                   the Runge example of Sec. 3.1 as an exact-rank test field).
* ``reactive``   - 512 x 256 grid x 12 species: two advecting, rotating flame
                   fronts with Arrhenius-like species profiles (Sec. 3.2).
* ``stochastic`` - 256 x 128 grid x 512 samples: mean plus a 16-term
                   Karhunen-Loeve expansion with Gaussian coefficients (Sec. 3.3,
                   with Monte-Carlo weights 1/s).
* ``channel``    - 192 x 129 x 192 x 3 velocity components: mean profile plus
                   random Fourier-mode fluctuations on a tanh-clustered
                   wall-normal grid (Sec. 3.4).
* ``batch``      - 64 independent 3-mode tensors of uneven sizes.
* ``runge``      - the time-dependent Runge function of Sec. 3.1 itself (closed form,
                   126^3, Delta t = 5e-3): the ranks must rise towards t = 1 and fall after.

Storage order: a snapshot of logical shape (N_1, ..., N_p) is a C-contiguous
torch tensor of shape (N_p, ..., N_1), i.e. column-major with mode 1 fastest.
``to_logical`` gives the numpy view with logical index order.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np
import torch

__all__ = ["Workload", "make_workload", "to_logical", "from_logical", "trapezoid_unit",
           "uniform_unit", "WORKLOADS"]


def trapezoid_unit(n: int) -> np.ndarray:
    """Trapezoid weights of n equispaced nodes on [0, 1]; they sum to 1."""
    h = 1.0 / (n - 1)
    w = np.full(n, h)
    w[0] = w[-1] = 0.5 * h
    return w


def trapezoid_nodes(y: np.ndarray) -> np.ndarray:
    """Trapezoid weights on arbitrary sorted nodes, scaled to sum to 1."""
    w = np.zeros_like(y)
    d = np.diff(y)
    w[:-1] += 0.5 * d
    w[1:] += 0.5 * d
    return w / w.sum()


def uniform_unit(n: int) -> np.ndarray:
    """n equal weights summing to 1 (periodic grid or Monte-Carlo samples)."""
    return np.full(n, 1.0 / n)


def to_logical(x: torch.Tensor) -> np.ndarray:
    """Storage-order tensor (N_p, ..., N_1) -> float64 numpy array indexed [i_1, ..., i_p]."""
    a = x.detach().to("cpu", torch.float64).numpy()
    return np.ascontiguousarray(np.transpose(a, tuple(range(a.ndim - 1, -1, -1))))


def from_logical(a: np.ndarray, dtype=torch.float64, device="cpu") -> torch.Tensor:
    """Inverse of :func:`to_logical`."""
    t = np.ascontiguousarray(np.transpose(a, tuple(range(a.ndim - 1, -1, -1))))
    return torch.from_numpy(t).to(device=device, dtype=dtype)


@dataclasses.dataclass
class Workload:
    name: str
    dims: List[int]                  # logical (N_1, ..., N_p)
    dtype: str                       # "f64" or "f32": snapshot element type
    dt: float
    steps: int
    rank: List[int]                  # initial ranks (0 = from gamma_th)
    rank_max: List[int]
    eps_th: float
    gamma_th: float
    weights: List[np.ndarray]
    _field: Callable = dataclasses.field(repr=False, default=None)
    _dfield: Optional[Callable] = dataclasses.field(repr=False, default=None)

    @property
    def ndim(self) -> int:
        return len(self.dims)

    @property
    def numel(self) -> int:
        return int(np.prod(self.dims))

    @property
    def torch_dtype(self):
        return torch.float64 if self.dtype == "f64" else torch.float32

    def snapshot(self, k: int, device="cpu", dtype=None) -> torch.Tensor:
        """Snapshot at step k (time k*dt), storage order, computed in float64 on
        ``device`` then cast to ``dtype`` (default: the workload's dtype)."""
        dtype = dtype or self.torch_dtype
        with torch.no_grad():
            v = self._field(k * self.dt, torch.device(device))
        return v.to(dtype).contiguous()

    def snapshot_dot(self, t: float, device="cpu") -> torch.Tensor:
        """Exact time derivative at time t (float64), where the field has one."""
        if self._dfield is None:
            raise ValueError(f"workload {self.name} has no analytic derivative")
        with torch.no_grad():
            return self._dfield(t, torch.device(device)).contiguous()

    def logical(self, k: int) -> np.ndarray:
        return to_logical(self.snapshot(k, dtype=torch.float64 if self.dtype == "f64" else torch.float32))


def _axis(vals: np.ndarray, mode: int, p: int, device) -> torch.Tensor:
    """Coordinate vector of mode ``mode`` shaped to broadcast in storage order."""
    shape = [1] * p
    shape[p - 1 - mode] = len(vals)
    return torch.as_tensor(vals, dtype=torch.float64, device=device).reshape(shape)


# ---------------------------------------------------------------------------
# analytic: exact multilinear rank 4 (64^3, FP64)
# ---------------------------------------------------------------------------

def _analytic(seed: int, n: int = 64, dt: float = 1e-3, steps: int = 200) -> Workload:
    rng = np.random.default_rng(seed)
    J = 4
    k = [rng.permutation(np.arange(1, J + 1)) for _ in range(3)]   # distinct integer wavenumbers per mode
    omega = rng.uniform(0.5, 2.0, size=J)
    c = rng.uniform(-5.0, 5.0, size=(J, 3))
    psi = rng.uniform(0.0, 2 * np.pi, size=(J, 3))
    base = np.array([2.0, 1.6, 1.3, 1.0])
    x = 2 * np.pi * np.arange(n) / n
    kinds = ("sin", "cos", "sin")

    def parts(t, device, deriv):
        # 1-D factors per term and mode (numpy), then one outer-product sum in storage order (i3, i2, i1)
        f = np.empty((3, J, n))
        df = np.empty((3, J, n))
        for m in range(3):
            arg = np.asarray(k[m], dtype=np.float64)[:, None] * x[None, :] + (c[:, m] * t + psi[:, m])[:, None]
            if kinds[m] == "sin":
                f[m], df[m] = np.sin(arg), c[:, m, None] * np.cos(arg)
            else:
                f[m], df[m] = np.cos(arg), -c[:, m, None] * np.sin(arg)
        a = base * (1.0 + 0.5 * np.sin(omega * t))          # >= 0.5, distinct sizes
        G = np.einsum("jc,jb->jcb", f[2], f[1])
        if not deriv:
            out = np.einsum("jcb,ja->cba", a[:, None, None] * G, f[0])
        else:
            da = base * 0.5 * omega * np.cos(omega * t)
            dG = np.einsum("jc,jb->jcb", df[2], f[1]) + np.einsum("jc,jb->jcb", f[2], df[1])
            out = (np.einsum("jcb,ja->cba", da[:, None, None] * G + a[:, None, None] * dG, f[0])
                   + np.einsum("jcb,ja->cba", a[:, None, None] * G, df[0]))
        return torch.from_numpy(np.ascontiguousarray(out)).to(device)

    w = [uniform_unit(n) for _ in range(3)]
    return Workload("analytic", [n, n, n], "f64", dt, steps, [4, 4, 4], [4, 4, 4], 0.0, 99.999, w,
                    lambda t, d: parts(t, d, False), lambda t, d: parts(t, d, True))


# ---------------------------------------------------------------------------
# runge: the time-dependent Runge function of Sec. 3.1 (FP64)
# ---------------------------------------------------------------------------

def _runge(seed: int, n: int = 126, dt: float = 5e-3, steps: int = 400, eps_th: float = 1e-4,
           gamma_th: float = 99.99999, rank_max: int = 8) -> Workload:
    """f(x, t) = 1 / (a(t)^2 + x_1^2 + x_2^2 + x_3^2) on [-pi, pi]^3 (uniform n^3 grid),
    a(t) = 1 - 0.5 exp(-0.5 (t - 1)^2): the peak sharpens towards t = 1 and relaxes
    after, so the ranks that keep the error below eps_th rise and fall again.  t runs
    over [0, steps * dt] (the default covers [0, 2]).  Deterministic: ``seed`` is unused.

    Thresholds: with the weights summing to one per mode the error is an RMS of the
    field (whose weighted norm is ~0.2), so the paper's 1e-6 (stated for its own, unstated
    scaling) would ask for ranks beyond 8 at every t; eps_th = 1e-4 with gamma_th =
    99.99999 % (the energy fraction that leaves an RMS tail of about eps_th) gives the
    rise from (5, 5, 5) to (6, 6, 5) towards t = 1 and the fall back after."""
    del seed
    x = np.linspace(-math.pi, math.pi, n)
    x2 = torch.from_numpy(x * x)

    def a_of(t):
        return 1.0 - 0.5 * math.exp(-0.5 * (t - 1.0) ** 2)

    def field(t, device, deriv=False):
        q = x2.to(device)
        r2 = q[:, None, None] + q[None, :, None] + q[None, None, :]      # storage order (i3, i2, i1): symmetric
        a = a_of(t)
        den = a * a + r2
        if not deriv:
            return 1.0 / den
        da = 0.5 * (t - 1.0) * math.exp(-0.5 * (t - 1.0) ** 2)
        return -2.0 * a * da / (den * den)

    w = [trapezoid_unit(n) for _ in range(3)]
    return Workload("runge", [n, n, n], "f64", dt, steps, [0, 0, 0], [rank_max] * 3, eps_th, gamma_th, w,
                    lambda t, d: field(t, d), lambda t, d: field(t, d, True))


# ---------------------------------------------------------------------------
# reactive: 2-D reactive-flow-like, 512 x 256 x 12 species (FP32)
# ---------------------------------------------------------------------------

def _reactive(seed: int, nx: int = 512, ny: int = 256, ns: int = 12, dt: float = 1e-3,
              steps: int = 1000) -> Workload:
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 1.0, nx)
    y = np.linspace(0.0, 1.0, ny)
    fronts = []
    for f in range(2):
        fronts.append(dict(
            theta0=rng.uniform(-0.15, 0.15) + 0.5 * np.pi * f,      # one front near-vertical, one near-horizontal
            omega=rng.uniform(-1.0, 1.0),                           # rotation rate (rad per unit time)
            c0=rng.uniform(0.3, 0.7, size=2),
            u=rng.uniform(-0.5, 0.5, size=2),                       # advection velocity
            amp_w=rng.uniform(0.01, 0.03),                          # wrinkle amplitude
            k_w=rng.uniform(1.0, 2.0),                              # wrinkle wavenumber (cycles per unit length)
            om_w=rng.uniform(3.0, 8.0),
            delta_T=rng.uniform(0.06, 0.1),
        ))
    A = rng.uniform(0.005, 0.03, size=ns)          # species scale: ||V||_W ~ 0.02
    xi_s = rng.uniform(-0.05, 0.05, size=ns)
    d_s = rng.uniform(0.06, 0.15, size=ns)
    E_s = rng.uniform(0.5, 4.0, size=ns)

    def field(t, device):
        X = _axis(x, 0, 3, device)
        Y = _axis(y, 1, 3, device)
        S = torch.arange(ns, device=device, dtype=torch.float64).reshape(ns, 1, 1)
        out = torch.zeros((ns, ny, nx), dtype=torch.float64, device=device)
        As = torch.as_tensor(A, device=device).reshape(ns, 1, 1)
        xs = torch.as_tensor(xi_s, device=device).reshape(ns, 1, 1)
        ds = torch.as_tensor(d_s, device=device).reshape(ns, 1, 1)
        Es = torch.as_tensor(E_s, device=device).reshape(ns, 1, 1)
        del S
        for fr in fronts:
            th = fr["theta0"] + fr["omega"] * t
            cx = fr["c0"][0] + fr["u"][0] * t
            cy = fr["c0"][1] + fr["u"][1] * t
            s_tan = -(X - cx) * math.sin(th) + (Y - cy) * math.cos(th)
            xi = (X - cx) * math.cos(th) + (Y - cy) * math.sin(th)
            xi = xi + fr["amp_w"] * torch.sin(2 * math.pi * fr["k_w"] * s_tan + fr["om_w"] * t)
            prog = 0.5 * (1.0 + torch.tanh(xi / fr["delta_T"]))      # 0 unburnt .. 1 burnt
            temp = 1.0 + 3.0 * prog
            out = out + As * torch.exp(-((xi - xs) / ds) ** 2) * torch.exp(-Es / temp)
        return out

    w = [trapezoid_unit(nx), trapezoid_unit(ny), np.ones(ns)]
    return Workload("reactive", [nx, ny, ns], "f32", dt, steps, [0, 0, 0], [16, 16, 12], 1e-4, 99.999, w,
                    field)


# ---------------------------------------------------------------------------
# stochastic: 256 x 128 grid x 512 Monte-Carlo samples (FP32)
# ---------------------------------------------------------------------------

def _stochastic(seed: int, nx: int = 256, ny: int = 128, ns: int = 512, dt: float = 1e-3,
                steps: int = 500, nkl: int = 16) -> Workload:
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 1.0, nx)
    y = np.linspace(0.0, 1.0, ny)
    lam = np.exp(-np.arange(1, nkl + 1) / 3.0)
    xi = rng.standard_normal((ns, nkl))                  # Gaussian KL coefficients, one row per sample
    a_k = rng.integers(0, 4, size=nkl)
    b_k = rng.integers(0, 4, size=nkl)
    psi = rng.uniform(0, 2 * np.pi, size=nkl)
    c_k = rng.uniform(0.1, 0.4, size=nkl)                 # advection speed of each mode's envelope
    x0 = rng.uniform(0.2, 0.5, size=nkl)
    ell = rng.uniform(0.25, 0.4, size=nkl)

    def field(t, device):
        X = _axis(x, 0, 3, device)
        Y = _axis(y, 1, 3, device)
        mean = 1.0 + 0.5 * torch.sin(2 * math.pi * (X - 0.3 * t)) * torch.cos(math.pi * Y)
        out = mean.expand(ns, ny, nx).clone()
        coef = torch.as_tensor(xi * np.sqrt(lam)[None, :], device=device)      # ns x nkl
        for k in range(nkl):
            env = torch.exp(-((X - x0[k] - c_k[k] * t) / ell[k]) ** 2)
            phi = env * torch.cos(2 * math.pi * (a_k[k] * X + b_k[k] * Y) + psi[k] + 2.0 * t)
            out = out + coef[:, k].reshape(ns, 1, 1) * phi
        return out

    w = [trapezoid_unit(nx), trapezoid_unit(ny), uniform_unit(ns)]
    return Workload("stochastic", [nx, ny, ns], "f32", dt, steps, [0, 0, 0], [20, 20, 20], 1e-3, 99.999, w,
                    field)


# ---------------------------------------------------------------------------
# channel: 192 x 129 x 192 x 3 (FP32)
# ---------------------------------------------------------------------------

def _channel(seed: int, nx: int = 192, ny: int = 129, nz: int = 192, nc: int = 3, dt: float = 1e-3,
             steps: int = 300, nmodes: int = 24) -> Workload:
    rng = np.random.default_rng(seed)
    beta = 2.0
    j = np.arange(ny)
    yy = np.tanh(beta * (2.0 * j / (ny - 1) - 1.0)) / np.tanh(beta)
    xx = np.pi * np.arange(nx) / nx              # streamwise length pi, periodic
    zz = 2 * np.pi * np.arange(nz) / nz          # spanwise length 2 pi, periodic
    alpha = 2.0 * rng.integers(1, 7, size=nmodes)        # streamwise wavenumbers (periodic on [0, pi))
    betaz = rng.integers(1, 9, size=nmodes).astype(float)
    amp = (alpha ** 2 + betaz ** 2) ** (-5.0 / 6.0)
    amp = 0.3 * amp / amp.max()
    ny_shape = rng.integers(1, 4, size=nmodes)
    psi = rng.uniform(0, 2 * np.pi, size=(nmodes, nc))
    comp = rng.uniform(0.3, 1.0, size=(nmodes, nc))
    om = rng.uniform(0.5, 2.0, size=nmodes)
    uc = 0.8

    def field(t, device):
        X = _axis(xx, 0, 4, device)
        Y = _axis(yy, 1, 4, device)
        Z = _axis(zz, 2, 4, device)
        out = torch.zeros((nc, nz, ny, nx), dtype=torch.float64, device=device)
        wall = (1.0 - Y * Y)
        for m in range(nmodes):
            prof = wall * torch.cos(0.5 * math.pi * ny_shape[m] * Y)
            a_t = 1.0 + 0.3 * math.sin(om[m] * t)
            for c in range(nc):
                wave = torch.cos(alpha[m] * (X - uc * t) + betaz[m] * Z + psi[m, c] + 0.5 * om[m] * t)
                out[c] += (amp[m] * comp[m, c] * a_t) * (prof * wave)[0]
        mean = 1.1 * (1.0 - Y.abs() ** 7)
        out[0] += mean[0]
        return out

    w = [uniform_unit(nx), trapezoid_nodes(yy), uniform_unit(nz), np.ones(nc)]
    return Workload("channel", [nx, ny, nz, nc], "f32", dt, steps, [0, 0, 0, 0], [30, 30, 30, 3], 3.3e-3,
                    99.999, w, field)


# ---------------------------------------------------------------------------
# batch: 64 uneven 3-mode tensors (FP32)
# ---------------------------------------------------------------------------

def _batch_member(seed: int, dims: Sequence[int], rank: Sequence[int], dt: float = 1e-3,
                  steps: int = 200, noise: float = 1e-3) -> Workload:
    rng = np.random.default_rng(seed)
    nterm = 6
    coords = [np.linspace(0.0, 1.0, d) for d in dims]
    kk = rng.integers(1, 4, size=(nterm, 3))
    ph = rng.uniform(0, 2 * np.pi, size=(nterm, 3))
    vel = rng.uniform(-1.0, 1.0, size=(nterm, 3))
    amp = rng.uniform(0.2, 1.0, size=nterm) * np.exp(-np.arange(nterm) / 2.0)
    noise_seed = int(rng.integers(0, 2 ** 31 - 1))

    def field(t, device):
        out = 0.0
        for q in range(nterm):
            term = amp[q]
            for m in range(3):
                C = _axis(coords[m], m, 3, device)
                term = term * torch.cos(2 * math.pi * kk[q, m] * C + ph[q, m] + vel[q, m] * t)
            out = out + term
        g = torch.Generator(device="cpu").manual_seed(noise_seed + int(round(t / dt)))
        nz = torch.randn(tuple(reversed(dims)), generator=g, dtype=torch.float64)
        return out + noise * nz.to(device)

    w = [uniform_unit(d) for d in dims]
    return Workload(f"batch{seed}", list(dims), "f32", dt, steps, list(rank), list(rank), 0.0, 99.999, w,
                    field)


def make_batch(seed: int = 1005, count: int = 64):
    """The 64-tensor batch: sizes U{32..128} per mode, ranks U{4..24} capped at the sizes."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        dims = [int(v) for v in rng.integers(32, 129, size=3)]
        r = int(rng.integers(4, 25))
        ranks = [min(r, d) for d in dims]
        out.append(_batch_member(seed * 1000 + i, dims, ranks))
    return out


# ---------------------------------------------------------------------------
# grouped modes (p < d): contiguous groups of grid dimensions as one mode
# ---------------------------------------------------------------------------

def group_modes(wl: Workload, groups: Sequence[Sequence[int]], rank_max: Optional[Sequence[int]] = None,
                name: Optional[str] = None) -> Workload:
    """The same snapshots with each group of consecutive modes taken as one mode (the
    disjoint decomposition of the independent variables into p groups of Sec. 2.1; the
    two-dimensional spatial bases of the TDB-2 scheme of Sec. 3.2).  With mode 1 fastest, a
    group (m, ..., m + g - 1) has the linear index i_m + N_m i_{m+1} + ..., so the storage
    tensor is only reshaped, and the group's quadrature weights are the products of its
    members' weights in that index order (the product rule of the group's grid)."""
    flat = [m for g in groups for m in g]
    if flat != list(range(wl.ndim)) or any(list(g) != list(range(g[0], g[0] + len(g))) for g in groups):
        raise ValueError("groups must be consecutive runs covering the modes in order")
    dims, weights = [], []
    for g in groups:
        n, w = 1, np.ones(1)
        for m in g:
            n *= wl.dims[m]
            w = np.kron(wl.weights[m], w)          # the later mode varies slower
        dims.append(n)
        weights.append(w)
    store = tuple(reversed(dims))
    if rank_max is None:
        rank_max = [min(32, n) for n in dims]

    def field(t, device):
        return wl._field(t, device).reshape(store)

    dfield = None
    if wl._dfield is not None:
        def dfield(t, device):
            return wl._dfield(t, device).reshape(store)

    return Workload(name or wl.name + "_grouped", dims, wl.dtype, wl.dt, wl.steps, [0] * len(dims),
                    list(rank_max), wl.eps_th, wl.gamma_th, weights, field, dfield)


def _reactive_dbo(seed: int, nx: int = 32, ny: int = 16, ns: int = 12, **kw) -> Workload:
    """The reactive flow as the TDB-2 (DBO) scheme of Sec. 3.2: one two-dimensional spatial
    mode (nx * ny points, product trapezoid weights) and the species mode."""
    return group_modes(_reactive(seed, nx=nx, ny=ny, ns=ns, **kw), [[0, 1], [2]], rank_max=[12, 12],
                       name="reactive_dbo")


def _reactive_tdb2(seed: int, nx: int = 251, ny: int = 76, ns: int = 23, **kw) -> Workload:
    """TDB-2 at the size of Sec. 3.2: the reactive recipe on a 251 x 76 grid with 23 species,
    the grid taken as one 19,076-point spatial mode beside the species mode."""
    return group_modes(_reactive(seed, nx=nx, ny=ny, ns=ns, **kw), [[0, 1], [2]], rank_max=[23, 23],
                       name="reactive_tdb2")


WORKLOADS = {
    "analytic": lambda seed=1001, **kw: _analytic(seed, **kw),
    "reactive": lambda seed=1002, **kw: _reactive(seed, **kw),
    "stochastic": lambda seed=1003, **kw: _stochastic(seed, **kw),
    "channel": lambda seed=1004, **kw: _channel(seed, **kw),
    "runge": lambda seed=1005, **kw: _runge(seed, **kw),
    "reactive_dbo": lambda seed=1006, **kw: _reactive_dbo(seed, **kw),
    "reactive_tdb2": lambda seed=1007, **kw: _reactive_tdb2(seed, **kw),
}


DEFAULT_SEEDS = {"analytic": 1001, "reactive": 1002, "stochastic": 1003, "channel": 1004, "runge": 1005,
                 "reactive_dbo": 1006, "reactive_tdb2": 1007}


def default_seed(name: str) -> int:
    """The seed a workload uses when none is given (1000 + its index)."""
    return DEFAULT_SEEDS[name]


def make_workload(name: str, seed: Optional[int] = None, **kw) -> Workload:
    """Build a workload by name; ``seed`` defaults to 1000 + its index."""
    f = WORKLOADS[name]
    return f(**kw) if seed is None else f(seed, **kw)
