"""The slab partition of one tensor over ranks, on two gloo ranks on the CPU (no GPU).

Split dV along the slowest mode p into contiguous slabs, one per rank.  Every first
contraction is linear in dV, so each rank's partial dS and partial Y_n (n < p) are sums
over its slab, and one all-reduce (sum) of them gives the full dS and Y_n of Eqs.
2.15/2.16; the rows of Y_p are local (rank k owns rows of its slab).  The rest of an
Euler step (Sec. 2.3) then needs two more all-reduces: U_p^T W_p X_p (the complement
projector of Sec. 2.2 on the row-partitioned mode p) and the basis Gram C_p = U_p'^T W_p
U_p' of the Cholesky-QR (reading C4); the core and the bases of modes n < p stay
replicated.  The error (Eq. 2.20) is one scalar all-reduce.  The test runs three such
distributed steps and compares every rank's state with the oracle's single-tensor
Euler steps (1e-12) and the all-reduced error with the oracle's (1e-12).  This checks the
decomposition itself, with real collectives; no multi-GPU build uses it (one GPU per box)."""

import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    rng = np.random.default_rng(77)
    dims, ranks = (11, 9, 8), (3, 3, 2)
    w = [rng.uniform(0.5, 1.5, N) for N in dims]
    w = [x / x.sum() for x in w]
    base = rng.standard_normal(dims)
    drift = rng.standard_normal(dims)
    V = [base + 0.05 * k * drift + 1e-3 * rng.standard_normal(dims) for k in range(4)]
    return dims, ranks, w, V


def _worker(rank, world, port, queue):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import datetime
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    import oracle as O

    def allreduce(x):
        t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
        dist.all_reduce(t)
        return t.numpy()

    dims, ranks, w, V = _case()
    p = len(dims)
    Np = dims[-1]
    lo, hi = Np * rank // world, Np * (rank + 1) // world      # this rank's slab of mode p
    T, U, _ = O.hosvd(V[0], w, list(ranks))                      # the same start on every rank
    Up = U[-1][lo:hi]                                            # local rows of U_p
    Ur = [u.copy() for u in U[:-1]]                              # replicated bases
    out = []
    for k in range(1, len(V)):
        dV = (V[k] - V[k - 1])[..., lo:hi]
        A = [w[n][:, None] * Ur[n] for n in range(p - 1)] + [w[-1][lo:hi, None] * Up]
        # partial first contractions over the slab, then one all-reduce of dS and Y_{n<p}
        dS = O.multi_mode_product(dV, [a.T for a in A])
        Yn = []
        for n in range(p - 1):
            Z = O.multi_mode_product(dV, [A[m].T if m != n else None for m in range(p)])
            Yn.append(O.unfold(Z, n))
        flat = np.concatenate([dS.ravel()] + [y.ravel() for y in Yn])
        flat = allreduce(flat)
        dS = flat[: dS.size].reshape(dS.shape)
        off = dS.size
        for n in range(p - 1):
            Yn[n] = flat[off: off + Yn[n].size].reshape(Yn[n].shape)
            off += Yn[n].size
        Yp = O.unfold(O.multi_mode_product(dV, [a.T for a in A[:-1]] + [None]), p - 1)   # local rows
        # replicated modes: the oracle's right side; mode p: local rows, P_p all-reduced
        dU = [O.basis_rhs(Yn[n], T, Ur[n], w[n], n) for n in range(p - 1)]
        Tp = O.unfold(T, p - 1)
        Xp = np.linalg.solve(Tp @ Tp.T, (Yp @ Tp.T).T).T
        Pp = allreduce(Up.T @ (w[-1][lo:hi, None] * Xp))
        dUp = Xp - Up @ Pp
        T1 = T + dS
        Ur1 = [Ur[n] + dU[n] for n in range(p - 1)]
        Up1 = Up + dUp
        # Cholesky-QR with core compensation: mode p's Gram all-reduced over the row blocks
        for n in range(p - 1):
            C = Ur1[n].T @ (w[n][:, None] * Ur1[n])
            R = np.linalg.cholesky(C).T
            Ur1[n] = np.linalg.solve(R.T, Ur1[n].T).T
            T1 = O.mode_product(T1, R, n)
        C = allreduce(Up1.T @ (w[-1][lo:hi, None] * Up1))
        R = np.linalg.cholesky(C).T
        Up1 = np.linalg.solve(R.T, Up1.T).T
        T1 = O.mode_product(T1, R, p - 1)
        T, Ur, Up = T1, Ur1, Up1
        # error: the slab's part of ||V - T x U||_W^2, then a scalar all-reduce
        rec = O.multi_mode_product(T, Ur + [Up])
        diff = V[k][..., lo:hi] - rec
        wt = w[0][:, None, None] * w[1][None, :, None] * w[2][None, None, lo:hi]
        e2 = float(allreduce(np.array([np.sum(wt * diff * diff)]))[0])
        out.append((T.copy(), [u.copy() for u in Ur], Up.copy(), np.sqrt(e2)))
    queue.put((rank, lo, hi, out))
    dist.destroy_process_group()


def test_slab_split_step_equals_single_tensor_step():
    import oracle as O
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        rank, lo, hi, out = queue.get(timeout=180)
        got[rank] = (lo, hi, out)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    dims, ranks, w, V = _case()
    T, U, _ = O.hosvd(V[0], w, list(ranks))
    for k in range(1, len(V)):
        T, U, _, _ = O.step_euler(T, U, w, V[k - 1], V[k])
        eo = O.error_exact(V[k], T, U, w)
        for rank in (0, 1):
            lo, hi, out = got[rank]
            Tg, Urg, Upg, eg = out[k - 1]
            assert np.abs(Tg - T).max() <= 1e-12 * np.abs(T).max(), (rank, k)
            for n in range(2):
                assert np.abs(Urg[n] - U[n]).max() <= 1e-12 * np.abs(U[n]).max(), (rank, k, n)
            assert np.abs(Upg - U[2][lo:hi]).max() <= 1e-12 * np.abs(U[2]).max(), (rank, k)
            assert abs(eg - eo) <= 1e-12 * eo, (rank, k, eg, eo)
