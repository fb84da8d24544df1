"""Batched members (the 64-tensor configuration's generator) against the oracle.

Four members of the batch, one of them with N_1 not a multiple of 4 (zero-padded copies
on the tensor-core path), are stepped together through the batch graph (every member's
step recorded into one graph over several streams) for 12 steps at fixed ranks; each
member's error and reconstruction track the FP64 oracle's Euler steps on the same float32
snapshots within the BF16 bounds of the single-tensor tests (epsilon 2e-2 relative,
T x U 5e-4)."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_06958_gb300 import synth as S

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@cuda
def test_batch_members_track_oracle():
    from paper_2201_06958_gb300 import build_lib, tdb
    build_lib.build()
    members = S.make_batch(seed=1005, count=64)
    pick = [m for m in members if m.dims[0] % 4 != 0][:1] + [m for m in members if m.dims[0] % 4 == 0][:3]
    steps = 12
    ctxs, slots, snaps, states = [], [], [], []
    for wl in pick:
        sn = [wl.snapshot(k, device="cuda") for k in range(steps + 1)]
        snaps.append(sn)
        V0 = S.to_logical(sn[0])
        T, U, _ = O.hosvd(V0, wl.weights, wl.rank)
        states.append((T, U, V0))
        c = tdb.TDB(wl.dims, wl.rank, weights=wl.weights, precision="bf16", error_mode="exact")
        sl = [torch.empty_like(sn[0]), sn[0].clone()]
        c.init_from_factors(T, U, sl[1]).set_input_slots(sl[0], sl[1])
        ctxs.append(c)
        slots.append(sl)
    batch = tdb.Batch(ctxs, nstreams=4)
    worst = 0.0
    for k in range(1, steps + 1):
        par = (k - 1) % 2
        for sl, sn in zip(slots, snaps):
            sl[par].copy_(sn[k])
        infos = batch.push(par)
        for i, (wl, info) in enumerate(zip(pick, infos)):
            T, U, Vp = states[i]
            Vk = S.to_logical(snaps[i][k])
            T, U, _, _ = O.step_euler(T, U, wl.weights, Vp, Vk)
            states[i] = (T, U, Vk)
            eo = O.error_exact(Vk, T, U, wl.weights)
            worst = max(worst, abs(info["eps"] - eo) / eo)
    for c, (T, U, _) in zip(ctxs, states):
        Tg, Ug = c.factors()
        assert rel(O.reconstruct(Tg, Ug), O.reconstruct(T, U)) <= 5e-4
    assert worst <= 2e-2, worst
    assert batch.counters()["graph_replays"] >= steps - 2
    batch.close()
    for c in ctxs:
        c.close()
