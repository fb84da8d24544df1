"""Recorded steps and batches give the results of plain pushes, bit for bit.

tdb_push_slot records a step's device work as a CUDA graph (once per slot parity and
rank configuration) and replays it; a batch records every member's step into one
graph over several streams.  Neither changes what a step computes, so the step records
and the final factors must equal those of tdb_push_snapshot on the same snapshots,
including across control actions (re-initialisations and rank changes re-record).
tdb_push_snapshot records a step once its (V_{k+1}, V_k, V_{k-1}) pointer tuple recurs, as a
ring of input buffers makes it do; its results equal those of pushes that never recur."""

import numpy as np
import pytest
import torch

from paper_2201_06958_gb300 import synth as S

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")

KEYS = ("eps", "eps_exact", "eps_step", "ranks", "reinit", "action", "dv_norm", "gamma", "sigma_min")


@pytest.fixture(scope="module")
def tdbmod():
    from paper_2201_06958_gb300 import build_lib, tdb
    build_lib.build()
    return tdb


def same_info(a, b):
    for k in KEYS:
        va, vb = a[k], b[k]
        if isinstance(va, float) and np.isnan(va):
            assert np.isnan(vb), k
        else:
            assert va == vb, (k, va, vb)


def same_factors(A, B):
    Ta, Ua = A.factors()
    Tb, Ub = B.factors()
    assert np.array_equal(Ta, Tb)
    assert all(np.array_equal(x, y) for x, y in zip(Ua, Ub))


@cuda
@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_slot_graph_steps_equal_pointer_pushes(tdbmod, precision):
    wl = S.make_workload("reactive")
    steps = 80
    snaps = [wl.snapshot(k, device="cuda") for k in range(steps + 1)]
    kw = dict(rank_max=wl.rank_max, weights=wl.weights, eps_th=8e-5, gamma_th=99.9, slope_window=5,
              precision=precision, error_mode="exact")
    A = tdbmod.TDB(wl.dims, wl.rank, **kw).init(snaps[0])
    B = tdbmod.TDB(wl.dims, wl.rank, **kw)
    slots = [torch.empty_like(snaps[0]), torch.empty_like(snaps[0])]
    slots[1].copy_(snaps[0])
    B.init(slots[1]).set_input_slots(slots[0], slots[1])
    actions = set()
    for k in range(1, steps + 1):
        parity = (k - 1) % 2
        slots[parity].copy_(snaps[k])
        ib = B.push_slot(parity)
        ia = A.push(snaps[k])
        same_info(ia, ib)
        actions.add(ia["action"])
    same_factors(A, B)
    assert actions - {"none"}, "the run should include a control action (re-recording the step)"
    c = B.counters()
    # every step after the first (which prepares the tensor-core weights) is a replay
    assert c["graph_replays"] >= steps - 1 and 2 <= c["graph_records"] < steps // 2, c


@cuda
def test_batch_equals_members_stepped_alone(tdbmod):
    members = S.make_batch(count=6)
    steps = 24
    A, B, snaps, slots = [], [], [], []
    for wl in members:
        prec = "bf16" if wl.dims[0] % 4 == 0 else "fp32"
        kw = dict(rank_max=wl.rank_max, weights=wl.weights, precision=prec, error_mode="every_k", error_every=5)
        sn = [wl.snapshot(k, device="cuda").to(torch.float32).contiguous() for k in range(steps + 1)]
        sl = [torch.empty_like(sn[0]), torch.empty_like(sn[0])]
        sl[1].copy_(sn[0])
        A.append(tdbmod.TDB(wl.dims, wl.rank, **kw).init(sn[0]))
        B.append(tdbmod.TDB(wl.dims, wl.rank, **kw).init(sl[1]).set_input_slots(sl[0], sl[1]))
        snaps.append(sn)
        slots.append(sl)
    batch = tdbmod.Batch(B, nstreams=3)
    for k in range(1, steps + 1):
        parity = (k - 1) % 2
        for i in range(len(members)):
            slots[i][parity].copy_(snaps[i][k])
        infos = batch.push(parity)
        for i in range(len(members)):
            same_info(A[i].push(snaps[i][k]), infos[i])
    for a, b in zip(A, B):
        same_factors(a, b)
    c = batch.counters()
    assert c["graph_replays"] >= steps - 1 and c["graph_records"] <= 3, c
    batch.close()


@cuda
def test_profiling_eager_and_recorded(tdbmod):
    """The per-phase timers work on plain pushes (eager events) and on recorded steps
    (external event-record nodes in the step graph), change no result, and the projection
    kernel's span (device global timer) is positive and below its event time."""
    wl = S.make_workload("reactive", nx=128, ny=64, ns=8)
    snaps = [wl.snapshot(k, device="cuda") for k in range(13)]
    kw = dict(rank_max=[6, 6, 4], weights=wl.weights, eps_th=0.0, precision="bf16", error_mode="exact")
    A = tdbmod.TDB(wl.dims, [6, 6, 4], **kw).init(snaps[0])
    B = tdbmod.TDB(wl.dims, [6, 6, 4], **kw)
    slots = [torch.empty_like(snaps[0]), torch.empty_like(snaps[0])]
    slots[1].copy_(snaps[0])
    B.init(slots[1])
    B.set_input_slots(slots[0], slots[1])
    for k in range(1, 4):
        A.push(snaps[k])
        slots[(k - 1) % 2].copy_(snaps[k])
        B.push_slot((k - 1) % 2)
    A.set_profiling(True)
    B.set_profiling(True)
    for k in range(4, 13):
        ia = A.push(snaps[k])
        slots[(k - 1) % 2].copy_(snaps[k])
        ib = B.push_slot((k - 1) % 2)
        same_info(ia, ib)
    for c, recorded in ((A, False), (B, True)):
        pr = c.profile()
        assert pr["steps"] == 9, pr
        for key in ("ms_project", "ms_project_main", "ms_update", "ms_error"):
            assert pr[key] > 0.0, (recorded, key, pr)
        assert pr["spans"] == 9, pr
        assert 0.0 < pr["us_project_span"] < pr["ms_project_main"] * 1e3, pr
    assert B.counters()["graph_replays"] >= 9
    same_factors(A, B)


@cuda
@pytest.mark.parametrize("precision,integrator,ring", [("bf16", "euler", 3), ("fp32", "euler", 3),
                                                       ("fp32", "rk2_central", 4)])
def test_pointer_ring_graph_steps_equal_unrecorded_pushes(tdbmod, precision, integrator, ring):
    wl = S.make_workload("reactive")
    steps = 60
    snaps = [wl.snapshot(k, device="cuda") for k in range(steps + 1)]
    kw = dict(rank_max=wl.rank_max, weights=wl.weights, eps_th=8e-5, gamma_th=99.9, slope_window=5,
              precision=precision, error_mode="exact", integrator=integrator)
    A = tdbmod.TDB(wl.dims, wl.rank, **kw).init(snaps[0])
    bufs = [torch.empty_like(snaps[0]) for _ in range(ring)]
    bufs[0].copy_(snaps[0])
    B = tdbmod.TDB(wl.dims, wl.rank, **kw).init(bufs[0])
    actions = set()
    for k in range(1, steps + 1):
        bufs[k % ring].copy_(snaps[k])
        ib = B.push(bufs[k % ring])
        ia = A.push(snaps[k])
        same_info(ia, ib)
        actions.add(ia["action"])
    same_factors(A, B)
    assert actions - {"none"}, "the run should include a control action (re-recording the step)"
    assert A.counters()["graph_replays"] == 0, A.counters()
    c = B.counters()
    assert c["graph_replays"] >= steps - 3 * ring and ring <= c["graph_records"] < steps // 2, c
