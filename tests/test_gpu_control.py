"""tdb_adapt_rank: the Sec. 2.5 rule through the C-ABI, against the oracle's controller.

The context steps with no error evaluation of its own (error_mode "none"), so every
decision comes from tdb_adapt_rank: the exact error of the state against a snapshot,
then one pass of the rule (Controller.act in the oracle).  FP64 throughout: ranks and
the number of re-initialisations equal the oracle's, epsilon after the rule within
1e-8 relative.  Every third call adapts against the NEXT snapshot instead of the one
just pushed (the rule then usually re-initialises from it); the following push must
difference against that snapshot, as the oracle does.
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_06958_gb300 import synth as S

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


@cuda
def test_adapt_rank_matches_oracle_controller():
    from paper_2201_06958_gb300 import build_lib, tdb
    build_lib.build()
    wl = S.make_workload("reactive", nx=48, ny=40, ns=6)
    w = wl.weights
    K = 5
    eps_th, gamma_th, rmax = 8e-5, 99.9, [8, 8, 6]
    n = 90
    snaps = [wl.snapshot(k, device="cuda", dtype=torch.float64) for k in range(n + 1)]
    V = [S.to_logical(x) for x in snaps]
    ctrl = O.ControllerConfig(eps_th, gamma_th, K, rmax)
    controller = O.Controller(ctrl, wl.dims, w)
    r0 = [4, 4, 3]
    To, Uo, _ = O.hosvd(V[0], w, r0)
    state = O.TDBState(To, Uo)
    c = tdb.TDB(wl.dims, r0, rank_max=rmax, weights=w, eps_th=eps_th, gamma_th=gamma_th, slope_window=K,
                precision="fp64", error_mode="none")
    c.init_from_factors(To, Uo, snaps[0])
    prev = 0
    k = 1
    reinits_o = 0
    acts = []
    while k <= n:
        c.push(snaps[k])
        T1, U1, _, _ = O.step_euler(state.T, state.U, w, V[prev], V[k])
        state = O.TDBState(T1, U1)
        target = k + 1 if (k % 3 == 0 and k < n) else k      # adapt against the next snapshot
        eps = O.error_exact(V[target], state.T, state.U, w)
        state, eps_o, n_re, action = controller.act(V[target], state, eps)
        reinits_o += n_re
        acts.append(action)
        r_g, eps_g = c.adapt_rank(snaps[target])
        assert r_g == state.ranks, (k, target, r_g, state.ranks, action)
        assert abs(eps_g - eps_o) <= 1e-8 * eps_o, (k, eps_g, eps_o)
        reinits_g = c.counters()["reinits"]
        assert reinits_g == reinits_o, (k, reinits_g, reinits_o)
        prev = target
        k = target + 1
    Tg, Ug = c.factors()
    assert np.linalg.norm(O.reconstruct(Tg, Ug) - O.reconstruct(state.T, state.U)) <= \
        1e-9 * np.linalg.norm(O.reconstruct(state.T, state.U))
    assert "reinit" in acts or "increase" in acts, set(acts)
    c.close()
