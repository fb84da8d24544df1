"""FP64 CPU oracle of the time-dependent-basis (TDB) in-situ compressor
(Zamani Ashtiani, Malik and Babaee, "Scalable in situ compression of transient
simulation data using time-dependent bases").

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package. The product path (the CUDA library and its Python
binding) never imports it, and this package imports nothing from the product.

Every function is a plain, slow restatement of a passage of the paper, written
with numpy in float64. Library primitives (tensordot, matmul, eigh, cholesky)
serve as single steps; nothing is blocked, fused or reordered beyond the
equation it restates.
"""

from .tdb_oracle import *  # noqa: F401,F403
from . import mlp_oracle  # noqa: F401
