"""CPU oracle for the SOAR spilled-IVF hot path.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
fp64 restatement of what the GPU library computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs
may import it.  It shares no code with the CUDA path and imports nothing from
the ``paper_2404_00774_gb300`` package; the only module both sides use is
``synth`` (seeded input generation, no method arithmetic).

Every function here is pinned by ``tests/test_oracle_pins.py`` against facts
the paper or the mathematics fixes (worked example of Figure 3, Theorem 3.1's
closed form, Corollaries 3.1.1-3.1.2, Lemma 3.2, KMR end points, brute-force
exhaustiveness, library routines on tiny inputs).
"""
from .soar_oracle import *  # noqa: F401,F403
from . import probe_mlp  # noqa: F401
