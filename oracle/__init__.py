"""Test oracle for DC N-1 topology evaluation and the MapElites operators.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 CPU restatement of
what the GPU library computes, written from the paper's definitions.  It shares
no code with the CUDA path (it imports only numpy/scipy and the seeded input
generators in ``synth``).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product path never does.

Modules:
  dcflow    -- brute-force post-split loadflow and per-outage re-solve, metrics,
               descriptors and archive cell (Sec. "Fitness function heuristics",
               Sec. "Repertoire design").
  philox    -- Philox4x32-10 counter-based generator (Salmon et al., SC'11).
  mapelites -- mutation (Algorithm 1, action part), sequential archive insert
               (Algorithm 3), MapElites iteration.
  mlp       -- FP64 MLP surrogate forward/backward/Adam.
"""
