"""Host logic of the benchmark: the node-update count of the metric is the
oracle's stencil size summed over the particles, and the algorithmic bytes
follow their definition (24 B per node, 208 B per particle)."""

import dataclasses
import os
import sys

import numpy as np

import erpp_inputs as I

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_stencil_node_count_matches_oracle_windows(oracle_lib):
    import bench
    for w in (I.CFG_SMALL, dataclasses.replace(I.CFG_CLUSTERED, n=(48, 40, 36)),
              I.CFG_SMALL.scaled("aniso", (40, 24, 20), 500, L=(6.0, 2.0, 1.5))):
        st = I.make_particles(w, None, n_particles=500)
        lo, hi = oracle_lib.windows(w.params(), st.x)
        expect = int(np.prod((hi - lo + 1).astype(np.int64), axis=0).sum())
        assert bench.stencil_nodes(st.x, w) == expect


def test_algorithmic_bytes():
    import bench
    w = I.CFG_SHEAR
    b = bench.algorithmic_bytes(w, w.n_particles)
    assert b["step"] == 24 * w.n_nodes + 208 * w.n_particles
    assert b["gather"] == b["scatter"] == 12 * w.n_nodes
    assert b["step"] == 1013306368
