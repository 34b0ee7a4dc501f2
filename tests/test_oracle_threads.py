"""The multi-threaded run of the oracle (used only to time it on all host
cores) computes the same step as the single-threaded oracle: particle results
bit for bit, the source up to the order of its FP64 sums."""

import numpy as np

import erpp_inputs as I


def test_threaded_step_equals_single_thread(oracle_lib):
    import oracle
    w = I.CFG_SMALL
    grid, field = I.make_grid(w)
    st = I.make_particles(w, field)
    p = w.params()
    ref = st.copy()
    S_ref = oracle.step(p, grid, ref, first_step=False)
    for nthreads in (1, 3, 4):
        got = st.copy()
        S = oracle.step_threads(p, grid, got, nthreads, first_step=False)
        for name in ("x", "v", "x_prev", "D"):
            assert np.array_equal(getattr(got, name), getattr(ref, name)), (nthreads, name)
        scale = np.abs(S_ref).max()
        assert np.abs(S - S_ref).max() <= 1e-13 * scale, nthreads
