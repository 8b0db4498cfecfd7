"""Host logic of the measurement legs, on the CPU: the error measures of
Sec. 6.5-6.6 as the bench computes them, and the whole-step serving stream
(nested meshes only, every step with the solve)."""
import numpy as np

import bench
from paper_2307_14837_gb300 import inputs as I
from paper_2307_14837_gb300.train import velocity_errors


def test_velocity_errors_closed_form():
    ref = [np.full((5, 3), 2.0), np.full((5, 3), 4.0)]
    vel = [r + 1.0 for r in ref]                       # error 1 at every entry
    e = velocity_errors(vel, ref)
    n_err = np.sqrt(15.0)
    assert np.allclose(e["e_v"], [n_err / np.sqrt(60.0), n_err / np.sqrt(240.0)], rtol=1e-15)
    # time-integrated: (sum of squared errors / sum of squared norms)^(1/2)
    assert abs(e["E_v"] - np.sqrt(30.0 / 300.0)) < 1e-15
    assert velocity_errors(ref, ref)["E_v"] == 0.0


def test_whole_step_serving_stream_uses_nested_meshes():
    reqs = bench.serving_requests_solve(n=6, seed=3)
    assert len(reqs) == 6 and all(r.solve for r in reqs)
    assert all(r.x0 is None for r in reqs)             # from rest with the Dirichlet data
    arrivals = [r.arrival for r in reqs]
    assert arrivals == sorted(arrivals) and arrivals[0] > 0
    for r in reqs:
        nc = len(r.mesh["cells"])
        assert 4000 <= nc <= 140000
        assert 10 <= r.n_steps <= 40
        lv = r.mesh["meta"]["mg_levels"]
        assert lv >= 2                                 # a hierarchy for the multigrid solve
        # cells come in groups of 8 children: the first level is nested
        assert nc % 8 == 0
