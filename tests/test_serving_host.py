"""Host logic of the serving layer (no GPU): Poisson arrivals and the
device-memory estimate used for admission."""
import numpy as np

from paper_2307_14837_gb300 import inputs as I
from paper_2307_14837_gb300.serve import Request, memory_estimate, poisson_requests


def test_poisson_arrivals():
    reqs = poisson_requests(4000, rate=50.0, seed=3,
                            make_request=lambda i, u: Request(f"r{i}", None, 0.01, 0.01, 1.0, 1 + int(3 * u)))
    t = np.array([r.arrival for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 1 / 50.0) < 0.05 / 50.0          # mean 1/rate (4000 draws)
    assert abs(np.median(gaps) - np.log(2) / 50.0) < 0.1 / 50.0  # exponential median
    assert {r.n_steps for r in reqs} == {1, 2, 3}
    again = poisson_requests(4000, 50.0, 3, lambda i, u: Request(f"r{i}", None, 0.01, 0.01, 1.0, 1))
    assert [r.arrival for r in again] == list(t)


def test_memory_estimate_grows_with_mesh_and_precision():
    m4, m6 = I.cavity_mesh(4), I.cavity_mesh(6)
    assert memory_estimate(m6, "bf16") > memory_estimate(m4, "bf16")
    assert memory_estimate(m4, "fp64") > memory_estimate(m4, "fp32") > memory_estimate(m4, "bf16")
    assert memory_estimate(m4, "bf16", solve=False) < memory_estimate(m4, "bf16")
    # per-cell cost is roughly constant for larger meshes
    a, b = memory_estimate(I.cavity_mesh(8), "bf16"), memory_estimate(I.cavity_mesh(16), "bf16")
    assert 6 < (b - (1 << 20)) / (a - (1 << 20)) < 10
