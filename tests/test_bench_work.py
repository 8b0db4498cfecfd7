"""The bench's work model for the element stages: the share of
parallelepiped cells (whose Jacobian is formed once per fine cell) on
meshes where it is known, and the element work it implies."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2307_14837_gb300 import inputs as I  # noqa: E402


def test_parallelepiped_share_known_meshes():
    assert bench.parallelepiped_fraction(I.cavity_mesh(4)) == 1.0            # unit cubes
    assert bench.parallelepiped_fraction(I.cavity_mesh(4, jitter=0.2, seed=1)) < 0.5
    # a sheared and stretched copy of the cube mesh is still all parallelepipeds
    m = I.cavity_mesh(4)
    A = np.array([[1.0, 0.3, 0.0], [0.0, 2.0, 0.1], [0.2, 0.0, 0.7]])
    sheared = dict(m, xyz=m["xyz"] @ A.T + np.array([1.5, -2.0, 0.25]))
    assert bench.parallelepiped_fraction(sheared) == 1.0
    # the channel: a far field of boxes and a bent band around the cylinder
    f = bench.parallelepiped_fraction(I.channel_mesh(10, seed=0))
    assert 0.0 < f < 1.0


def test_element_work_counts_the_saved_jacobians():
    for name in ("residual", "rhs_restrict"):
        full = bench.element_flop(name, 0.0)
        assert full == bench.STAGE_WORK[name]["flop"]
        saved = full - bench.element_flop(name, 1.0)
        assert saved == bench.JACOBIAN_OPS * 7 * 64 * 2 // 8        # 7 of 8 Gauss points, 64 per patch
        assert bench.element_flop(name, 0.5) == full - saved / 2
