"""CPU checks of the per-region parity statistic (tests/planes.py): a
mistake confined to one face plane that the all-node relative L2 error
dilutes below the bar is reported on that plane."""
import numpy as np

from planes import region_errors, regions


def test_regions_cover_faces_and_interior():
    n = (6, 5, 4)
    r = regions(n, (0, 3, 1), (0, 2, 1))
    names = [k for k, _ in r]
    assert names == ["axis 1 low face", "axis 1 high face", "axis 2 low face", "axis 2 high face", "interior"]
    m = dict(r)
    assert m["axis 1 low face"].sum() == 6 * 4 and m["interior"].sum() == 6 * 3 * 2
    assert (np.logical_or.reduce([v for k, v in r if k != "interior"]) ^ m["interior"]).all()


def test_one_plane_error_is_not_diluted():
    n = (64, 128, 64)
    N = int(np.prod(n))
    rng = np.random.default_rng(0)
    ro = 1 + 0.01 * rng.standard_normal(N)
    uo = 0.05 * rng.standard_normal((3, N))
    wall = dict(regions(n, (0, 0, 1), (0, 0, 1)))["axis 2 high face"]
    uo[:, wall] = 0.0  # a wall at rest
    ug = uo.copy()
    ug[:, wall] = 5e-5 * 0.05  # a plane-wide slip on the wall, 5e-5 of the flow speed
    glob = np.linalg.norm(ug - uo) / np.linalg.norm(uo)
    assert glob < 1e-5  # passes the all-node bar
    e = region_errors(ro, ug, ro, uo, n, (0, 0, 1), (0, 0, 1))
    assert e["axis 2 high face"][1] > 4e-5 and e["interior"] == (0.0, 0.0)
