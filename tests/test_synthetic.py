"""The seeded input generator (no method arithmetic) pinned to SplitMix64's published outputs."""
import numpy as np

import synthetic as S
from tests.oracle_pins import read_rows


def test_splitmix64_published_values():
    ref = [int(r[0], 16) for r in read_rows("splitmix64_seed0.txt")]
    assert [int(v) for v in S.splitmix64(0, 3)] == ref
    # counter form: offsets index into the same stream
    assert int(S.splitmix64(0, 1, offset=2)[0]) == ref[2]


def test_uniform_range_and_mesh_layout():
    u = S.uniform_pm1(5, 100000)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01
    V = S.structured_vertices(3, 4, 5, 0.1, 1910)
    assert V.shape == (4 * 5 * 6, 3)
    # boundary vertices stay on the cube faces; interior ones move by <= 0.1 h
    V0 = S.structured_vertices(3, 4, 5, 0.0)
    d = np.abs(V - V0)
    assert np.all(d <= 0.1 * np.array([1 / 3, 1 / 4, 1 / 5]) + 1e-15)
    on_face = (np.isclose(V0, 0) | np.isclose(V0, 1)).any(1)
    assert np.all(d[on_face] == 0) and np.all(d[~on_face].max(1) > 0)
    EV = S.structured_elem_vert(3, 4, 5)
    assert EV.shape == (60, 8)
    # corner c = cx + 2 cy + 4 cz of element 0 sits at (cx h, cy h, cz h)
    for c in range(8):
        np.testing.assert_allclose(V0[EV[0, c]], [(c & 1) / 3, ((c >> 1) & 1) / 4, ((c >> 2) & 1) / 5])
    p = S.permutation(50, 3)
    assert sorted(p.tolist()) == list(range(50))
