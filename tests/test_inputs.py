"""The synthetic input recipe: seeded O-grids around the 12%-thick symmetric 4-digit
airfoil (closed trailing edge), the workload sizes, and seeded reproducibility."""
import numpy as np
import pytest

from pp_inputs import CONFIGS, config_mesh, config_mu, fourier6_samples, free_stream_state
from pp_inputs.mesh import _naca_half_thickness, ogrid


def _areas(m):
    a, b, c = (m.verts[m.tris[:, k]] for k in range(3))
    return 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))


@pytest.mark.parametrize("name,nt", [("tiny", 32), ("c0", 64), ("c1", 2048)])
def test_workload_sizes_and_orientation(name, nt):
    m = config_mesh(name)
    c = CONFIGS[name]
    assert m.nt == nt == 2 * c["n_theta"] * c["n_r"]
    assert np.all(_areas(m) > 0)                       # counter-clockwise, none inverted
    # one wall face and one far-field face per angular cell
    assert np.sum(m.ftag == 1) == c["n_theta"] and np.sum(m.ftag == 2) == c["n_theta"]


def test_interior_faces_are_shared_exactly_once():
    m = config_mesh("c0")
    seen = {}
    for e in range(m.nt):
        for f in range(3):
            a, b = m.tris[e, f], m.tris[e, (f + 1) % 3]
            seen.setdefault((min(a, b), max(a, b)), []).append(m.ftag[e, f])
    for tags in seen.values():
        assert (len(tags) == 2 and tags == [0, 0]) or (len(tags) == 1 and tags[0] in (1, 2))


def test_wall_on_the_airfoil_with_uniform_arclength_spacing():
    m = ogrid(64, 4, seed=1)
    wall = m.verts.reshape(64, 5, 2)[:, 0]
    # on the closed-trailing-edge thickness law, chord [0, 1]
    assert np.allclose(np.abs(wall[:, 1]), _naca_half_thickness(wall[:, 0]), atol=1e-12)
    assert wall[:, 0].min() == 0.0 and np.isclose(wall[:, 0].max(), 1.0)
    seg = np.linalg.norm(np.roll(wall, -1, 0) - wall, axis=1)
    assert seg.max() / seg.min() < 1.06                 # equal arc length (chords of the arcs)
    # the cosine clustering it replaces puts far smaller cells at the leading/trailing edges
    cw = ogrid(64, 4, seed=1, clustering="cosine").verts.reshape(64, 5, 2)[:, 0]
    cseg = np.linalg.norm(np.roll(cw, -1, 0) - cw, axis=1)
    assert cseg.max() / cseg.min() > 3.0


def test_far_field_circle_and_jitter_bound():
    m0 = ogrid(16, 4, seed=0, jitter=0.0)
    m1 = ogrid(16, 4, seed=0)
    far = m1.verts.reshape(16, 5, 2)[:, -1]
    assert np.allclose(np.hypot(far[:, 0] - 0.5, far[:, 1]), 10.0)
    P0, P1 = m0.verts.reshape(16, 5, 2), m1.verts.reshape(16, 5, 2)
    assert np.array_equal(P0[:, [0, -1]], P1[:, [0, -1]])   # wall and far field not jittered
    for k in range(16):
        for j in range(1, 4):
            nbrs = [P0[(k + 1) % 16, j], P0[(k - 1) % 16, j], P0[k, j + 1], P0[k, j - 1]]
            h = min(np.linalg.norm(P0[k, j] - x) for x in nbrs)
            # 10% of the spacing at the time of the move (neighbours already moved count),
            # i.e. at most ~12% of the unjittered spacing
            assert np.max(np.abs(P1[k, j] - P0[k, j])) <= 0.12 * h


def test_seeded_reproducibility():
    a, b, c = ogrid(16, 4, seed=3), ogrid(16, 4, seed=3), ogrid(16, 4, seed=4)
    assert np.array_equal(a.verts, b.verts) and not np.array_equal(a.verts, c.verts)
    assert np.array_equal(config_mu("c1"), config_mu("c1"))
    assert np.array_equal(fourier6_samples(4, 7), fourier6_samples(4, 7))


def test_fourier_motion_within_twenty_percent_box_and_free_stream():
    from pp_inputs import MU_F6_BASE, MU_F6_SCALE
    mu = fourier6_samples(256, 5)
    assert np.all(np.abs(mu - MU_F6_BASE) <= 0.2 * MU_F6_SCALE + 1e-15)
    u = free_stream_state(3, 2).reshape(3, 4, -1)
    g, M = 1.4, 0.2
    assert np.allclose(u[:, 0], 1.0) and np.allclose(u[:, 1], 1.0) and np.allclose(u[:, 2], 0.0)
    assert np.allclose(u[:, 3], 1.0 / (g * (g - 1.0) * M * M) + 0.5)
