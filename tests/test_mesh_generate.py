"""The library's O-grid generator (pp_ogrid_generate, host code through the C ABI) against
the package's input generator: identical triangles and face tags, vertex coordinates equal
to the rounding of the libm calls; the counter-based SplitMix64 stream against its
published first output; mesh validity (positive areas, closed boundary rings)."""
import numpy as np
import pytest

from pp_inputs import CONFIGS, ogrid
from pp_inputs.mesh import splitmix64

A = pytest.importorskip("paper_1512_00616_gb300.api")


def test_splitmix64_published_first_output():
    # SplitMix64 seeded with state 0: first output 0xE220A8397B1DCDAF (reference implementation)
    assert splitmix64(0, 0) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("n_theta,n_r,seed", [(8, 2, 0), (16, 2, 0), (64, 16, 1), (128, 32, 2), (13, 5, 99)])
def test_library_ogrid_equals_input_generator(n_theta, n_r, seed):
    m = ogrid(n_theta, n_r, seed=seed)
    v, t, g = A.pp_ogrid_generate(n_theta, n_r, 10.0, seed)
    assert np.array_equal(t, m.tris)
    assert np.array_equal(g, m.ftag)
    assert np.max(np.abs(v - m.verts)) <= 1e-12
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    area2 = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    assert np.all(area2 > 0)
    assert np.sum(g == 1) == n_theta and np.sum(g == 2) == n_theta


def test_config_meshes_are_the_library_meshes():
    for name in ("c0", "c1"):
        c = CONFIGS[name]
        v, t, g = A.pp_ogrid_generate(c["n_theta"], c["n_r"], 10.0, c["seed"])
        assert t.shape[0] == 2 * c["n_theta"] * c["n_r"]


def test_bad_arguments_rejected():
    with pytest.raises(A.PPError):
        A.pp_ogrid_generate(2, 4)
    with pytest.raises(A.PPError):
        A.pp_ogrid_generate(8, 2, r_far=0.5)
