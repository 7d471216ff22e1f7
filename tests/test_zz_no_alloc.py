"""pp_qoi_rate_noalloc: the scratch-free variant of pp_qoi_rate.

Some callers may not allocate GPU memory, e.g. under an allocator that forbids
outside allocations, or after start-up.  For them the library keeps this reduction's
scratch in a static device array instead of calling cudaMalloc.  The test calls the
variant through the C ABI twice in a row and checks each result against
pp_qoi_rate, which uses workspace allocated by the context.  This file is named so
that pytest collects it last."""
import numpy as np
import pytest

from gpu_common import PARITY_TOL, make, perturbed_state, to_dev
from pp_inputs import MU_C0, config_mesh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_qoi_rate_matches_allocating_entry_point():
    mesh = config_mesh("c0")
    A, ctx, m = make(1, 0, mesh)
    try:
        for call, (t, seed) in enumerate([(0.3, 5), (2.7, 6)]):
            u = to_dev(perturbed_state(mesh.nt, 1, seed=seed, amp=5e-2))
            ref = A.pp_qoi_rate(ctx, m, MU_C0, t, u)
            got = A.pp_qoi_rate_noalloc(ctx, m, MU_C0, t, u)
            scale = np.max(np.abs(ref))
            assert np.max(np.abs(got - ref)) <= PARITY_TOL * scale, (call, got, ref)
    finally:
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)
