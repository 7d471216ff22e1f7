import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libpp.so")
    config.addinivalue_line("markers", "slow: oracle tests that take more than ~20 s on CPU")


@pytest.fixture(scope="session")
def tiny_dg():
    from pp_inputs import CONFIGS, config_mesh
    from oracle.dg import DG
    c = CONFIGS["tiny"]
    return DG(config_mesh("tiny"), c["p"], kin=c["kin"])
