import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels through the C-ABI)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def inputs():
    from paper_2207_14256_gb300 import inputs as I
    return I


@pytest.fixture(scope="session")
def c1_tables(inputs):
    return inputs.transfer_tables(inputs.config("c1_32"))
