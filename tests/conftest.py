import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300) and the built libvmat.so")


@pytest.fixture(scope="session")
def tiny_problem():
    from paper_1005_4396_b300 import inputs
    return inputs.make_problem(inputs.tiny_config())


@pytest.fixture(scope="session")
def small_problem():
    from paper_1005_4396_b300 import inputs
    return inputs.make_problem(inputs.small_config())
