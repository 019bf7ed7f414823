import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libfrax")
    config.addinivalue_line("markers", "slow: long CPU-only check")


@pytest.fixture(scope="session")
def models():
    import gen
    return {
        "chain7": gen.chain7(0),
        "humanoid": gen.humanoid(0),
        "tree_a": gen.random_tree(101),
        "tree_b": gen.random_tree(117),
    }
