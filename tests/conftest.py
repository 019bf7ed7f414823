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


def pytest_collection_modifyitems(config, items):
    """GPU tests need a CUDA device; without one (this CPU container) they are
    skipped, never silently routed elsewhere."""
    try:
        import torch
        has_cuda = torch.cuda.is_available()
    except Exception:
        has_cuda = False
    if has_cuda:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)
