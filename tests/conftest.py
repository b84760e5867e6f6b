import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300); run with -m gpu")
    config.addinivalue_line("markers", "slow: oracle runs of several seconds")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def trained_surrogate():
    """The chemistry surrogate trained on lognormal boxes of the 128^3 recipe (seeds 100-107,
    disjoint from every evaluation box) by the library's own kernels; shared by the GPU tests
    of the surrogate in the step."""
    from paper_1004_2503_b300 import surrogate as S
    m, nrec, dt = S.train_on_lognormal_boxes(seeds=range(100, 108), steps=80, train_steps=1500)
    yield m
    m.close()
