import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def bslib():
    """Build (if stale) and load libbs.so."""
    from paper_2309_07027_gb300 import _build
    _build.build()
    import paper_2309_07027_gb300 as bs
    bs.load()
    return bs


@pytest.fixture(scope="session")
def ctx(bslib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = bslib.Context(0)
    yield c
    c.close()
