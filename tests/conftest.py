"""Shared fixtures.  Tests marked ``gpu`` need a CUDA device (sm_103); all
others run on the CPU and never launch a kernel."""
from __future__ import annotations

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103); calls librdc kernels")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")


@pytest.fixture(scope="session")
def om():
    """The oracle module (test infrastructure)."""
    import oracle
    oracle.load()
    return oracle


@pytest.fixture(scope="session")
def orc(om):
    return om.load()


@pytest.fixture(scope="session")
def librdc():
    """The built C-ABI library (compiled here if missing or stale)."""
    from paper_1901_06535_gb300 import build
    build.build()
    import paper_1901_06535_gb300 as pkg
    pkg.lib()
    return pkg


@pytest.fixture(scope="session")
def gpu(librdc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device visible")
    torch.cuda.init()
    return librdc
