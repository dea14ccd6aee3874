"""Shared test configuration.

Markers: `gpu` tests need a CUDA device and the built libmg.so; everything else
runs on the CPU (the oracle against its pins, host logic, the C ABI's exports).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and libmg.so built for sm_103a")
    config.addinivalue_line("markers", "slow: larger CPU cases")


@pytest.fixture(scope="session")
def cuda_lib():
    """The loaded library on a machine with a GPU (built on demand)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1912_02868_gb300 as mg
    mg.build()
    return mg.load()
