"""Shared fixtures.  GPU tests are marked ``gpu``; everything else runs on CPU."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled library")


@pytest.fixture(scope="session")
def gpu_lib():
    """The compiled CUDA library (fails loudly if the extension is missing)."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    from paper_2511_12450_gb300 import lfmm

    return lfmm
