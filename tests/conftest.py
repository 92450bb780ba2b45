"""Shared pytest configuration.

Markers: ``gpu`` tests need a CUDA device and the built library; everything
else runs on a CPU-only machine.  The repository root is put on sys.path so
``synth``, ``oracle`` and the package import without installation.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running")


@pytest.fixture(scope="session")
def orc():
    import oracle
    return oracle.default()


@pytest.fixture(scope="session")
def mmlib():
    """The CUDA library, initialised once per session on cuda:0."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected on a machine without a GPU")
    import paper_1306_6192_gb300 as mm
    st = mm.mm_init(device=0)
    assert st == mm.MM_OK, mm.mm_strerror(st)
    yield mm
    mm.mm_shutdown()
