import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def gfem():
    """The CUDA library (built in-tree) and its binding, for -m gpu tests."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_0066_gb300 as fem
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fem.nat.load()
    return fem


def rel_err_per_element(A, Aref):
    """Per element: max_ij |A - Aref| / max_ij |Aref| (FP64, numpy)."""
    import numpy as np
    A = np.asarray(A, dtype=np.float64)
    d = np.abs(A - Aref).reshape(A.shape[0], -1).max(1)
    s = np.abs(Aref).reshape(A.shape[0], -1).max(1)
    return d / np.where(s > 0, s, 1.0)
