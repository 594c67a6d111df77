import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: full-size oracle work (tens of seconds)")


_KEYS = {}


def oracle_keys(params):
    """Oracle key set for a parameter dict, cached per process."""
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    key = tuple(sorted(params.items()))
    if key not in _KEYS:
        _KEYS[key] = o.keygen(params, W.CRS_SEED, W.party_seeds(params["k"]))
    return _KEYS[key]


def to_dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def from_dev(t):
    a = t.cpu().numpy()
    if a.dtype == np.int32:
        a = a.view(np.uint32)
    return a


@pytest.fixture(scope="session")
def gpu_ready():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_05825_gb300 import build
    build.build()
    return True
