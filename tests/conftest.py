import os

import pytest


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built library")


@pytest.fixture(scope="session")
def rng():
    import numpy as np
    return np.random.default_rng(20260103)


def random_blocks(shapes, rng, scale=0.3):
    """Random complex amplitude blocks; the same-spin T2 blocks (index 2, 4)
    are antisymmetrised in (i,j) and (a,b)."""
    import numpy as np
    t = [scale * (rng.standard_normal(s) + 1j * rng.standard_normal(s)) for s in shapes]
    for k in (2, 4):
        if len(t) > k:
            t[k] = t[k] - t[k].transpose(1, 0, 2, 3)
            t[k] = t[k] - t[k].transpose(0, 1, 3, 2)
    return t
