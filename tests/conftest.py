import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


_cache = {}


def cached(key, fn):
    if key not in _cache:
        _cache[key] = fn()
    return _cache[key]


@pytest.fixture(scope="session")
def sector_event():
    import synth
    return cached("sector", lambda: synth.one_sector(seed=0, truth=True))


@pytest.fixture(scope="session")
def sector_oracle(sector_event):
    import oracle
    return cached("sector_oracle", lambda: oracle.run(sector_event.clusters))


@pytest.fixture(scope="session")
def small_event():
    """Six sectors on both sides, 600 tracks: several tiles per row and a ragged tail."""
    import synth
    p = synth.GenParams(seed=11, n_primaries=600, n_secondaries=120, sectors=(0, 1, 2, 18, 19, 20))
    return cached("small", lambda: synth.generate(p, truth=True))


@pytest.fixture(scope="session")
def small_oracle(small_event):
    import oracle
    return cached("small_oracle", lambda: oracle.run(small_event.clusters))
