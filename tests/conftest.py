import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")


@pytest.fixture(scope="session")
def pairs():
    """The seeded single-pair workloads, generated once per session."""
    from paper_2512_04996_gb300 import synth
    cache = {}

    def get(k):
        if k not in cache:
            cache[k] = synth.make_config(k)
        return cache[k]

    return get


@pytest.fixture()
def oracle_threads():
    """The oracle on all host cores for the duration of one test (its
    OpenMP build gives the same results as the single-threaded one)."""
    import oracle
    n = oracle.use_threads(os.cpu_count() or 1)
    yield n
    oracle.use_threads(1)
