"""The oracle's OpenMP build against its single-threaded build: the same keys,
counts, offsets, CSR ids, root and ring labels, correspondences, fallback
flags, poses and RMSE histories, bit for bit.  Only loops whose iterations
are independent run in parallel, so the two builds must agree exactly; a
race or a shared temporary in a parallel loop would show up here."""
import numpy as np
import pytest

import oracle
from paper_2512_04996_gb300 import synth


@pytest.fixture()
def threaded():
    n = oracle.use_threads(4)
    yield n
    oracle.use_threads(1)


def _both(fn):
    oracle.use_threads(1)
    a = fn()
    oracle.use_threads(4)
    b = fn()
    oracle.use_threads(1)
    return a, b


def test_threads_are_used(threaded):
    if threaded == 1:
        pytest.skip("gcc without OpenMP: only the single-threaded oracle exists")
    assert oracle.threads() == threaded == 4


def test_build_and_search_identical(threaded):
    if threaded == 1:
        pytest.skip("gcc without OpenMP")
    p = synth.make_config(2)
    g = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
    a, b = _both(lambda: oracle.build_grid(g, p.target, 10))
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    T = synth.random_rigid(np.random.default_rng(3), 20.0, 0.2)
    ra, rb = _both(lambda: oracle.correspond(g, a, p.target, p.source, T))
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)
    assert ra[2].sum() > 0     # the global search ran in both


def test_registration_identical(threaded):
    if threaded == 1:
        pytest.skip("gcc without OpenMP")
    p = synth.make_config(1)
    g = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
    a, b = _both(lambda: oracle.register(g, 10, p.target, p.source, np.eye(4), max_iters=6, eps=0.0))
    assert a[0] == b[0] and a[2] == b[2]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[3], b[3])
