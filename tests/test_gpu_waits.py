"""Bounded device waits, exercised without any fault: a grid barrier that
one CTA never reaches must end in about the set time with BLOWCHOC_ETIMEOUT,
and the context must stay usable (a filter works afterwards)."""
import time

import numpy as np
import pytest

import workloads
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


def test_grid_barrier_gives_up_and_context_survives():
    import paper_2501_18977_gb300 as bc
    t0 = time.perf_counter()
    rc = bc.blowchoc_barrier_selftest(ctas=8, seconds=0.3)
    dt = time.perf_counter() - t0
    assert rc == bc.BLOWCHOC_ETIMEOUT
    assert dt < 5.0
    f = bc.Filter(256, 10, 2, bc.COST_MIX, 50.0, hash_seed=1, batch=20000)
    try:
        keys = workloads.uniform_keys(9, 50000)
        f.insert(to_dev(keys))
        bm = f.query(to_dev(keys)).cpu().numpy().view(np.uint64)
        assert np.unpackbits(bm.view(np.uint8), bitorder="little")[:50000].all()
        assert f.stats().inserted + f.stats().skipped == 50000
    finally:
        f.close()
