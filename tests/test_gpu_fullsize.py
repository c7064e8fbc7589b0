"""Parity at the full sizes of the skewed and mid configurations, in the launch
configuration bench.py times (default pi_create, per-batch rebuild).

Every result of every checked batch is compared with the oracle, then the final live
(key, value) set and the index levels. At 2^27 keys the oracle needs ~6 GB of host
memory and about a minute; these are the slowest GPU tests.
"""
import numpy as np
import pytest

from paper_1601_00159_gb300 import workloads as wl
from tests.parity import assert_results_equal, assert_state_equal, make_index, run_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    from paper_1601_00159_gb300 import build, load_library
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return load_library()


def _run(w, n_batches, levels_every):
    import oracle
    oracle.build()
    idx = make_index(w.keys, w.vals, w.promote_p, w.hash_seed)
    orc = oracle.Oracle(w.keys, w.vals, w.promote_p, w.hash_seed)
    gen = w.batches() if callable(w.batches) else iter(w.batches)
    for b in range(n_batches):
        batch = next(gen)
        got = run_batch(idx, batch)
        exp = orc.execute(batch.ops, batch.keys, batch.vals)
        assert_results_equal(got, exp, f"{w.name} batch {b}")
        if (b + 1) % levels_every == 0:
            assert_state_equal(idx, orc, f"{w.name} batch {b}")
    info = assert_state_equal(idx, orc, f"{w.name} end")
    idx.close()
    orc.close()
    return info


def test_mid_config_full_size():
    """2^24 keys, p = 1/4, 16 batches of 2^20 (50% search / 50% new inserts)."""
    info = _run(wl.mid(), 16, 8)
    assert info["live"] > (1 << 24) + 16 * (1 << 18)


def test_skewed_config_full_size():
    """2^27 keys, p = 1/4, Zipf(0.99) batches of 2^22 (90/5/5): two batches."""
    info = _run(wl.skewed(n_batches=2), 2, 2)
    assert info["size"] == 1 << 27 and info["tombstones"] > 0
