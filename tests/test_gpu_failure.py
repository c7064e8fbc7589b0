"""Failure paths, exercised on the GPU without a fault: an allocation failure injected on
the host must return PI_ERR_OOM and leave the index as it was; a bounded wait on a flag
that nothing sets must give up with PI_ERR_TIMEOUT and leave the context usable."""
import pytest

from paper_1601_00159_gb300 import workloads as wl
from tests.parity import assert_results_equal, assert_state_equal, make_index, run_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def orc_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    from paper_1601_00159_gb300 import build, load_library
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return load_library()


@pytest.mark.parametrize("warm", [False, True])
def test_injected_allocation_failure_leaves_index_unchanged(orc_mod, warm):
    """warm=False: the first batch's scratch allocation fails. warm=True: batches of new
    keys run until the next one must grow the storage layer, and that growth fails."""
    import paper_1601_00159_gb300 as pkg
    q = 200000
    w = wl.random_small(31, 5000, q, 1 << 40, p=0.25, n_batches=6)  # a third insert new keys
    idx = make_index(w.keys, w.vals, w.promote_p, w.hash_seed)
    orc = orc_mod.Oracle(w.keys, w.vals, w.promote_p, w.hash_seed)
    b = 0
    if warm:
        while True:
            info = idx.info()
            if info["size"] + q > info["storage_capacity"] and b > 0:
                break  # batch b must grow the storage layer
            batch = w.batches[b]
            assert_results_equal(run_batch(idx, batch), orc.execute(batch.ops, batch.keys, batch.vals), f"batch {b}")
            b += 1
            assert b < len(w.batches) - 1, "the storage layer never filled up"
    cap0 = idx.info()["storage_capacity"]
    pkg.test_fail_allocations(1)
    try:
        with pytest.raises(pkg.PiError) as ei:
            run_batch(idx, w.batches[b])
    finally:
        pkg.test_fail_allocations(0)
    assert ei.value.code == pkg.PI_ERR_OOM
    assert idx.info()["storage_capacity"] == cap0
    assert_state_equal(idx, orc, "after the refused batch")
    for k in range(b, len(w.batches)):  # the refused batch and the rest now run and match
        batch = w.batches[k]
        assert_results_equal(run_batch(idx, batch), orc.execute(batch.ops, batch.keys, batch.vals), f"batch {k}")
    info = assert_state_equal(idx, orc, "end")
    assert info["storage_capacity"] > cap0
    idx.close()
    orc.close()


def test_bounded_wait_gives_up_and_context_stays_usable(orc_mod):
    import paper_1601_00159_gb300 as pkg
    rc, word = pkg.selftest_wait()
    assert rc == pkg.PI_ERR_TIMEOUT
    assert word & 1  # the timeout bit
    w = wl.random_small(3, 2000, 6000, 1 << 20, p=0.5, n_batches=2)
    idx = make_index(w.keys, w.vals, w.promote_p, w.hash_seed)
    orc = orc_mod.Oracle(w.keys, w.vals, w.promote_p, w.hash_seed)
    for b, batch in enumerate(w.batches):
        assert_results_equal(run_batch(idx, batch), orc.execute(batch.ops, batch.keys, batch.vals), f"batch {b}")
    assert_state_equal(idx, orc, "after the self-test")
    idx.close()
    orc.close()
