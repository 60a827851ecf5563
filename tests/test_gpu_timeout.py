"""Failure detection without a GPU fault: bounded waits in the tensor-core kernel.

Every wait of the persistent tcgen05 kernel on an mbarrier gives up after about two seconds,
raises RICI_ERR_TIMEOUT in the status word and lets the CTA free its tensor memory and return.
The test hook RICI_SEARCH_TEST_WITHHOLD_LOAD makes one CTA withhold its first tile load (a
barrier that nothing completes).  The call must end by itself, report the timeout, and leave the
context usable: the next search returns exact results.
"""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_withheld_load_times_out_and_context_stays_usable(oracle_mod):
    import torch

    import paper_2007_02306_gb300 as p
    from paper_2007_02306_gb300 import build

    build.build()
    p.load_library()
    rng = np.random.default_rng(4)
    nd, hay, m = synth.images.needle_haystack_set(rng, 200, 1500, 64)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    t0 = time.time()
    p.crss_search(d(nd), d(hay), d(m), mode=p.SEARCH_TENSOR | p.binding.SEARCH_TEST_WITHHOLD_LOAD)
    status = p.sync_status()
    elapsed = time.time() - t0
    assert status & p.binding.ERR_TIMEOUT
    assert elapsed < 30.0
    r = p.crss_search(d(nd), d(hay), d(m), mode=p.SEARCH_TENSOR)
    assert p.sync_status() == 0
    ref = oracle_mod.crss_search(nd, hay, m)
    for k in ("rank", "true_distance", "top1"):
        assert np.array_equal(r[k].cpu().numpy(), ref[k]), k
