"""Failure detection without a GPU fault: the library's bounded device waits
(decoupled look-back, bulk-copy mbarrier phases) are made to run out on
purpose -- a predecessor that never publishes, a barrier phase that never
completes -- and must report LCO_ERR_TIMEOUT and finish, leaving the context
usable."""
import time

import pytest
import torch

import paper_1802_02619_gb300 as lco
import synth
from gpu_util import assert_contract_matches, dev

pytestmark = pytest.mark.gpu

LCO_ERR_TIMEOUT = 5


def test_waits_run_out_and_report_timeout():
    t0 = time.perf_counter()
    lb, mb = lco.selftest_wait(budget_cycles=1_000_000)        # ~0.5 ms at 2 GHz
    assert lb == LCO_ERR_TIMEOUT and mb == LCO_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0


def test_context_usable_after_timeouts():
    for _ in range(3):
        assert lco.selftest_wait(budget_cycles=200_000) == (LCO_ERR_TIMEOUT, LCO_ERR_TIMEOUT)
    cfg = synth.config_fd2d(16)
    C, info = lco.contract(dev(cfg["A"]), dev(cfg["B"]), cfg["modes_a"], cfg["modes_b"], return_info=True)
    assert info["status"] == 0          # the default budget is back in force
    assert_contract_matches(C, cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])
    torch.cuda.synchronize()
