"""Failure detection on the device path, with every fault made on the host
(no fault, trap or hang of the GPU is caused):

* an injected allocation failure at each of the first allocations of a call
  surfaces as SU_ENOMEM, and the next call works and gives the same result;
* a NaN injected into a coefficient table surfaces as SU_ENONFINITE (single
  instance and batched plans), never as a wrong number;
* a batched work queue cut short surfaces at finalize (the missing samples
  are counted), and the next execute is complete again;
* the proposal network's bounded tensor-core wait: with its MMA commit
  withheld (an mbarrier that nothing completes) the launch gives up after
  about a second with SU_ETIMEOUT, frees its tensor memory, and the next call
  (same device context) works and matches the result of an undisturbed one;
* the device-timed execute returns a positive time and the same tuples.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1105_0542_gb300 as su  # noqa: E402
from oracle import proposal as pr  # noqa: E402

pytestmark = pytest.mark.gpu
SU_ENOMEM, SU_ECUDA, SU_ETIMEOUT, SU_ENONFINITE = -2, -3, -4, -5
ARGS = ("aho", [1.0, 10.0], 0.0, 1.0, 1.0, 6, 6, 5000, 11)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    torch.cuda.set_device(0)
    yield
    su.su_fault_inject("clear")


def test_allocation_failures_are_reported_and_recovered():
    ref = su.speedup_amplitude(*ARGS)
    failed = 0
    for k in range(1, 6):
        su.su_fault_inject("alloc", k)
        try:
            got = su.speedup_amplitude(*ARGS)
        except su.SpeedupError as e:
            assert e.code == SU_ENOMEM, (k, e)
            failed += 1
            continue
        finally:
            su.su_fault_inject("clear")
        assert got[6]["amp"] == ref[6]["amp"]   # past the call's allocations: untouched
    assert failed >= 2                          # tables and the tuple/scratch buffer
    again = su.speedup_amplitude(*ARGS)
    assert again[6]["amp"] == ref[6]["amp"] and again[6]["err"] == ref[6]["err"]


def test_nan_in_a_coefficient_table_is_reported():
    su.su_fault_inject("table_nan")
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_amplitude(*ARGS)
    assert e.value.code == SU_ENONFINITE
    su.su_fault_inject("table_nan")
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_amplitude_batch("aho", [1.0, 1.0], 10, [(0.0, 1.0, 1.0, 4), (1.0, 2.0, 0.5, 3)], 1000, 3)
    assert e.value.code == SU_ENONFINITE
    assert np.isfinite(su.speedup_amplitude(*ARGS)[6]["amp"])


def test_truncated_work_queue_is_detected():
    inst = [(0.1 * i, -0.2 * i, 0.5, 2 + i % 5) for i in range(40)]
    pl = su.BatchPlan("aho", [1.0, 1.0], 10, inst, 2000, 5, precision="fp32", n_blocks=4)
    t = torch.empty(pl.tuple_bytes // 8, dtype=torch.float64, device="cuda")
    sc = torch.empty(pl.scratch_bytes, dtype=torch.uint8, device="cuda")
    su.su_fault_inject("queue_stop", 7)
    pl.su_batch_plan_execute(t, sc)
    torch.cuda.synchronize()
    with pytest.raises(su.SpeedupError) as e:
        pl.su_batch_plan_finalize(t.cpu().numpy(), sc)
    assert e.value.code == SU_ECUDA and "ended early" in str(e.value)
    pl.su_batch_plan_execute(t, sc)
    torch.cuda.synchronize()
    res = pl.su_batch_plan_finalize(t.cpu().numpy(), sc)
    assert all(r["n"] == 2000 for r in res)


def test_withheld_mma_commit_times_out_and_the_context_survives():
    th = pr.init(3)
    P = su.Proposal(th)
    args = ("dw", [1.0], -1.0, 1.0, 1.0, 8, 5, 20000, 13, P)
    ref = su.speedup_amplitude_proposal(*args, n_blocks=10)
    su.su_fault_inject("withhold_mma")
    t0 = time.perf_counter()
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_amplitude_proposal(*args, n_blocks=10)
    dt = time.perf_counter() - t0
    assert e.value.code == SU_ETIMEOUT
    assert 0.5 < dt < 30.0, dt
    got = su.speedup_amplitude_proposal(*args, n_blocks=10)
    assert got[5]["amp"] == ref[5]["amp"] and got[5]["err"] == ref[5]["err"]


def test_device_timed_execute():
    pl = su.Plan(*ARGS, n_blocks=16)
    t = torch.empty(pl.tuple_bytes // 8, dtype=torch.float64, device="cuda")
    sc = torch.empty(pl.scratch_bytes, dtype=torch.uint8, device="cuda")
    pl.su_plan_execute(t, sc)
    torch.cuda.synchronize()
    a = t.cpu().numpy().copy()
    n, ms = pl.su_plan_execute_timed(t, sc)
    assert n == 2 and ms > 0
    assert np.array_equal(a, t.cpu().numpy())
