"""The launch-shape autotuner (no counterpart in the paper: a search over this
implementation's launch parameters) and the shapes it chooses between.

* every shape (bisection levels kept in registers 2^seg_log2 slices at a
  time, paths per thread per work item) gives the same amplitudes up to the
  order of floating-point sums, and per-sample weights equal to the oracle's;
* su_autotune returns the fastest shape it timed, later plans with automatic
  shape use it, explicit shapes override it, and clearing the table restores
  the built-in rule.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1105_0542_gb300 as su  # noqa: E402
from oracle import mc  # noqa: E402

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
CASE = ("aho", [1.0, 10.0], 0.0, 1.0, 1.0)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    torch.cuda.set_device(0)
    su.su_autotune_clear()
    yield
    su.su_autotune_clear()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_every_shape_gives_the_same_amplitudes(prec, tol):
    p, s, n = 6, 8, 20000
    ref = su.speedup_amplitude(*CASE, p, s, n, 77, precision=prec, n_blocks=16)
    for f in range(1, 6):
        for r in (1, 2, 4, 8):
            got = su.speedup_amplitude(*CASE, p, s, n, 77, precision=prec, n_blocks=16, seg_log2=f, rounds=r)
            for lev in range(1, s + 1):
                assert got[lev]["amp"] == pytest.approx(ref[lev]["amp"], rel=tol), (f, r, lev)
                assert got[lev]["err"] == pytest.approx(ref[lev]["err"], rel=1e3 * tol), (f, r, lev)


@pytest.mark.parametrize("f", [3, 4])
def test_small_segments_per_sample_weights_match_oracle(f):
    """(seg_log2 = 1, 2 at s = 10 would keep 2^(s - seg_log2) + 1 segment
    endpoints per thread in shared memory, more than a CTA has: refused.)"""
    p, s, n = 10, 10, 96
    w = torch.zeros((n, s), dtype=torch.float64, device="cuda")
    su.speedup_logweights(*CASE, p, s, 500, n, 5, w, seg_log2=f)
    torch.cuda.synchronize()
    o = mc.Oracle(CASE[0], CASE[1], p)
    ref, _ = o.logweights(*CASE[2:], s, 5, n, sample0=500, threads=THREADS)
    got = w.cpu().numpy()
    scale = np.maximum(np.abs(ref), np.median(np.abs(ref), axis=0))
    assert float(np.max(np.abs(got - ref) / scale)) <= 1e-12


def test_autotune_stores_the_fastest_shape():
    su.su_autotune_clear()
    p, s = 10, 10
    best, all_ = su.su_autotune(*CASE, p, s, 100_000, 3, precision="fp64", n_blocks=100)
    assert len(all_) >= 10
    assert best["ms"] == min(t["ms"] for t in all_)
    assert all(t["ms"] > 0 for t in all_)
    shapes = {(t["seg_log2"], t["rounds"]) for t in all_}
    assert (best["seg_log2"], best["rounds"]) in shapes
    pl = su.Plan(*CASE, p, s, 1_000_000, 9, precision="fp64", n_blocks=100)
    assert pl.su_plan_shape() == (best["seg_log2"], best["rounds"])
    pl2 = su.Plan(*CASE, p, s, 1_000_000, 9, precision="fp64", n_blocks=100, seg_log2=3, rounds=2)
    assert pl2.su_plan_shape() == (3, 2)
    # other keys are untouched: single precision still uses the rule
    pl3 = su.Plan(*CASE, p, s, 1_000_000, 9, precision="fp32", n_blocks=100)
    assert pl3.su_plan_shape() == (5, 1)
    su.su_autotune_clear()
    pl4 = su.Plan(*CASE, p, s, 1_000_000, 9, precision="fp64", n_blocks=100)
    assert pl4.su_plan_shape() == (4, 1)


def test_shape_that_does_not_fit_is_refused():
    with pytest.raises(su.SpeedupError) as e:
        su.Plan(*CASE, 10, 10, 1000, 9, precision="fp64", seg_log2=1)
    assert e.value.code == -6
