"""The allocation-free entry point against the allocating one and the oracle.

speedup_amplitude_noalloc is for callers that cannot allocate device memory
(an allocator that owns all of the GPU's memory, a memory-capped process, a
loop where cudaMalloc/cudaFree are not allowed).  It keeps its scratch in a
static device array of the library but builds the same tables and launch
shape as speedup_amplitude, so two calls in a row must both give the
allocating entry point's results bit for bit, and the oracle's estimator on
the same samples within the tolerances of the other amplitude tests.

This file is collected last so that a run stopping at its first failure has
run every other test already; it also passes on its own in a fresh process.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1105_0542_gb300 as su  # noqa: E402
from oracle import mc  # noqa: E402

pytestmark = pytest.mark.gpu

CASE = ("aho", [1.0, 10.0], 0.0, 1.0, 1.0, 10, 8, 300_000, 1234)
KEYS = ("amp", "log_amp", "err", "err_naive", "ess", "n")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_no_alloc_matches_the_allocating_entry_point_twice(prec):
    ref = su.speedup_amplitude(*CASE, precision=prec, n_blocks=20)
    for _ in range(2):
        got = su.speedup_amplitude_noalloc(*CASE, precision=prec, n_blocks=20)
        for r, g in zip(ref, got):
            for k in KEYS:
                assert g[k] == r[k], (prec, r["level"], k)


@pytest.mark.parametrize("prec,bits,tol", [("fp64", 53, 1e-10), ("fp32", 24, 1e-4)])
def test_no_alloc_matches_the_oracle_estimator(prec, bits, tol):
    model, params, a, b, T, p, s, n, seed, nb = "dw", [1.0], -1.0, 1.0, 1.0, 6, 6, 4099, 77, 9
    got = su.speedup_amplitude_noalloc(model, params, a, b, T, p, s, n, seed, precision=prec, n_blocks=nb)
    o = mc.Oracle(model, params, p)
    w, _ = o.logweights(a, b, T, s, seed, n, bits=bits, threads=os.cpu_count() or 1)
    ref = mc.estimate(w, o.level0(a, b, T), a, b, T, nb)
    for lev in range(s + 1):
        assert got[lev]["n"] == n
        assert abs(got[lev]["log_amp"] - ref[lev]["log_amp"]) <= tol, lev
        if lev:
            assert abs(got[lev]["err"] - ref[lev]["err"]) <= 100 * tol * ref[lev]["err"], lev


def test_no_alloc_raises_rounds_to_fit_and_keeps_the_samples():
    # 1e7 samples, ten levels: the per-item tuples of one path per thread
    # (25 MB) exceed the array, so the call takes four paths per thread
    args = ("aho", [1.0, 10.0], 0.0, 1.0, 1.0, 10, 10, 10_000_000, 5)
    got = su.speedup_amplitude_noalloc(*args, precision="fp32", n_blocks=64)
    ref = su.speedup_amplitude(*args, precision="fp32", n_blocks=64, rounds=4)
    for r, g in zip(ref, got):
        assert g["n"] == 10_000_000
        for k in KEYS:
            assert g[k] == r[k], (r["level"], k)
    assert np.isfinite([g["amp"] for g in got]).all()


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_amplitude_noalloc("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 10, 1 << 36, 1, n_blocks=1 << 20)
    assert e.value.code == -6
    # the array is still usable afterwards
    ok = su.speedup_amplitude_noalloc("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 1000, 1)
    assert ok[4]["n"] == 1000
