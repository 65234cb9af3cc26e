"""The allocation-free entry point against the allocating one.

speedup_amplitude_noalloc is for callers that cannot allocate device memory
(an allocator that owns all of the GPU's memory, a memory-capped process, a
loop where cudaMalloc/cudaFree are not allowed).  It keeps its scratch in a
static device array of the library, so two calls in a row must both give the
results of speedup_amplitude on the same samples, within the tolerances the
other amplitude tests use (the two entry points may split the samples into
reduction items differently, which changes only the summation order).

This file is collected last so that a run stopping at its first failure has
run every other test already; it also passes on its own in a fresh process.
"""
import pytest

torch = pytest.importorskip("torch")

import paper_1105_0542_gb300 as su  # noqa: E402

pytestmark = pytest.mark.gpu

CASE = ("aho", [1.0, 10.0], 0.0, 1.0, 1.0, 10, 8, 300_000, 1234)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_no_alloc_matches_the_allocating_entry_point_twice(prec, tol):
    ref = su.speedup_amplitude(*CASE, precision=prec, n_blocks=20)
    for _ in range(2):
        got = su.speedup_amplitude_noalloc(*CASE, precision=prec, n_blocks=20)
        for r, g in zip(ref, got):
            assert g["n"] == r["n"]
            assert abs(g["amp"] - r["amp"]) <= tol * r["amp"]
            assert abs(g["log_amp"] - r["log_amp"]) <= tol
            if r["level"]:
                assert abs(g["err"] - r["err"]) <= 100 * tol * r["err"]


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_amplitude_noalloc("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 10, 1 << 36, 1, n_blocks=1 << 20)
    assert e.value.code == -6
    # the array is still usable afterwards
    ok = su.speedup_amplitude_noalloc("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 1000, 1)
    assert ok[4]["n"] == 1000
