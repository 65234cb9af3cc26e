"""The single-precision samplers with the table shape compiled in.

A plan whose collapsed W_p tables (Eq. SNp in powers of xb^2 and z) have one
of the shapes compiled into the library -- the harmonic oscillator's and the
quartic potentials' even-ring shapes at p <= 18 -- runs a sampler with the
nested Horner unrolled for that shape.  It performs the same operations in
the same order as the generic sampler, so both give the same bits; the
per-sample parity of either against the oracle is in test_gpu_parity.py
(its single-precision cases with s >= 5 run the compiled shapes).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1105_0542_gb300 as su  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    torch.cuda.set_device(0)


def _w(model, params, p, s, n, seed, kernel):
    w = torch.full((n, s), float("nan"), dtype=torch.float64, device="cuda")
    su.speedup_logweights(model, params, -0.3, 0.8, 1.0, p, s, 11, n, seed, w, precision="fp32", kernel=kernel)
    torch.cuda.synchronize()
    return w.cpu().numpy()


SHAPES = [("ho", [1.0], 1), ("ho", [2.0], 7)] + [("aho", [1.0, 10.0], p) for p in range(1, 19)]


@pytest.mark.parametrize("model,params,p", SHAPES, ids=[f"{m}-p{p}" for m, _, p in SHAPES])
def test_compiled_shape_gives_the_generic_bits(model, params, p):
    # s = 7: four segments of 32 slices, the coarse levels from the segment ends;
    # n = 389: a ragged last chunk
    k = su.su_fixed_shape(model, params, p)
    assert k >= 0
    pl = su.Plan(model, params, -0.3, 0.8, 1.0, p, 7, 389, 5, precision="fp32")
    assert pl.su_plan_kernel() == k
    fixed = _w(model, params, p, 7, 389, 5, "auto")
    generic = _w(model, params, p, 7, 389, 5, "generic")
    assert np.isfinite(fixed).all()
    assert np.array_equal(fixed, generic)


def test_compiled_shape_amplitudes_equal_generic():
    args = ("dw", [5.0], -1.0, 1.0, 1.0, 12, 9, 200_003, 17)
    got = su.speedup_amplitude(*args, precision="fp32", n_blocks=13)
    ref = su.speedup_amplitude(*args, precision="fp32", n_blocks=13, kernel="generic")
    for g, r in zip(got, ref):
        for key in ("amp", "log_amp", "err", "err_naive", "ess", "n"):
            assert g[key] == r[key], (r["level"], key)


@pytest.mark.parametrize("kw,expect_fixed", [
    ({"precision": "fp32"}, True),
    ({"precision": "fp32", "kernel": "generic"}, False),
    ({"precision": "fp64"}, False),                       # double: FP64-pipe bound, generic
    ({"precision": "fp32", "seg_log2": 4}, False),        # 16-slice segments
    ({"precision": "fp32", "width_factor": 2 ** 0.5}, False),
])
def test_plan_reports_the_sampler_it_launches(kw, expect_fixed):
    pl = su.Plan("aho", [1.0, 10.0], 0.0, 1.0, 1.0, 10, 10, 1000, 1, **kw)
    assert (pl.su_plan_kernel() >= 0) == expect_fixed
    assert su.Plan("mpt", [3.0, 1.0], 0.0, 1.0, 1.0, 10, 10, 1000, 1, precision="fp32").su_plan_kernel() == -1


def _batch(inst, p, kernel, **kw):
    pl = su.BatchPlan("aho", [1.0, 1.0], p, inst, 20_011, 9, precision="fp32", n_blocks=7, kernel=kernel, **kw)
    t = torch.empty(pl.tuple_bytes // 8, dtype=torch.float64, device="cuda")
    sc = torch.empty(pl.scratch_bytes, dtype=torch.uint8, device="cuda")
    pl.su_batch_plan_execute(t, sc)
    torch.cuda.synchronize()
    return pl.su_batch_plan_kernel(), pl.su_batch_plan_finalize(t.cpu().numpy(), sc)


def test_batched_kernel_with_the_shape_compiled_in_gives_the_generic_bits():
    # one level p: the compiled shape; depths 2..8 (segments of 4..32 slices),
    # the top level only and every level
    inst = [(-1.0 + 0.3 * i, 0.5 - 0.2 * i, (0.25, 0.5, 1.0, 2.0)[i % 4], 2 + i % 7) for i in range(21)]
    inst += [{"a": 0.2, "b": -0.4, "T": 1.0, "s": 8, "hierarchy": 1}, {"a": 0.0, "b": 1.0, "T": 0.5, "s": 6,
                                                                        "hierarchy": 1}]
    k_auto, got = _batch(inst, 12, "auto")
    k_gen, ref = _batch(inst, 12, "generic")
    assert k_auto == su.su_fixed_shape("aho", [1.0, 1.0], 12) and k_gen == -1
    flat = lambda res: [lev for x in res for lev in (x if isinstance(x, list) else [x])]  # noqa: E731
    got, ref = flat(got), flat(ref)
    assert len(got) == len(ref) == 21 + 9 + 7
    for g, r in zip(got, ref):
        for key in ("amp", "log_amp", "err", "err_naive", "ess", "n"):
            assert g[key] == r[key] or (np.isnan(g[key]) and np.isnan(r[key])), key


def test_batched_levels_p_each_with_their_compiled_shape_give_the_generic_bits():
    # levels 4 and 10 (two compiled-shape kernels) and 21 (beyond the compiled
    # shapes: the generic kernel) in one plan
    inst = [{"a": -0.5 + 0.1 * i, "b": 0.8 - 0.05 * i, "T": (0.5, 1.0)[i % 2], "s": 3 + i % 6, "p": (4, 10, 21)[i % 3],
             "hierarchy": i % 2} for i in range(18)]
    k_auto, got = _batch(inst, 10, "auto")
    k_gen, ref = _batch(inst, 10, "generic")
    assert k_auto == -2 and k_gen == -1
    flat = lambda res: [lev for x in res for lev in (x if isinstance(x, list) else [x])]  # noqa: E731
    got, ref = flat(got), flat(ref)
    assert len(got) == len(ref)
    for g, r in zip(got, ref):
        for key in ("amp", "log_amp", "err", "err_naive", "ess", "n"):
            assert g[key] == r[key] or (np.isnan(g[key]) and np.isnan(r[key])), key


def test_batched_levels_without_a_compiled_shape_stay_generic():
    pl = su.BatchPlan("poly", [0.2, -0.5, 0.3, 0.25, 0.1], 5, [(0.0, 0.5, 1.0, 6), (0.1, -0.2, 0.5, 4)], 1000, 3,
                      precision="fp32")
    assert pl.su_batch_plan_kernel() == -1
    one = su.BatchPlan("aho", [1.0, 1.0], 7, [(0.0, 0.5, 1.0, 6)], 1000, 3, precision="fp32")
    assert one.su_batch_plan_kernel() == su.su_fixed_shape("aho", [1.0, 1.0], 7)
