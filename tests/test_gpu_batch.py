"""GPU parity of the batched persistent path (many (a, b, T, s, p, n_mc)
instances in one graph-replayed launch) against the oracle and the
single-instance path.

Instance i of a batch draws from Philox stream (opt.instance + i); its
amplitudes (the top level, or every level of the hierarchy) must equal the
oracle's estimator on the same samples, and the single-instance entry point
run with that stream id, whatever level p, sample count and register segment
each instance has.  The full-size
amplitude matrix (256 x 256 endpoints over [-5, 5], T and s drawn per
instance, p = 10, 1e5 samples, single-precision W_p) is checked on sampled
instances one by one and through the symmetries A(a,b) = A(b,a) and
A(a,b) = A(-a,-b) of an even potential.
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1105_0542_gb300 as su  # noqa: E402
import workloads  # noqa: E402
from oracle import mc  # noqa: E402

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    torch.cuda.set_device(0)


def _small_batch(n, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        out.append((float(rng.uniform(-3, 3)), float(rng.uniform(-3, 3)),
                    float(rng.choice([0.25, 0.5, 1.0, 2.0])), int(rng.integers(0, 9))))
    return out


@pytest.mark.parametrize("prec,bits,tol", [("fp64", 53, 1e-10), ("fp32", 24, 1e-4)])
def test_batch_equals_oracle_estimator_per_instance(prec, bits, tol):
    inst = _small_batch(24)
    n_mc, nb, seed, p = 1500, 4, 11, 10
    res = su.speedup_amplitude_batch("aho", [1.0, 1.0], p, inst, n_mc, seed, precision=prec, n_blocks=nb,
                                     instance=100)
    o = mc.Oracle("aho", [1.0, 1.0], p)
    for i, (a, b, T, s) in enumerate(inst):
        if s == 0:
            ref = mc.estimate(np.zeros((n_mc, 0)), o.level0(a, b, T), a, b, T, nb)[0]
        else:
            w, _ = o.logweights(a, b, T, s, seed, n_mc, instance=100 + i, bits=bits, threads=THREADS)
            ref = mc.estimate(w, o.level0(a, b, T), a, b, T, nb)[s]
        g = res[i]
        assert g["n"] == n_mc
        assert abs(g["log_amp"] - ref["log_amp"]) <= tol, (i, s)
        if s:
            assert abs(g["err"] - ref["err"]) <= 100 * tol * ref["err"], i


def test_batch_equals_single_instance_path():
    inst = [(0.3, -1.2, 1.0, 8), (-2.0, 2.5, 0.25, 2), (1.0, 1.0, 2.0, 6), (0.0, 0.5, 0.5, 5)]
    res = su.speedup_amplitude_batch("aho", [1.0, 1.0], 10, inst, 20000, 5, n_blocks=8)
    for i, (a, b, T, s) in enumerate(inst):
        one = su.speedup_amplitude("aho", [1.0, 1.0], a, b, T, 10, s, 20000, 5, n_blocks=8, hierarchy=False,
                                   instance=i)
        assert res[i]["amp"] == pytest.approx(one[s]["amp"], rel=1e-12)
        assert res[i]["err"] == pytest.approx(one[s]["err"], rel=1e-9)


def test_graph_replay_is_deterministic():
    inst = _small_batch(300, seed=9)
    pl = su.BatchPlan("aho", [1.0, 1.0], 10, inst, 3000, 2, precision="fp32", n_blocks=6)
    t = torch.empty(pl.tuple_bytes // 8, dtype=torch.float64, device="cuda")
    sc = torch.empty(pl.scratch_bytes, dtype=torch.uint8, device="cuda")
    outs = []
    for _ in range(3):
        assert pl.su_batch_plan_execute(t, sc) == 1
        torch.cuda.synchronize()
        outs.append(t.cpu().numpy().copy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    res = pl.su_batch_plan_finalize(outs[0], sc)
    assert all(math.isfinite(r["log_amp"]) for r in res)


def test_full_amplitude_matrix():
    """The 65,536-instance amplitude matrix in one launch (the workload of the
    batched benchmark entry)."""
    inst = workloads.config3()
    tup = [(x.a, x.b, x.T, x.s) for x in inst]
    n_mc, nb, seed = inst[0].n_mc, inst[0].n_blocks, inst[0].seed
    pl = su.BatchPlan("aho", [1.0, 1.0], 10, tup, n_mc, seed, precision="fp32", n_blocks=nb)
    t = torch.empty(pl.tuple_bytes // 8, dtype=torch.float64, device="cuda")
    sc = torch.empty(pl.scratch_bytes, dtype=torch.uint8, device="cuda")
    pl.su_batch_plan_execute(t, sc)
    torch.cuda.synchronize()
    res = pl.su_batch_plan_finalize(t.cpu().numpy(), sc)
    assert len(res) == 256 * 256
    # sampled instances, one by one through the single-instance path (same stream)
    for k in (0, 1, 257, 12345, 40000, 65535):
        x = inst[k]
        one = su.speedup_amplitude("aho", [1.0, 1.0], x.a, x.b, x.T, 10, x.s, n_mc, seed, precision="fp32",
                                   n_blocks=nb, hierarchy=False, instance=k)
        assert res[k]["log_amp"] == pytest.approx(one[x.s]["log_amp"], abs=1e-6)
    # symmetries of the even potential where the two instances share T and s
    n = 256
    checked = 0
    for i in range(0, n, 17):
        for j in range(0, n, 13):
            for (i2, j2) in ((j, i), (n - 1 - i, n - 1 - j)):
                a, b = inst[i * n + j], inst[i2 * n + j2]
                if (a.T, a.s) != (b.T, b.s) or (i, j) == (i2, j2):
                    continue
                ra, rb = res[i * n + j], res[i2 * n + j2]
                sig = math.hypot(ra["err"], rb["err"])
                assert abs(ra["amp"] - rb["amp"]) <= 5 * sig + 1e-300, (i, j, i2, j2)
                checked += 1
    assert checked > 10


def _mixed_batch(seed=17):
    """p = 1..18, depths 0..8, uneven sample counts, every third instance
    with the hierarchy."""
    rng = np.random.default_rng(seed)
    out = []
    for i, p in enumerate(list(range(1, 19)) + [10, 4, 18, 1]):
        out.append((float(rng.uniform(-2, 2)), float(rng.uniform(-2, 2)), float(rng.choice([0.25, 0.5, 1.0])),
                    int(rng.integers(0, 9)), p, int(rng.integers(300, 2500)), i % 3 == 0))
    return out


@pytest.mark.parametrize("prec,bits,tol", [("fp64", 53, 1e-10), ("fp32", 24, 1e-4)])
def test_mixed_p_batch_equals_oracle_per_instance(prec, bits, tol):
    inst = _mixed_batch()
    nb, seed = 5, 21
    res = su.speedup_amplitude_batch("aho", [1.0, 1.0], 10, inst, 1000, seed, precision=prec, n_blocks=nb,
                                     instance=40)
    for i, (a, b, T, s, p, n, hier) in enumerate(inst):
        o = mc.Oracle("aho", [1.0, 1.0], p)
        w, _ = o.logweights(a, b, T, s, seed, n, instance=40 + i, bits=bits, threads=THREADS)
        ref = mc.estimate(w, o.level0(a, b, T), a, b, T, nb)
        got = res[i] if hier else [None] * s + [res[i]]
        assert len(got) == s + 1
        for lev in (range(s + 1) if hier else [s]):
            g, r = got[lev], ref[lev]
            assert g["n"] == n and g["level"] == lev
            assert abs(g["log_amp"] - r["log_amp"]) <= tol, (i, p, s, lev)
            if lev:
                assert abs(g["err"] - r["err"]) <= 100 * tol * r["err"], (i, p, s, lev)


def test_convergence_sweep_as_one_batched_launch():
    """The convergence sweep (AHO g = 10, T = 1, a = 0, b = 1, s = 10, every
    level of the hierarchy, p = 1..18) as one launch: each instance equals the
    single-instance plan on the same stream at every level (the reductions
    differ in order only)."""
    x = workloads.config2(1)
    n = 20_000
    inst = [(x.a, x.b, x.T, x.s, p, n, 1) for p in range(1, 19)]
    for prec, tol in (("fp64", 1e-11), ("fp32", 1e-5)):
        pl = su.BatchPlan(x.model, list(x.params), 1, inst, n, x.seed, precision=prec, n_blocks=20)
        t = torch.empty(pl.tuple_bytes // 8, dtype=torch.float64, device="cuda")
        sc = torch.empty(pl.scratch_bytes, dtype=torch.uint8, device="cuda")
        assert pl.su_batch_plan_execute(t, sc) == 1
        torch.cuda.synchronize()
        res = pl.su_batch_plan_finalize(t.cpu().numpy(), sc)
        assert pl.n_results == 18 * (x.s + 1)
        assert pl.slice_actions == 18 * n * (2 * 2 ** x.s - 2)
        for i, p in enumerate(range(1, 19)):
            one = su.speedup_amplitude(x.model, list(x.params), x.a, x.b, x.T, p, x.s, n, x.seed, precision=prec,
                                       n_blocks=20, instance=i)
            for lev in range(x.s + 1):
                assert res[i][lev]["log_amp"] == pytest.approx(one[lev]["log_amp"], abs=tol), (prec, p, lev)
                assert res[i][lev]["n"] == n


def test_batch_autotuner_chooses_and_reports_shapes():
    inst = [(0.2 * k, -0.1 * k, 0.5, s, p, 3000, h) for k, (s, p, h) in
            enumerate([(8, 10, 0), (8, 10, 0), (6, 4, 1), (6, 4, 1), (3, 18, 0)])]
    su.su_autotune_clear()
    base = su.BatchPlan("aho", [1.0, 1.0], 10, inst, 3000, 9, precision="fp64", n_blocks=6)
    assert [base.su_batch_plan_shape(i) [0] for i in range(len(inst))] == [4, 4, 4, 4, 3]   # the rule
    assert all(base.su_batch_plan_shape(i)[2] == 0 for i in range(len(inst)))
    got = su.su_batch_autotune("aho", [1.0, 1.0], 10, inst, 3000, 9, max_probe=2, precision="fp64", n_blocks=6)
    assert sorted((g["p"], g["s"], g["hierarchy"]) for g in got) == [(4, 6, 1), (10, 8, 0), (18, 3, 0)]
    assert all(1 <= g["seg_log2"] <= min(g["s"], 5) and g["ns_per_slice"] > 0 for g in got)
    tuned = su.BatchPlan("aho", [1.0, 1.0], 10, inst, 3000, 9, precision="fp64", n_blocks=6)
    pick = {(g["p"], g["s"], g["hierarchy"]): g["seg_log2"] for g in got}
    for i, (a, b, T, s, p, n, h) in enumerate(inst):
        f, k, fr = tuned.su_batch_plan_shape(i)
        assert fr == 1 and f == pick[(p, s, h)] and k >= 1
    res = []
    for pl in (base, tuned):
        t = torch.empty(pl.tuple_bytes // 8, dtype=torch.float64, device="cuda")
        sc = torch.empty(pl.scratch_bytes, dtype=torch.uint8, device="cuda")
        pl.su_batch_plan_execute(t, sc)
        torch.cuda.synchronize()
        res.append(pl.su_batch_plan_finalize(t.cpu().numpy(), sc))
    flat = lambda r: [x for y in r for x in (y if isinstance(y, list) else [y])]  # noqa: E731
    for g, r in zip(flat(res[1]), flat(res[0])):
        assert g["amp"] == pytest.approx(r["amp"], rel=1e-12)
    su.su_autotune_clear()
    again = su.BatchPlan("aho", [1.0, 1.0], 10, inst, 3000, 9, precision="fp64", n_blocks=6)
    assert all(again.su_batch_plan_shape(i)[2] == 0 for i in range(len(inst)))
