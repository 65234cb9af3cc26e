"""Sharded runs on CPU ranks (gloo, world size 2) and host-side failure paths.

The sharding helpers of paper_1105_0542_gb300.distributed split the samples
into contiguous per-rank ranges and all-gather the per-block log-sum-exp
tuples.  Per-rank tuples are formed here from the oracle's per-sample weights
(the GPU forms them the same way); the gathered set must reproduce the
single-run estimate exactly.
"""
import math
import os
import socket

import numpy as np
import pytest

import paper_1105_0542_gb300 as su
from paper_1105_0542_gb300 import distributed as sd
from oracle import mc

torch = pytest.importorskip("torch")

MODEL, PARAMS, A, B, T, P, S, SEED = "aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 1234


def _tuples(w, n_blocks):
    """(n_blocks, levels, 4) log-sum-exp tuples of contiguous sample blocks."""
    out = []
    for lo, hi in mc.block_bounds(w.shape[0], n_blocks):
        x = w[lo:hi]
        m = x.max(axis=0)
        e = np.exp(x - m)
        out.append(np.stack([m, e.sum(0), (e * e).sum(0), np.full(m.shape, hi - lo, dtype=float)], axis=1))
    return np.stack(out)


def _estimate_from_tuples(tup):
    M = tup[:, :, 0].max(axis=0)
    f = np.exp(tup[:, :, 0] - M)
    Ssum = (tup[:, :, 1] * f).sum(axis=0)
    mu = tup[:, :, 1] * f / tup[:, :, 3]
    return Ssum / tup[:, :, 3].sum(axis=0), M, mu.std(axis=0, ddof=1) / math.sqrt(tup.shape[0])


def _rank_main(rank, world, port, n_mc, blocks_per_rank, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s0, n = sd.shard_range(n_mc, rank, world)
    w, _ = mc.Oracle(MODEL, PARAMS, P).logweights(A, B, T, S, SEED, n, sample0=s0)
    merged = sd.gather_block_tuples(_tuples(w, blocks_per_rank))
    if rank == 0:
        q.put(merged)
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_ranges_partition_the_samples():
    for n in (1, 7, 1000, 10_000_001):
        for world in (1, 2, 3, 8):
            parts = [sd.shard_range(n, r, world) for r in range(world)]
            assert parts[0][0] == 0
            assert sum(k for _, k in parts) == n
            for (a0, k0), (a1, _) in zip(parts, parts[1:]):
                assert a0 + k0 == a1


def test_two_gloo_ranks_reproduce_the_single_run():
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    n_mc, bpr, world = 4000, 5, 2
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n_mc, bpr, q)) for r in range(world)]
    for p_ in procs:
        p_.start()
    merged = q.get(timeout=120)
    for p_ in procs:
        p_.join(timeout=60)
        assert p_.exitcode == 0
    w, _ = mc.Oracle(MODEL, PARAMS, P).logweights(A, B, T, S, SEED, n_mc)
    whole = _tuples(w, world * bpr)
    assert merged.shape == whole.shape
    np.testing.assert_allclose(merged, whole, rtol=1e-15, atol=0)
    mean_m, M_m, err_m = _estimate_from_tuples(merged)
    ref = mc.estimate(w, 0.0, A, B, T, world * bpr)
    for lev in range(1, S + 1):
        assert mean_m[lev - 1] * math.exp(M_m[lev - 1] + mc.log_A_free(A, B, T)) == pytest.approx(
            ref[lev]["amp"], rel=1e-12)
        assert err_m[lev - 1] * math.exp(M_m[lev - 1] + mc.log_A_free(A, B, T)) == pytest.approx(
            ref[lev]["err"], rel=1e-9)


@pytest.mark.parametrize("params,prec", [([0.0, 0.0, 1e300, 0.0, 1e300], "fp32"),
                                         ([0.0, 0.0, 1e300, 0.0, 1e300], "fp64"),
                                         ([1e200, 1e200], "fp64")])
def test_non_finite_coefficients_fail_loudly(params, prec):
    model = "poly" if len(params) > 2 else "aho"
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_amplitude(model, params, 0.0, 1.0, 1.0, 6, 4, 100, 1, precision=prec)
    assert e.value.code == -5
