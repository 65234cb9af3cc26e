"""The seeded synthetic workloads have the shapes the input recipe states
(CPU only): the small case, the convergence sweep, the amplitude matrix,
the double-well / Poeschl-Teller set and the learned-proposal instance."""
import numpy as np

import workloads as wl


def test_small_case_and_sweep():
    assert [(i.model, i.params, i.p, i.s, i.n_mc, i.n_blocks) for i in wl.CONFIG1] == [
        ("aho", (1.0, 1.0), 4, 4, 100_000, 10), ("ho", (1.0,), 4, 4, 100_000, 10)]
    assert wl.CONFIG2_P == tuple(range(1, 19))
    for p in wl.CONFIG2_P:
        i = wl.config2(p)
        assert (i.model, i.params, i.a, i.b, i.T, i.p, i.s, i.n_mc, i.n_blocks) == \
            ("aho", (1.0, 10.0), 0.0, 1.0, 1.0, p, 10, 10_000_000, 100)
    # one s = 10 run per (p, precision): 1e7 x (2^11 - 2) hierarchy slice-actions
    assert wl.CONFIG2_NMC * (2 * 2 ** wl.CONFIG2_S - 2) == 20_460_000_000


def test_amplitude_matrix():
    inst = wl.config3()
    assert len(inst) == 65_536
    assert sorted(i.instance for i in inst) == list(range(65_536))
    grid = np.linspace(-5.0, 5.0, 256)
    assert {i.a for i in inst} == set(grid.tolist()) and {i.b for i in inst} == set(grid.tolist())
    assert {i.T for i in inst} == {0.25, 0.5, 1.0, 2.0}
    s = np.array([i.s for i in inst])
    assert set(s.tolist()) == set(range(2, 9))
    freq = np.bincount(s, minlength=9)[2:] / len(s)
    assert np.all(np.abs(freq - 1 / 7) < 0.01)
    assert all(i.p == 10 and i.n_mc == 100_000 and i.model == "aho" for i in inst)
    # top-level slice-actions: E[N] = 508/7 per sample, about 4.8e11 in all
    total = sum(i.n_mc * 2 ** i.s for i in inst)
    assert abs(total / (65_536 * 100_000 * 508 / 7) - 1) < 0.02
    # the same seed gives the same matrix
    assert [(i.T, i.s) for i in wl.config3()[:100]] == [(i.T, i.s) for i in inst[:100]]


def test_double_well_and_poeschl_teller_set_and_proposal_instance():
    c4 = wl.config4()
    assert [(i.model, i.params, i.T) for i in c4] == [
        ("dw", (1.0,), 1.0), ("dw", (5.0,), 1.0), ("mpt", (3.0, 1.0), 1.0),
        ("dw", (1.0,), 5.0), ("dw", (5.0,), 5.0), ("mpt", (3.0, 1.0), 5.0)]
    assert all((i.a, i.b, i.p, i.s, i.n_mc) == (-1.0, 1.0, 12, 6, 100_000_000) for i in c4)
    c5 = wl.CONFIG5
    assert (c5.model, c5.params, c5.a, c5.b, c5.T, c5.p, c5.s, c5.n_mc) == \
        ("dw", (5.0,), -1.0, 1.0, 5.0, 12, 6, 10_000_000)
