"""Seeded synthetic workloads for the amplitude estimator.

This module only describes inputs: which potential, its parameters, the
endpoints a and b, the propagation time T, the effective-action level p,
the bisection depth s (N = 2^s time slices), the number of Monte Carlo
samples and blocks, and the seed.  It holds none of the method's
arithmetic; the tests, the benchmark and the oracle all read their inputs
from here.

The paper measures on no dataset; every workload is synthetic by
construction, with the shapes of the paper's own examples (a 1D anharmonic
oscillator V = A x^2/2 + g x^4/24, a double well, and the modified
Poeschl-Teller potential -lambda/cosh^2(alpha x), Sec. 3.3 and Sec. 4.2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MODELS = {"ho": 0, "aho": 1, "dw": 2, "mpt": 3, "poly": 4}


@dataclass(frozen=True)
class Instance:
    model: str
    params: tuple
    a: float
    b: float
    T: float
    p: int
    s: int
    n_mc: int
    seed: int = 1234
    n_blocks: int = 64
    instance: int = 0


# 1: anharmonic oscillator g = 1 and the harmonic oscillator, p = 4, N = 16,
#    1e5 samples in 10 blocks (the small case the oracle finishes in seconds).
CONFIG1 = [
    Instance("aho", (1.0, 1.0), 0.0, 1.0, 1.0, 4, 4, 100_000, 1234, 10),
    Instance("ho", (1.0,), 0.0, 1.0, 1.0, 4, 4, 100_000, 1234, 10),
]

# 2: convergence sweep, anharmonic oscillator g = 10, every p = 1..18 with one
#    s = 10 run (the hierarchy gives N = 1..1024), 1e7 samples in 100 blocks,
#    W_p in double and in single precision.
CONFIG2_P = tuple(range(1, 19))
CONFIG2_S = 10
CONFIG2_NMC = 10_000_000
CONFIG2_BLOCKS = 100


def config2(p, n_mc=CONFIG2_NMC):
    return Instance("aho", (1.0, 10.0), 0.0, 1.0, 1.0, p, CONFIG2_S, n_mc, 1234, CONFIG2_BLOCKS)


# 3: amplitude matrix, anharmonic oscillator g = 1, a and b on a 256 x 256
#    grid over [-5, 5], T per instance from {0.25, 0.5, 1, 2}, s per instance
#    from {2..8}, p = 10, 1e5 samples per instance.
def config3(n_side=256, n_mc=100_000, seed=1234, n_blocks=16):
    grid = np.linspace(-5.0, 5.0, n_side)
    rng = np.random.default_rng(seed)
    n = n_side * n_side
    Ts = rng.choice(np.array([0.25, 0.5, 1.0, 2.0]), size=n)
    ss = rng.integers(2, 9, size=n)
    out = []
    for i in range(n_side):
        for j in range(n_side):
            k = i * n_side + j
            out.append(Instance("aho", (1.0, 1.0), float(grid[i]), float(grid[j]), float(Ts[k]),
                                10, int(ss[k]), n_mc, seed, n_blocks, k))
    return out


# 4: double well V = h (q^2 - 1)^2, h in {1, 5}, and Poeschl-Teller
#    V = -l(l-1)/(2 cosh^2 q), l = 3 (lambda = 3, alpha = 1); T in {1, 5},
#    a = -1, b = 1, p = 12, N = 64, 1e8 samples.
def config4(n_mc=100_000_000):
    out = []
    for T in (1.0, 5.0):
        for h in (1.0, 5.0):
            out.append(Instance("dw", (h,), -1.0, 1.0, T, 12, 6, n_mc, 1234, 64))
        out.append(Instance("mpt", (3.0, 1.0), -1.0, 1.0, T, 12, 6, n_mc, 1234, 64))
    return out


# 5: the learned-proposal instance: double well h = 5, T = 5, p = 12, N = 64;
# n_mc = 1e7 is the number of plain paths the proposal is trained on.
CONFIG5 = Instance("dw", (5.0,), -1.0, 1.0, 5.0, 12, 6, 10_000_000, 1234, 64)

# The learned proposal where the bridge is a poor proposal but the truncated
# action is bounded below: the harmonic oscillator omega = 4 at T = 4
# (a = 0, b = 0.5, p = 4, N = 64); the bridge's per-sample relative variance
# is about 28.  n_mc = 1e7 plain paths to train on.
PROPOSAL_GAIN = Instance("ho", (4.0,), 0.0, 0.5, 4.0, 4, 6, 10_000_000, 2024, 50)
