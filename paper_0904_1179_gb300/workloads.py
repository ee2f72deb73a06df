"""Seeded synthetic workloads (inputs only; no arithmetic of the method).

The paper's workloads are Monte Carlo chains started from generated
configurations at beta = 5.7 on 8^4 ... 32^4 lattices (Berg & Wu, Sec. 2.1,
Table 1: 512 / 101 / 32 / 2 sweeps, chosen so every column is the same
number of link updates), so these recipes are the workloads themselves, not
stand-ins for a dataset.
"""

BETA = 5.7

# Table 1 of the paper: lattice and sweep count per column (same number of link updates).
TABLE1 = [((8, 8, 8, 8), 512), ((12, 12, 12, 12), 101), ((16, 16, 16, 16), 32), ((32, 32, 32, 32), 2)]

# Headline: the 32^4 column, hot start from Philox seed 7.
HEADLINE_DIMS = (32, 32, 32, 32)
HEADLINE_SEED = 7
HEADLINE_SWEEPS_PER_STEP = 2

# Cold-start smoke case: 4^4, seed 1, 20 sweeps with the plaquette after each.
SMOKE_DIMS = (4, 4, 4, 4)
SMOKE_SEED = 1
SMOKE_SWEEPS = 20


def batch_96():
    """96 replicas of uneven extents: 32x 8^4, 32x 12^4, 16x 16^4, 16x 8^3x16;
    beta_r = 5.5 + 0.7 (r + 1/2)/96 spread evenly over [5.5, 6.2]; seed_r = 1000 + r;
    hot starts, FP32-mixed."""
    dims = [(8, 8, 8, 8)] * 32 + [(12, 12, 12, 12)] * 32 + [(16, 16, 16, 16)] * 16 + [(8, 8, 8, 16)] * 16
    betas = [5.5 + 0.7 * (r + 0.5) / 96 for r in range(96)]
    seeds = [1000 + r for r in range(96)]
    return dims, betas, seeds


def updates_per_sweep(dims):
    n = 0
    for L in dims:
        v = 1
        for x in L:
            v *= x
        n += 4 * v
    return n
