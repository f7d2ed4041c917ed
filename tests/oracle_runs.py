"""Oracle disk evolutions for the statistical tests, one per worker process
(test infrastructure: it imports only the oracle and numpy, so spawned
workers start quickly)."""
import numpy as np

import oracle


def evolve(P, grid, seed, disk, dt, steps, edges):
    """One disk from the oracle's initial state through `steps` steps of dt;
    returns (status, m, M, r, per-bin sums, accreted mass, initial swarm mass)."""
    N = grid[0] * grid[1] * grid[2]
    s = oracle.init_disk(P, N, seed=seed, disk=disk)
    M0 = float(s.M.sum())
    st = oracle.run(P, grid[0], grid[1], s, 0.0, dt, 0, steps, seed=seed, disk=disk, nthreads=1)
    return st, s.m, s.M, s.r, oracle.moments(s.m, s.M, s.r, np.asarray(edges)), s.accreted, M0
