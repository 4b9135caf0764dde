"""Per-network query counts for the grouped (many-bodies) workload."""

import numpy as np

from .rng import Stream


def grouped_counts(n_nets=16, seed=1234, lo=2000, hi=400000):
    """floor(exp(U(ln lo, ln hi))) per network: a log-uniform spread of sizes."""
    s = Stream(seed, tag=301)
    u = s.uniform(n_nets, np.log(lo), np.log(hi))
    return np.floor(np.exp(u)).astype(np.int64)
