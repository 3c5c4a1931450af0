"""Seeded synthetic raw-candidate lists for the merge tests.

A raw candidate is (trial index, width index, boxcar start, exact boxcar sum);
with the per-trial sigmas it is the input of candidate merging (Section II-B,
"Candidate Merging and Clustering").  The lists here imitate what a search
over many trials finds: clusters around bright pulses spread over neighbouring
trials, times and widths, on top of isolated noise detections, appended in no
particular order.  This module only draws numbers; it holds none of the
merge's arithmetic, so the oracle and the CUDA merge can both be fed from it.
"""
from __future__ import annotations

import numpy as np

RAW_FIELDS = (("dm_idx", "<i4"), ("width_idx", "<i4"), ("sample", "<i8"), ("S", "<i8"))
RAW_DTYPE = np.dtype(list(RAW_FIELDS))


def raw_list(seed: int, n: int, ndm: int, nout: int, nw: int, cluster_frac: float = 0.7,
             members: tuple = (20, 400), dm_spread: int = 12, t_spread: int = 300):
    """About ``n`` raw candidates with unique (trial, start, width) keys.

    ``cluster_frac`` of them sit in clusters: each cluster has a centre trial,
    start and width, and members drawn within +-``dm_spread`` trials,
    +-``t_spread`` samples and +-2 width indices of it; the rest are uniform
    over trials, starts and widths.  Sums S are integers in [40, 4000] and the
    per-trial sigmas floats in [2, 20], so S / (sigma sqrt(W)) stays below
    ~2000.  Returns (raw records in a shuffled order, sigma[ndm])."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 77])))
    n_cl = int(n * cluster_frac)
    sizes = []
    while sum(sizes) < n_cl:
        sizes.append(int(rng.integers(members[0], members[1] + 1)))
    k = len(sizes)
    c_dm = rng.integers(0, ndm, k)
    c_t = rng.integers(0, nout, k)
    c_w = rng.integers(0, nw, k)
    rep = np.repeat(np.arange(k), sizes)
    dm = np.clip(c_dm[rep] + rng.integers(-dm_spread, dm_spread + 1, rep.size), 0, ndm - 1)
    t = np.clip(c_t[rep] + rng.integers(-t_spread, t_spread + 1, rep.size), 0, nout - 1)
    w = np.clip(c_w[rep] + rng.integers(-2, 3, rep.size), 0, nw - 1)
    m = max(0, n - rep.size)
    dm = np.concatenate([dm, rng.integers(0, ndm, m)])
    t = np.concatenate([t, rng.integers(0, nout, m)])
    w = np.concatenate([w, rng.integers(0, nw, m)])
    key = (dm.astype(np.int64) * nout + t) * nw + w
    _, first = np.unique(key, return_index=True)
    first = rng.permutation(first)
    out = np.zeros(first.size, RAW_DTYPE)
    out["dm_idx"] = dm[first]
    out["width_idx"] = w[first]
    out["sample"] = t[first]
    out["S"] = rng.integers(40, 4001, first.size)
    sigma = rng.uniform(2.0, 20.0, ndm)
    return out, sigma
