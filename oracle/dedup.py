"""Grouping of duplicated samples into unique states with counts.  TEST INFRASTRUCTURE ONLY.

Scaling section of arXiv:2011.12453: after sampling, duplicated states are grouped into
unique states with counts before the data go to the workers; the ISGO weights then carry
log count_x (Eq. isgo with counts).

Output convention (fixed here, the paper does not give one): unique configurations in
the order of their first occurrence in the batch, each with the log Psi^0 of that first
occurrence and its number of copies.
"""
from __future__ import annotations

import numpy as np


def group(spins: np.ndarray, logpsi0: np.ndarray):
    """(unique spins [U][N], their log Psi^0 [U][...], counts float64 [U])."""
    spins = np.asarray(spins)
    first: dict[bytes, int] = {}
    order: list[int] = []
    counts: list[int] = []
    for x in range(spins.shape[0]):
        key = spins[x].tobytes()
        if key in first:
            counts[first[key]] += 1
        else:
            first[key] = len(order)
            order.append(x)
            counts.append(1)
    idx = np.array(order, dtype=np.int64)
    return spins[idx], np.asarray(logpsi0)[idx], np.array(counts, dtype=np.float64)
