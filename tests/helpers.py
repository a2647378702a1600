"""Test helpers: random symmetric structures for brute-force pins. Builds inputs only."""
import numpy as np

import workloads as W


def random_legs(rng, mods, rank, max_sectors=3, max_dim=3):
    """Random legs for the given symmetry: a few charges per leg, small dimensions."""
    nsym = len(mods)
    legs = []
    for _ in range(rank):
        avail = 1
        for m in mods:
            avail *= m if m else 5
        ns = int(rng.integers(1, min(max_sectors, avail) + 1))
        charges = set()
        while len(charges) < ns:
            q = []
            for m in mods:
                q.append(int(rng.integers(0, m)) if m else int(rng.integers(-2, 3)))
            charges.add(tuple(q))
        ts = sorted(charges)
        ds = [int(rng.integers(1, max_dim + 1)) for _ in ts]
        legs.append(W.Leg(int(rng.choice([-1, 1])), ts, ds))
    return legs


def random_pair(rng, mods, rankA, rankB, ncon, **kw):
    """Random A, B whose first ``ncon`` legs of B are dual to ``ncon`` random legs of A."""
    legsA = random_legs(rng, mods, rankA, **kw)
    axa = tuple(int(a) for a in rng.permutation(rankA)[:ncon])
    legsB = random_legs(rng, mods, rankB, **kw)
    axb = tuple(int(b) for b in rng.permutation(rankB)[:ncon])
    for a, b in zip(axa, axb):
        legsB[b] = legsA[a].conj()
    nA = tuple(int(rng.integers(0, m)) if m else int(rng.integers(-1, 2)) for m in mods)
    nB = tuple(int(rng.integers(0, m)) if m else int(rng.integers(-1, 2)) for m in mods)
    seed = int(rng.integers(1 << 30))
    A = W.random_tensor(mods, legsA, nA, seed)
    B = W.random_tensor(mods, legsB, nB, seed + 1)
    return A, B, axa, axb, legsA, legsB


def leg_map(leg):
    return {q: d for q, d in zip(leg.t, leg.D)}
