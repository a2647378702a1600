"""Test helpers: random symmetric structures for brute-force pins, and inputs built
with the oracle's fuse (fused tensors with chosen fusion histories). Builds inputs only."""
import numpy as np

import oracle as O
import workloads as W


def random_legs(rng, mods, rank, max_sectors=3, max_dim=3):
    """Random legs for the given symmetry: a few charges per leg, small dimensions.
    U(1) components range over -2..2 alone and over -1..1 in product groups (so that
    blocks of several legs still meet often)."""
    nsym = len(mods)
    span = 2 if nsym == 1 else 1
    legs = []
    for _ in range(rank):
        avail = 1
        for m in mods:
            avail *= m if m else 2 * span + 1
        ns = int(rng.integers(1, min(max_sectors, avail) + 1))
        charges = set()
        while len(charges) < ns:
            q = []
            for m in mods:
                q.append(int(rng.integers(0, m)) if m else int(rng.integers(-span, span + 1)))
            charges.add(tuple(q))
        ts = sorted(charges)
        ds = [int(rng.integers(1, max_dim + 1)) for _ in ts]
        legs.append(W.Leg(int(rng.choice([-1, 1])), ts, ds))
    return legs


def random_pair(rng, mods, rankA, rankB, ncon, dtype="f64", **kw):
    """Random A, B whose first ``ncon`` legs of B are dual to ``ncon`` random legs of A
    (``dtype`` "f64" or "c128" for both)."""
    legsA = random_legs(rng, mods, rankA, **kw)
    axa = tuple(int(a) for a in rng.permutation(rankA)[:ncon])
    legsB = random_legs(rng, mods, rankB, **kw)
    axb = tuple(int(b) for b in rng.permutation(rankB)[:ncon])
    for a, b in zip(axa, axb):
        legsB[b] = legsA[a].conj()
    nA = tuple(int(rng.integers(0, m)) if m else int(rng.integers(-1, 2)) for m in mods)
    nB = tuple(int(rng.integers(0, m)) if m else int(rng.integers(-1, 2)) for m in mods)
    seed = int(rng.integers(1 << 30))
    A = W.random_tensor(mods, legsA, nA, seed, dtype=dtype)
    B = W.random_tensor(mods, legsB, nB, seed + 1, dtype=dtype)
    return A, B, axa, axb, legsA, legsB


def leg_map(leg):
    return {q: d for q, d in zip(leg.t, leg.D)}


def fusion_mismatch_pair(drop_a=1, drop_b=None, seed=0):
    """A = fuse(T_A, (0, 1), (2,)) and B = fuse(T_B, (0, 1), (2,)) on dual constituent
    legs, where T_A lacks every block with charge ``drop_a`` on its leg 0 (and T_B those
    with ``drop_b``), so the two fusion records of the contracted fused leg differ.
    Returns A, B and the zero-padded A_pad, B_pad whose records are the union."""
    l0 = W.Leg(1, [(-1,), (0,), (1,)], [2, 3, 1])
    l1 = W.Leg(1, [(0,), (1,)], [2, 2])
    l2 = W.Leg(-1, [(-1,), (0,), (1,), (2,)], [1, 2, 2, 1])
    l3 = W.Leg(1, [(-1,), (0,), (1,), (2,)], [2, 1, 3, 1])
    TA = O.from_record(W.random_tensor((0,), [l0, l1, l2], (0,), 11 + seed))
    TB = O.from_record(W.random_tensor((0,), [l0.conj(), l1.conj(), l3], (0,), 12 + seed))

    def drop(T, q):
        keep = {k: v for k, v in T.blocks.items() if q is None or k[0] != (q,)}
        pad = {k: (v if q is None or k[0] != (q,) else np.zeros_like(v)) for k, v in T.blocks.items()}
        return O.OTensor(T.mods, T.sig, T.n, keep), O.OTensor(T.mods, T.sig, T.n, pad)

    a, a_pad = drop(TA, drop_a)
    b, b_pad = drop(TB, drop_b)
    g = ((0, 1), (2,))
    return O.fuse(a, g), O.fuse(b, g), O.fuse(a_pad, g), O.fuse(b_pad, g), a, b


def random_network(rng, mods, kind):
    """A random network: legs, tensors and ncon labels. kind: 'chain' (three tensors
    in a loop), 'trace' (a tensor with a traced pair), 'outer' (two disconnected
    pieces)."""
    # small charges so that the blocks of neighbouring tensors meet
    pool = {(0,): [(-1,), (0,), (1,)], (2,): [(0,), (1,)],
            (0, 0): [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, -1)]}[tuple(mods)]
    L = []
    for _ in range(7):
        k = int(rng.integers(2, len(pool) + 1))
        qs = sorted(pool[int(i)] for i in rng.choice(len(pool), size=k, replace=False))
        L.append(W.Leg(int(rng.choice([-1, 1])), qs, [int(d) for d in rng.integers(1, 4, size=k)]))
    n0 = (0,) * len(mods)
    if kind == "chain":
        legs = [[L[0], L[1], L[2]], [L[1].conj(), L[3], L[4]], [L[2].conj(), L[4].conj(), L[5]]]
        labels = [[-1, 1, 2], [1, -2, 3], [2, 3, -3]]
    elif kind == "trace":
        legs = [[L[0], L[1], L[1].conj(), L[2]], [L[2].conj(), L[3]]]
        labels = [[-2, 5, 5, 1], [1, -1]]
    else:
        legs = [[L[0], L[1]], [L[1].conj(), L[2]], [L[3], L[4]]]
        labels = [[-3, 1], [1, -1], [-2, -4]]
    ts = [W.random_tensor(mods, lg, n0, 100 + k) for k, lg in enumerate(legs)]
    return legs, ts, labels
