"""Seeded synthetic inputs for block-sparse symmetric tensor contractions.

This module is shared by the CPU oracle (``oracle/``), the tests and ``bench.py``.
It holds no contraction, fusion or trace arithmetic. It only builds *inputs*:

* legs ``(s, t, D)`` -- a signature, a list of charge sectors and their dimensions
  (Sec. II.A, the ``Leg`` definition);
* random symmetric tensors with every block allowed by the block charge-conservation
  rule (Sec. II.A, block-sparse form of Eq. ``elemchargecon``) stored, the values drawn
  N(0,1) from NumPy's PCG64 in canonical block order (the analogue of the paper's
  ``rand(config, legs, n)``);
* the workload shapes of the paper's iPEPS / CTM examples (Sec. III, Fig. 3), with bond
  dimension D, environment dimension chi and the symmetry groups named there.

Data layout shared by every consumer (a plain-array "tensor record"):

``{"mods": (m_0..m_{k-1}), "sig": (s_0..s_{r-1}), "n": (n_0..n_{k-1}),
   "t": int32[nblocks, rank, nsym], "D": int64[nblocks, rank], "data": float64[size]}``

``mods[c] == 0`` means the c-th charge component is U(1) (an integer), ``mods[c] == m > 1``
means Z_m (an integer in [0, m)). Blocks are in canonical order: ascending lexicographic
order of the flattened (rank x nsym) charge tuple. Each block is dense and row-major
(C order) and the blocks are packed back to back in that order.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "Leg", "random_tensor", "record_size", "block_offsets",
    "config1", "config2", "config3", "config5", "config5b", "serving_runs",
    "double_layer_leg", "gaussian_sector_sizes", "random_composition",
]


class Leg:
    """A leg V(s, t, D): signature ``s`` (+1 or -1), charge sectors ``t`` (tuples of
    ``nsym`` integers) and their dimensions ``D`` (Sec. II.A, Leg definition)."""

    def __init__(self, s, t, D):
        if s not in (1, -1):
            raise ValueError("signature must be +1 or -1")
        t = [tuple(int(c) for c in (q if isinstance(q, (tuple, list)) else (q,))) for q in t]
        D = [int(d) for d in D]
        if len(t) != len(D):
            raise ValueError("t and D must have the same length")
        if len(set(t)) != len(t):
            raise ValueError("duplicate charge sector on a leg")
        order = sorted(range(len(t)), key=lambda i: t[i])
        self.s = int(s)
        self.t = [t[i] for i in order]
        self.D = [D[i] for i in order]

    @property
    def nsym(self):
        return len(self.t[0]) if self.t else 0

    @property
    def dim(self):
        return sum(self.D)

    def conj(self):
        """The dual leg: the signature is flipped (Sec. II.A, footnote on conjugation)."""
        return Leg(-self.s, self.t, self.D)

    def __repr__(self):
        return f"Leg(s={self.s}, t={self.t}, D={self.D})"


def _reduce(q, mods):
    return tuple((c % m) if m else c for c, m in zip(q, mods))


def random_tensor(mods, legs, n, seed, fill="normal", dtype="f64"):
    """A symmetric tensor with every charge-conserving block stored.

    A block (rho_1..rho_N) is allowed when sum_i s_i rho_i == n, component-wise and
    modulo ``mods[c]`` for Z_m components (Sec. II.A, block conservation rule). This
    rule defines which inputs are valid symmetric tensors; the oracle and the library
    each re-check it independently.

    ``fill``: "normal" draws N(0,1) (PCG64, ``default_rng(seed)``), "integer" draws
    integers uniform in [-8, 8] (exactly representable and exactly summable, used to
    test the split-precision path), "ones" fills with 1.0.
    ``dtype``: "f64", or "c128" (complex: real and imaginary parts drawn alike, as
    consecutive pairs of the same stream; the record gets ``dtype: "c128"`` and a
    complex128 data array, stored interleaved).
    """
    mods = tuple(int(m) for m in mods)
    nsym = len(mods)
    n = _reduce(tuple(n), mods)
    rank = len(legs)
    t, D = _allowed_blocks(mods, legs, n)
    size = int(np.prod(D, axis=1).sum()) if len(D) else 0
    rng = np.random.default_rng(seed)
    cplx = dtype == "c128"
    if dtype not in ("f64", "c128"):
        raise ValueError(dtype)
    m = 2 * size if cplx else size
    if fill == "normal":
        data = rng.standard_normal(m)
    elif fill == "integer":
        data = rng.integers(-8, 9, m).astype(np.float64)
    elif fill == "ones":
        data = np.ones(m)
    else:
        raise ValueError(fill)
    data = np.ascontiguousarray(data, dtype=np.float64)
    rec = {"mods": mods, "sig": tuple(l.s for l in legs), "n": n, "t": t, "D": D,
           "data": data.view(np.complex128) if cplx else data}
    if cplx:
        rec["dtype"] = "c128"
    return rec


def _allowed_blocks(mods, legs, n):
    """Every block (one sector per leg) with sum_i s_i rho_i == n, in canonical order.

    The first rank-1 legs are enumerated; the last leg's charge is then fixed by the
    conservation rule and looked up among that leg's sectors."""
    mods = np.array(mods, dtype=np.int64)
    nsym = len(mods)
    rank = len(legs)
    if rank == 0:
        ok = all(int(x) == 0 for x in _reduce(tuple(n), tuple(mods)))
        return (np.zeros((1 if ok else 0, 0, nsym), np.int32), np.zeros((1 if ok else 0, 0), np.int64))
    def red(x):
        return np.where(mods > 0, np.mod(x, np.where(mods > 0, mods, 1)), x)
    grids = np.meshgrid(*[np.arange(len(l.t)) for l in legs[:-1]], indexing="ij")
    idx = [g.ravel() for g in grids] if rank > 1 else []
    ncomb = idx[0].size if idx else 1
    tot = np.zeros((ncomb, nsym), dtype=np.int64)
    for leg, ii in zip(legs[:-1], idx):
        tarr = np.array(leg.t, dtype=np.int64).reshape(len(leg.t), nsym)
        tot += leg.s * tarr[ii]
    last = legs[-1]
    need = red(last.s * (np.array(n, dtype=np.int64)[None, :] - tot))
    lookup = {tuple(int(c) for c in _reduce(q, tuple(int(m) for m in mods))): i for i, q in enumerate(last.t)}
    # the last leg's own charges must already be reduced for Z_m components
    li = np.array([lookup.get(tuple(int(c) for c in row), -1) for row in need], dtype=np.int64)
    keep = li >= 0
    idx = [ii[keep] for ii in idx] + [li[keep]]
    nb = int(keep.sum())
    t = np.zeros((nb, rank, nsym), dtype=np.int64)
    D = np.zeros((nb, rank), dtype=np.int64)
    for a, (leg, ii) in enumerate(zip(legs, idx)):
        t[:, a, :] = np.array(leg.t, dtype=np.int64).reshape(len(leg.t), nsym)[ii]
        D[:, a] = np.array(leg.D, dtype=np.int64)[ii]
    flat = t.reshape(nb, rank * nsym)
    order = np.lexsort(flat.T[::-1]) if nb else np.zeros(0, dtype=np.int64)
    return t[order].astype(np.int32), D[order]


def block_offsets(D):
    """Packed element offsets of blocks stored back to back in the given order."""
    sizes = np.prod(D, axis=1) if len(D) else np.zeros(0, dtype=np.int64)
    off = np.zeros(len(sizes), dtype=np.int64)
    if len(sizes) > 1:
        off[1:] = np.cumsum(sizes)[:-1]
    return off


def record_size(rec):
    return int(np.prod(rec["D"], axis=1).sum()) if len(rec["D"]) else 0


# ---------------------------------------------------------------------------------
# Workload shapes (Sec. III). Sizes are the ones the workloads are quoted at.
# ---------------------------------------------------------------------------------

def double_layer_leg(leg, s=None, mods=None):
    """The D^2 leg of a double-layer tensor built from a ket leg and its bra (dual) leg.

    Workload shape only: the ket/bra pair of a PEPS bond fused into one leg has, for a
    fully populated site tensor, charges rho - rho' (ket minus bra) with dimension
    sum D_rho D_rho' per charge (Sec. II.B, fused charges and dimensions). Used to size
    the chi = D^2 environment legs and the double-layer legs of the synthetic inputs.
    """
    acc = {}
    for q1, d1 in zip(leg.t, leg.D):
        for q2, d2 in zip(leg.t, leg.D):
            q = tuple(a - b for a, b in zip(q1, q2))
            if mods is not None:
                q = _reduce(q, mods)
            acc[q] = acc.get(q, 0) + d1 * d2
    ts = sorted(acc)
    return Leg(leg.s if s is None else s, ts, [acc[q] for q in ts])


def gaussian_sector_sizes(D, candidates, width, seed, min_size=0):
    """Split a bond dimension D over candidate charges with a discrete Gaussian around
    the zero charge: sizes = min_size + multinomial(D - min_size*len, p ~ exp(-|q|^2/2w^2)).
    Sectors of size 0 are dropped."""
    cand = [tuple(q) for q in candidates]
    w = np.array([math.exp(-sum(c * c for c in q) / (2.0 * width * width)) for q in cand])
    w = w / w.sum()
    rng = np.random.default_rng(seed)
    extra = rng.multinomial(D - min_size * len(cand), w)
    sizes = [min_size + int(e) for e in extra]
    keep = [(q, d) for q, d in zip(cand, sizes) if d > 0]
    return [q for q, _ in keep], [d for _, d in keep]


def random_composition(total, parts, rng):
    """A random composition of ``total`` into ``parts`` positive integers."""
    if parts > total:
        raise ValueError("more parts than total")
    cuts = sorted(rng.choice(np.arange(1, total), size=parts - 1, replace=False)) if parts > 1 else []
    bounds = [0] + [int(c) for c in cuts] + [total]
    return [bounds[i + 1] - bounds[i] for i in range(parts)]


def config1(seed=1001):
    """U(1) rank-3 tensordot: A = B with legs (virtual s=+1, charges -2..2, sizes
    [3,6,8,6,3]), (physical s=+1, charges -1,+1, sizes [1,1]), (virtual s=-1, as the
    first); total charge 0. Contract A leg 2 with B leg 0."""
    v = Leg(1, [(-2,), (-1,), (0,), (1,), (2,)], [3, 6, 8, 6, 3])
    p = Leg(1, [(-1,), (1,)], [1, 1])
    legs = [v, p, v.conj()]
    A = random_tensor((0,), legs, (0,), seed)
    B = random_tensor((0,), legs, (0,), seed + 1)
    return {"A": A, "B": B, "axa": (2,), "axb": (0,), "name": "U(1) rank-3 MPS-like tensordot"}


def _peps_site_legs(vleg, pleg):
    # PEPS site legs (t, l, b, r, p) with signatures (-1, +1, +1, -1, +1).
    return [Leg(-1, vleg.t, vleg.D), Leg(1, vleg.t, vleg.D), Leg(1, vleg.t, vleg.D),
            Leg(-1, vleg.t, vleg.D), Leg(1, pleg.t, pleg.D)]


def config2(seed=2001, D_half=4, chi_half=32):
    """Z2 double-layer PEPS: site tensor rank 5 (physical Z2 {0:1, 1:1}, four virtual
    legs D=8 split 4+4), its conjugate, and a CTMRG edge tensor T (chi, D^2, chi) with
    chi = 64 split 32+32."""
    v = Leg(1, [(0,), (1,)], [D_half, D_half])
    p = Leg(1, [(0,), (1,)], [1, 1])
    A = random_tensor((2,), _peps_site_legs(v, p), (0,), seed)
    dl = double_layer_leg(v, mods=(2,))
    chi = Leg(1, [(0,), (1,)], [chi_half, chi_half])
    # T contracts its D^2 leg with the double layer's t leg (s=-1), so it carries s=+1.
    T = random_tensor((2,), [chi, Leg(1, dl.t, dl.D), chi.conj()], (0,), seed + 1)
    return {"A": A, "T": T, "vleg": v, "pleg": p, "mods": (2,),
            "name": "Z2 double-layer PEPS, D=8, chi=64"}


def _u1u1_charges(r):
    return [(a, b) for a in range(-r, r + 1) for b in range(-r, r + 1)]


def config3(seed=3001):
    """U(1)xU(1) spinful-fermion iPEPS CTMRG step: physical dim 4 (charges (0,0),
    (1,0), (0,1), (1,1)), virtual D=12 over 9 charges {-1,0,1}^2 with sizes
    1 + multinomial(3, p ~ exp(-|q|^2/2)) (seed 0), chi = D^2 = 144.

    Returns the site tensor A and the random environment stand-ins: corner C (chi, chi),
    edge T (chi, D^2, chi) and X2 (chi, D^2, D^2, chi), a random stand-in for C.T.T whose
    D^2 legs are dual to the double layer's t and l legs."""
    ts, ds = gaussian_sector_sizes(12, _u1u1_charges(1), 1.0, 0, min_size=1)
    v = Leg(1, ts, ds)
    p = Leg(1, [(0, 0), (1, 0), (0, 1), (1, 1)], [1, 1, 1, 1])
    mods = (0, 0)
    A = random_tensor(mods, _peps_site_legs(v, p), (0, 0), seed)
    dl = double_layer_leg(v)
    chi = Leg(1, dl.t, dl.D)
    C = random_tensor(mods, [chi, chi.conj()], (0, 0), seed + 1)
    T = random_tensor(mods, [chi, Leg(1, dl.t, dl.D), chi.conj()], (0, 0), seed + 2)
    X2 = random_tensor(mods, [chi, Leg(1, dl.t, dl.D), Leg(-1, dl.t, dl.D), chi.conj()],
                       (0, 0), seed + 3)
    return {"A": A, "C": C, "T": T, "X2": X2, "vleg": v, "pleg": p, "dleg": dl,
            "mods": mods, "name": "U(1)xU(1) CTMRG step, D=12, chi=144"}


def _x2_a(mods, dl, seed):
    chi = Leg(1, dl.t, dl.D)
    X2 = random_tensor(mods, [chi, Leg(1, dl.t, dl.D), Leg(-1, dl.t, dl.D), chi.conj()],
                       (0,) * len(mods), seed)
    a = random_tensor(mods, [Leg(-1, dl.t, dl.D), Leg(1, dl.t, dl.D), Leg(1, dl.t, dl.D),
                             Leg(-1, dl.t, dl.D)], (0,) * len(mods), seed + 1)
    return X2, a


def ctm_corner_network(cfg):
    """The enlarged corner of a CTMRG step as an ncon network: corner C, two edges T
    and the double layer a (random, on the D^2 legs of the U(1)xU(1) D=12 workload).
    Output legs: T1's chi, T2's chi, a's two outer D^2 legs."""
    dl = cfg["dleg"]
    _, a = _x2_a(cfg["mods"], dl, 3101)
    tensors = [cfg["C"], cfg["T"], cfg["T"], a]
    labels = [[1, 2], [2, 3, -1], [-2, 4, 1], [3, -3, -4, 4]]
    return tensors, labels


def config5(seed=5001, D=20):
    """Large U(1)xU(1) Hubbard-like environment contraction X2 . a over two legs:
    D=20 over the 25 candidate charges {-2..2}^2 with sizes multinomial(20,
    p ~ exp(-|q|^2 / (2*1.5^2))) (seed 0), zero sectors dropped; chi = D^2 = 400."""
    ts, ds = gaussian_sector_sizes(D, _u1u1_charges(2), 1.5, 0, min_size=0)
    v = Leg(1, ts, ds)
    dl = double_layer_leg(v)
    X2, a = _x2_a((0, 0), dl, seed)
    return {"A": X2, "B": a, "axa": (1, 2), "axb": (0, 1), "vleg": v, "dleg": dl,
            "name": f"U(1)xU(1) X2.a, D={D}, chi={dl.dim}"}


def _keep_blocks(T, keep):
    """The record T with only the blocks where keep is true (block order kept)."""
    keep = np.asarray(keep, dtype=bool)
    size = np.prod(T["D"], axis=1)
    off = np.concatenate([[0], np.cumsum(size)])
    idx = np.nonzero(keep)[0]
    R = dict(T)
    R["t"] = T["t"][idx].copy()
    R["D"] = T["D"][idx].copy()
    R["data"] = (np.concatenate([T["data"][off[i]:off[i + 1]] for i in idx]) if len(idx)
                 else np.zeros(0, dtype=T["data"].dtype))
    return R


def config5_sectors(seed=5001, frac=0.25, pick=2, D=20):
    """A profiling-size part of the D=20 contraction X2 . a: every block of a random
    fraction of its contraction sectors (a sector: the charge carried through the
    contracted legs, X2's legs 1, 2 = a's legs 0, 1). The kept blocks and sectors have
    the full workload's sizes; with the defaults, 7.05e7 elements per tensor against
    3.36e8, mean block 3046 elements against 3242."""
    cfg = config5(seed=seed, D=D)
    X2, a = cfg["A"], cfg["B"]
    kx = X2["t"][:, 1, :] - X2["t"][:, 2, :]
    ka = a["t"][:, 0, :] - a["t"][:, 1, :]
    keys = sorted(set(map(tuple, kx)))
    rng = np.random.default_rng(pick)
    chosen = {keys[i] for i in rng.choice(len(keys), max(1, int(frac * len(keys))), replace=False)}
    return {"A": _keep_blocks(X2, [tuple(k) in chosen for k in kx]),
            "B": _keep_blocks(a, [tuple(k) in chosen for k in ka]),
            "axa": (1, 2), "axb": (0, 1), "dleg": cfg["dleg"],
            "name": f"U(1)xU(1) X2.a, D={D}: blocks of {len(chosen)} of its {len(keys)} sectors"}


def config5b(seed=5101, D=20):
    """Alternative reading of the large workload: D=20 over the 9 charges {-1,0,1}^2
    with minimum size 1, so the D^2 and chi legs have exactly 25 sectors."""
    ts, ds = gaussian_sector_sizes(D, _u1u1_charges(1), 1.5, 0, min_size=1)
    v = Leg(1, ts, ds)
    dl = double_layer_leg(v)
    X2, a = _x2_a((0, 0), dl, seed)
    return {"A": X2, "B": a, "axa": (1, 2), "axb": (0, 1), "vleg": v, "dleg": dl,
            "name": f"U(1)xU(1) X2.a (25-sector reading), D={D}, chi={dl.dim}"}


def serving_runs(nruns=64, seed=4001, Ds=(4, 6, 8, 10, 12)):
    """Structures of the independent U(1) spin-1/2 iPEPS runs of the serving stream.

    Per run: D uniform in ``Ds``; chi uniform in [4D, 8D]; D split into 3 (D < 6) or 5
    centred charges and chi into 9 charges -4..4, both by random composition. The
    request of a run is X2_r . a_r over two legs (X2: (chi, D^2, D^2, chi))."""
    rng = np.random.default_rng(seed)
    runs = []
    for r in range(nruns):
        D = int(rng.choice(Ds))
        chi = int(rng.integers(4 * D, 8 * D + 1))
        nv = 3 if D < 6 else 5
        v = Leg(1, [(q,) for q in range(-(nv // 2), nv // 2 + 1)], random_composition(D, nv, rng))
        dl = double_layer_leg(v)
        c = Leg(1, [(q,) for q in range(-4, 5)], random_composition(chi, 9, rng))
        runs.append({"run": r, "D": D, "chi": chi, "vleg": v, "dleg": dl, "chileg": c,
                     "seed": seed * 100 + r})
    return runs


def serving_request(run, seed_offset=0):
    """Tensors (X2_r, a_r) of one serving run, drawn from the run's seed."""
    dl, c = run["dleg"], run["chileg"]
    mods = (0,)
    X2 = random_tensor(mods, [c, Leg(1, dl.t, dl.D), Leg(-1, dl.t, dl.D), c.conj()], (0,),
                       run["seed"] + seed_offset)
    a = random_tensor(mods, [Leg(-1, dl.t, dl.D), Leg(1, dl.t, dl.D), Leg(1, dl.t, dl.D),
                             Leg(-1, dl.t, dl.D)], (0,), run["seed"] + seed_offset + 7)
    return X2, a
