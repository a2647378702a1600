"""CPU FP64 oracle for abelian-symmetric block-sparse tensors.

TEST INFRASTRUCTURE. This module is the plain, slow, reference statement of what the
library computes. Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it. It shares no code with the CUDA
library and imports nothing from it; the library never calls it.

It follows the paper "YASTN: Yet another symmetric tensor networks" (arXiv 2405.12196):

* Sec. II.A -- a tensor is a set of dense blocks, one per tuple of charge sectors
  (rho_1..rho_N), one sector per leg V(s, t, D); stored blocks satisfy
  sum_i s_i rho_i = n (block form of Eq. ``elemchargecon``), component-wise and modulo
  m for Z_m components (charges of U(1) live in Z, of Z_m in Z_m, of product groups in
  products of these).
* Sec. II.B -- fusion: fused charge nu = s_r (s_i rho + s_j rho') and fused dimension
  D_nu = sum of D_rho D_rho' over the pairs that give nu; fusion is lazy (only charges
  of blocks that exist); the fused tensor records the original structure so that the
  fusion can be undone.
* Sec. II.B, contraction equation -- tensordot = fuse into matrices, multiply, unfuse;
  the result is, by definition, the sum over the contracted indices of the products of
  the elements, which for block-sparse tensors is a sum over matching block pairs.

Readings where the paper is silent (each is listed in the design notes):
contraction compatibility = opposite signatures and equal dimensions of every charge
present on both legs; n_C = n_A + n_B; output legs = A's free legs then B's; blocks in
ascending lexicographic order of their charge tuple, row-major elements; fused signature
= signature of the group's first leg; fused sub-blocks ordered by ascending constituent
charge tuple; fusion records of contracted fused legs must be conjugate of one another
(else an error); trace over leg pairs sums the diagonals of blocks whose paired charges
are equal.

Pins (``tests/test_oracle_*.py``): brute force against the dense embedding on random
U(1), Z2, Z3 and U(1)xU(1) tensors, the trivial-symmetry special case, the closed form
(S1.S2)^2 = 3/16 - S1.S2/2 on the paper's two-spin example, hand-derived structure
counts, fuse/unfuse round trips and singular-value invariance of fused matrices.
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = [
    "OTensor", "OracleError", "SignatureError", "DimMismatchError", "FusionMismatchError",
    "ChargeError", "InvalidError", "UnsupportedError",
    "from_record", "to_record", "conj", "tensordot", "fuse", "unfuse", "trace",
    "to_dense", "leg_sectors", "useful_flops", "tensordot_block", "vdot", "swap_gate", "charge_parity", "ncon", "einsum", "svd", "eigh", "truncation", "slice_leg", "philox4x32", "normal_fill",
]


class OracleError(Exception):
    pass


class InvalidError(OracleError):
    pass


class SignatureError(OracleError):
    pass


class DimMismatchError(OracleError):
    pass


class FusionMismatchError(OracleError):
    pass


class ChargeError(OracleError):
    pass


class UnsupportedError(OracleError):
    pass


def _red(q, mods):
    """Reduce a charge tuple: Z components as they are, Z_m components modulo m."""
    return tuple((int(c) % m) if m else int(c) for c, m in zip(q, mods))


def _add(q1, q2, mods):
    return _red(tuple(a + b for a, b in zip(q1, q2)), mods)


def _scale(s, q, mods):
    return _red(tuple(s * c for c in q), mods)


class FusionRecord:
    """What a fused leg remembers about its origin (Sec. II.B: the fused tensor records
    the original structure).

    ``sig``: signatures of the constituent legs. ``entries``: for each fused charge nu,
    the list of (constituent charges, constituent dims) that were present, in ascending
    order of the constituent charge tuple; each occupies prod(dims) consecutive indices
    of the fused sector, in that order."""

    def __init__(self, sig, entries):
        self.sig = tuple(int(s) for s in sig)
        self.entries = {nu: sorted(lst) for nu, lst in entries.items()}

    def dim(self, nu):
        return sum(int(np.prod(d)) for _, d in self.entries[nu])

    def offsets(self, nu):
        out, off = [], 0
        for ch, d in self.entries[nu]:
            out.append((ch, d, off))
            off += int(np.prod(d))
        return out

    def conj(self):
        return FusionRecord(tuple(-s for s in self.sig), self.entries)

    def key(self):
        return (self.sig, tuple(sorted((nu, tuple(l)) for nu, l in self.entries.items())))


class OTensor:
    """A block-sparse symmetric tensor: ``blocks`` maps a tuple of per-leg charge tuples
    to a dense FP64 array whose shape is the per-leg sector dimensions."""

    def __init__(self, mods, sig, n, blocks=None, fus=None, dtype=None):
        self.mods = tuple(int(m) for m in mods)
        self.sig = tuple(int(s) for s in sig)
        self.n = _red(n, self.mods)
        self.blocks = {} if blocks is None else blocks
        self.fus = list(fus) if fus is not None else [None] * len(self.sig)
        # element type: float64, or complex128 (given, or found in the blocks)
        if dtype is None:
            dtype = np.complex128 if any(np.iscomplexobj(b) for b in self.blocks.values()) else np.float64
        self.dtype = np.dtype(dtype)

    @property
    def rank(self):
        return len(self.sig)

    @property
    def nsym(self):
        return len(self.mods)

    def keys(self):
        """Block keys in canonical order: ascending lexicographic charge tuples."""
        return sorted(self.blocks)

    def validate(self):
        """Check the block conservation rule and that a charge has one dimension per leg."""
        dims = [dict() for _ in range(self.rank)]
        for key, blk in self.blocks.items():
            if len(key) != self.rank or blk.ndim != self.rank:
                raise InvalidError("block rank does not match the tensor rank")
            tot = tuple([0] * self.nsym)
            for s, q in zip(self.sig, key):
                tot = _add(tot, _scale(s, q, self.mods), self.mods)
            if tot != self.n:
                raise ChargeError(f"block {key} violates charge conservation")
            for a, (q, d) in enumerate(zip(key, blk.shape)):
                if dims[a].setdefault(q, d) != d:
                    raise DimMismatchError(f"leg {a} charge {q} has two dimensions")
                if self.fus[a] is not None:
                    if q not in self.fus[a].entries or self.fus[a].dim(q) != d:
                        raise InvalidError("fused leg block does not match its record")
        return self


def leg_sectors(T, axis):
    """Charge -> dimension map of one leg, read from the stored blocks (and, for a fused
    leg, from its record)."""
    out = {}
    for key, blk in T.blocks.items():
        out[key[axis]] = blk.shape[axis]
    if T.fus[axis] is not None:
        for nu in T.fus[axis].entries:
            out.setdefault(nu, T.fus[axis].dim(nu))
    return out


# ------------------------------------------------------------------ plain-array records

def from_record(rec):
    """Build an OTensor from the plain-array record of ``workloads`` (canonical order,
    packed row-major blocks); ``rec['fus']`` (optional) holds per-leg fusion records in
    plain-array form. Blocks are views of ``rec['data']``."""
    mods = tuple(rec["mods"])
    t = np.asarray(rec["t"])
    D = np.asarray(rec["D"])
    dtype = np.complex128 if rec.get("dtype") == "c128" else np.float64
    data = np.asarray(rec["data"], dtype=dtype)
    blocks = {}
    off = 0
    for b in range(len(t)):
        key = tuple(tuple(int(c) for c in t[b, a]) for a in range(t.shape[1]))
        shape = tuple(int(d) for d in D[b])
        sz = int(np.prod(shape))
        if key in blocks:
            raise InvalidError("duplicate block")
        blocks[key] = data[off:off + sz].reshape(shape)  # a view: inputs are never modified
        off += sz
    if off != data.size:
        raise InvalidError("data size does not match the block dimensions")
    fus = None
    if rec.get("fus") is not None:
        fus = [None if f is None else _record_from_plain(f) for f in rec["fus"]]
    return OTensor(mods, rec["sig"], rec["n"], blocks, fus, dtype=dtype).validate()


def _record_from_plain(f):
    entries = {}
    nu = np.asarray(f["nu"])
    ct = np.asarray(f["t"])
    cd = np.asarray(f["D"])
    for e in range(len(nu)):
        key = tuple(int(c) for c in nu[e])
        ch = tuple(tuple(int(c) for c in ct[e, i]) for i in range(ct.shape[1]))
        dd = tuple(int(d) for d in cd[e])
        entries.setdefault(key, []).append((ch, dd))
    return FusionRecord(f["sig"], entries)


def _record_to_plain(fr, nsym):
    rows = [(nu, ch, d) for nu in sorted(fr.entries) for ch, d in fr.entries[nu]]
    m = len(fr.sig)
    nu = np.array([r[0] for r in rows], dtype=np.int32).reshape(len(rows), nsym)
    t = np.array([r[1] for r in rows], dtype=np.int32).reshape(len(rows), m, nsym)
    D = np.array([r[2] for r in rows], dtype=np.int64).reshape(len(rows), m)
    return {"sig": fr.sig, "nu": nu, "t": t, "D": D}


def to_record(T):
    """Plain-array record of an OTensor (canonical block order, packed data)."""
    keys = T.keys()
    nb = len(keys)
    t = np.zeros((nb, T.rank, T.nsym), dtype=np.int32)
    D = np.zeros((nb, T.rank), dtype=np.int64)
    parts = []
    for b, key in enumerate(keys):
        for a in range(T.rank):
            t[b, a, :] = key[a]
        D[b, :] = T.blocks[key].shape
        parts.append(np.ascontiguousarray(T.blocks[key]).ravel())
    data = np.concatenate(parts).astype(T.dtype) if parts else np.zeros(0, dtype=T.dtype)
    fus = [None if f is None else _record_to_plain(f, T.nsym) for f in T.fus]
    rec = {"mods": T.mods, "sig": T.sig, "n": T.n, "t": t, "D": D, "data": data,
           "fus": fus if any(f is not None for f in fus) else None}
    if T.dtype == np.complex128:
        rec["dtype"] = "c128"
    return rec


# ------------------------------------------------------------------ basic operations

def conj(T):
    """Conjugate: every leg's signature flips (Sec. II.A footnote), so the total charge
    becomes -n, and every element is complex-conjugated (real data is unchanged)."""
    fus = [None if f is None else f.conj() for f in T.fus]
    return OTensor(T.mods, tuple(-s for s in T.sig), _scale(-1, T.n, T.mods),
                   {k: np.conj(v) for k, v in T.blocks.items()}, fus, dtype=T.dtype)


def _check_pairs(rankA, rankB, axa, axb):
    axa, axb = tuple(int(a) for a in axa), tuple(int(b) for b in axb)
    if len(axa) != len(axb):
        raise InvalidError("axes lists differ in length")
    if len(set(axa)) != len(axa) or len(set(axb)) != len(axb):
        raise InvalidError("repeated axis")
    if any(a < 0 or a >= rankA for a in axa) or any(b < 0 or b >= rankB for b in axb):
        raise InvalidError("axis out of range")
    return axa, axb


def _check_compatible(A, a, B, b):
    """Contracted legs must be compatible: opposite signatures, equal dimension for each
    charge present on both, conjugate fusion records (Sec. II.B footnote)."""
    if A.sig[a] != -B.sig[b]:
        raise SignatureError(f"leg {a} of A and leg {b} of B have equal signatures")
    da, db = leg_sectors(A, a), leg_sectors(B, b)
    for q in set(da) & set(db):
        if da[q] != db[q]:
            raise DimMismatchError(f"charge {q}: dimension {da[q]} vs {db[q]}")
    fa, fb = A.fus[a], B.fus[b]
    if (fa is None) != (fb is None):
        raise FusionMismatchError("a fused leg is contracted with a plain leg")
    if fa is not None and fa.key() != fb.conj().key():
        raise FusionMismatchError("fusion records of contracted legs differ")


def _mismatched(A, a, B, b):
    fa, fb = A.fus[a], B.fus[b]
    return fa is not None and fb is not None and fa.key() != fb.conj().key()


def _check_resolvable(fa, fb):
    """Two fused legs with different histories can be contracted when they were fused
    from the same constituent legs (same count, opposite signatures) and agree on the
    dimensions of every constituent charge tuple both records list."""
    if len(fa.sig) != len(fb.sig) or any(x != -y for x, y in zip(fa.sig, fb.sig)):
        raise FusionMismatchError("contracted fused legs come from different constituent legs")
    da = {ch: d for lst in fa.entries.values() for ch, d in lst}
    db = {ch: d for lst in fb.entries.values() for ch, d in lst}
    for ch in set(da) & set(db):
        if da[ch] != db[ch]:
            raise DimMismatchError(f"constituent charges {ch}: dimensions {da[ch]} vs {db[ch]}")


def _expand_axes(T, axes, unf):
    """Positions of legs after unfusing the legs in ``unf``: each unfused leg becomes
    its constituents, in order, at its place."""
    pos, p = [], 0
    for a in range(T.rank):
        n = len(T.fus[a].sig) if a in unf else 1
        pos.append(list(range(p, p + n)))
        p += n
    return [q for a in axes for q in pos[a]]


def tensordot(A, B, axa, axb):
    """C = sum over the contracted indices of A * B (Sec. II.B, contraction equation).

    Every pair (alpha, beta) of stored blocks whose charges agree on all contracted legs
    contributes tensordot(A_alpha, B_beta) to the C block keyed by A's free charges
    followed by B's free charges. Blocks of C exist when at least one pair contributed
    (lazy storage, Sec. II.A).

    Contracted fused legs with different fusion histories (Sec. II.B footnote: a charge
    of the history missing on one side but present on the other) are resolved: a
    missing constituent charge tuple counts as a zero sub-block, so the contraction
    over the fused index is the contraction over its constituent legs. The oracle
    unfuses those legs on both sides and contracts over the constituents."""
    if A.mods != B.mods:
        raise InvalidError("tensors have different symmetries")
    axa, axb = _check_pairs(A.rank, B.rank, axa, axb)
    mism = [k for k, (a, b) in enumerate(zip(axa, axb)) if _mismatched(A, a, B, b)]
    if mism:
        for k in mism:
            if A.sig[axa[k]] != -B.sig[axb[k]]:
                raise SignatureError(f"leg {axa[k]} of A and leg {axb[k]} of B have equal signatures")
            _check_resolvable(A.fus[axa[k]], B.fus[axb[k]])
        ua, ub = {axa[k] for k in mism}, {axb[k] for k in mism}
        A2, B2 = unfuse(A, sorted(ua)), unfuse(B, sorted(ub))
        return tensordot(A2, B2, _expand_axes(A, axa, ua), _expand_axes(B, axb, ub))
    for a, b in zip(axa, axb):
        _check_compatible(A, a, B, b)
    freeA = [i for i in range(A.rank) if i not in axa]
    freeB = [i for i in range(B.rank) if i not in axb]
    C = OTensor(A.mods, tuple(A.sig[i] for i in freeA) + tuple(B.sig[i] for i in freeB),
                _add(A.n, B.n, A.mods),
                fus=[A.fus[i] for i in freeA] + [B.fus[i] for i in freeB],
                dtype=np.result_type(A.dtype, B.dtype))
    byx = {}
    for kb in B.keys():
        byx.setdefault(tuple(kb[b] for b in axb), []).append(kb)
    for ka in A.keys():
        x = tuple(ka[a] for a in axa)
        for kb in byx.get(x, []):
            kc = tuple(ka[i] for i in freeA) + tuple(kb[i] for i in freeB)
            prod = np.tensordot(A.blocks[ka], B.blocks[kb], axes=(axa, axb))
            if kc in C.blocks:
                C.blocks[kc] = C.blocks[kc] + prod
            else:
                C.blocks[kc] = np.array(prod, dtype=C.dtype)
    return C


def tensordot_block(A, B, axa, axb, kc):
    """One output block of tensordot(A, B), summed over its matching pairs in canonical
    order -- the same definition as ``tensordot``, evaluated for one key (used to check
    sampled outputs of large contractions)."""
    axa, axb = tuple(axa), tuple(axb)
    freeA = [i for i in range(A.rank) if i not in axa]
    freeB = [i for i in range(B.rank) if i not in axb]
    ia, ib = kc[:len(freeA)], kc[len(freeA):]
    rowsA = [ka for ka in A.keys() if tuple(ka[i] for i in freeA) == ia]
    colsB = {}
    for kb in B.keys():
        if tuple(kb[i] for i in freeB) == ib:
            colsB[tuple(kb[b] for b in axb)] = kb
    out = None
    for ka in rowsA:
        kb = colsB.get(tuple(ka[a] for a in axa))
        if kb is None:
            continue
        prod = np.tensordot(A.blocks[ka], B.blocks[kb], axes=(axa, axb))
        out = prod if out is None else out + prod
    return out


def useful_flops(A, B, axa, axb):
    """FLOPs of the block-sparse contraction: 2 |I| |x| |J| per matching block pair."""
    axa, axb = tuple(axa), tuple(axb)
    byx = {}
    for kb, blk in B.blocks.items():
        byx.setdefault(tuple(kb[b] for b in axb), []).append(blk.size)
    total = 0
    for ka, blk in A.blocks.items():
        x = tuple(ka[a] for a in axa)
        kx = int(np.prod([blk.shape[a] for a in axa])) if axa else 1
        for szb in byx.get(x, []):
            total += 2 * (blk.size // kx) * kx * (szb // kx)
    return total


# ------------------------------------------------------------------ fusion

def _normalise_groups(groups, rank):
    gs = [tuple(g) if isinstance(g, (tuple, list)) else (int(g),) for g in groups]
    flat = [a for g in gs for a in g]
    if sorted(flat) != list(range(rank)):
        raise InvalidError("fusion groups must list every leg exactly once")
    if any(len(g) == 0 for g in gs):
        raise InvalidError("empty fusion group")
    return gs


def fuse(A, groups):
    """Fuse groups of legs into single legs (Sec. II.B).

    For a group of legs i..j the fused leg gets the signature of the group's first leg
    s_r, charges nu = s_r * sum_i s_i rho_i, and dimension D_nu = sum over the charge
    tuples present in some stored block of prod_i D_rho_i (lazy fusion). Sub-blocks sit
    in ascending order of their constituent charge tuple, each row-major over the group's
    legs. Every stored block is transposed to the group order and copied to its place in
    the fused block; fused-block entries with no stored block are zero."""
    gs = _normalise_groups(groups, A.rank)
    mods = A.mods
    # a single leg passes through; a group of two or more legs must consist of plain legs
    for g in gs:
        if len(g) > 1 and any(A.fus[a] is not None for a in g):
            raise UnsupportedError("fusing an already fused leg")
    rec = []
    for g in gs:
        if len(g) == 1:
            rec.append(None)
            continue
        entries = {}
        seen = set()
        for key, blk in A.blocks.items():
            ch = tuple(key[a] for a in g)
            if ch in seen:
                continue
            seen.add(ch)
            tot = tuple([0] * A.nsym)
            for a in g:
                tot = _add(tot, _scale(A.sig[a], key[a], mods), mods)
            nu = _scale(A.sig[g[0]], tot, mods)
            entries.setdefault(nu, []).append((ch, tuple(blk.shape[a] for a in g)))
        rec.append(FusionRecord(tuple(A.sig[a] for a in g), entries))
    sig = tuple(A.sig[g[0]] for g in gs)
    fus = [A.fus[g[0]] if len(g) == 1 else rec[i] for i, g in enumerate(gs)]
    out = OTensor(mods, sig, A.n, fus=fus, dtype=A.dtype)
    order = [a for g in gs for a in g]
    for key in A.keys():
        blk = A.blocks[key]
        newkey, shape, box = [], [], []
        for i, g in enumerate(gs):
            if len(g) == 1:
                newkey.append(key[g[0]])
                shape.append(blk.shape[g[0]])
                box.append((0, blk.shape[g[0]]))
            else:
                ch = tuple(key[a] for a in g)
                tot = tuple([0] * A.nsym)
                for a in g:
                    tot = _add(tot, _scale(A.sig[a], key[a], mods), mods)
                nu = _scale(A.sig[g[0]], tot, mods)
                newkey.append(nu)
                shape.append(rec[i].dim(nu))
                for c, d, off in rec[i].offsets(nu):
                    if c == ch:
                        box.append((off, int(np.prod(d))))
                        break
        newkey = tuple(newkey)
        if newkey not in out.blocks:
            out.blocks[newkey] = np.zeros(shape, dtype=A.dtype)
        sub = np.transpose(blk, order).reshape([b[1] for b in box])
        out.blocks[newkey][tuple(slice(o, o + n) for o, n in box)] = sub
    return out


def unfuse(A, axes):
    """Undo the fusion of the given fused legs using their records (Sec. II.B).

    Every fused block is cut into its recorded sub-blocks; each sub-block is reshaped to
    the constituent dimensions and stored under the constituent charges. All recorded
    sub-blocks of stored fused blocks are emitted, including ones that are zero."""
    axes = sorted(set(int(a) for a in axes))
    for a in axes:
        if a < 0 or a >= A.rank or A.fus[a] is None:
            raise InvalidError(f"leg {a} is not a fused leg")
    sig, fus = [], []
    for a in range(A.rank):
        if a in axes:
            sig.extend(A.fus[a].sig)
            fus.extend([None] * len(A.fus[a].sig))
        else:
            sig.append(A.sig[a])
            fus.append(A.fus[a])
    out = OTensor(A.mods, tuple(sig), A.n, fus=fus, dtype=A.dtype)
    for key in A.keys():
        blk = A.blocks[key]
        choices = []
        for a in range(A.rank):
            if a in axes:
                choices.append(A.fus[a].offsets(key[a]))
            else:
                choices.append([((key[a],), (blk.shape[a],), 0)])
        for combo in itertools.product(*choices):
            sl = tuple(slice(off, off + int(np.prod(d))) for _, d, off in combo)
            newkey = tuple(q for ch, _, _ in combo for q in ch)
            shape = tuple(x for _, d, _ in combo for x in d)
            out.blocks[newkey] = np.array(blk[sl]).reshape(shape)
    return out


# ------------------------------------------------------------------ trace

def trace(A, ax1, ax2):
    """Sum over the diagonals of leg pairs (ax1[k], ax2[k]).

    The paper does not describe a trace; this follows from the block structure: a pair
    of legs is traced when its signatures are opposite; a block contributes when its two
    charges of every pair are equal, and adds sum_d block[..d..d..] to the output block
    keyed by its remaining charges. The total charge is unchanged."""
    ax1, ax2 = tuple(int(a) for a in ax1), tuple(int(b) for b in ax2)
    if len(ax1) != len(ax2) or len(set(ax1 + ax2)) != 2 * len(ax1):
        raise InvalidError("trace axes must be disjoint pairs")
    if any(a < 0 or a >= A.rank for a in ax1 + ax2):
        raise InvalidError("axis out of range")
    for a, b in zip(ax1, ax2):
        _check_compatible(A, a, A, b)
    rest = [i for i in range(A.rank) if i not in ax1 + ax2]
    out = OTensor(A.mods, tuple(A.sig[i] for i in rest), A.n, fus=[A.fus[i] for i in rest], dtype=A.dtype)
    for key in A.keys():
        if any(key[a] != key[b] for a, b in zip(ax1, ax2)):
            continue
        blk = A.blocks[key]
        P = int(np.prod([blk.shape[a] for a in ax1])) if ax1 else 1
        R = [blk.shape[i] for i in rest]
        m = np.transpose(blk, rest + list(ax1) + list(ax2)).reshape(int(np.prod(R)) if R else 1, P, P)
        val = np.trace(m, axis1=1, axis2=2).reshape(R)
        kc = tuple(key[i] for i in rest)
        out.blocks[kc] = out.blocks[kc] + val if kc in out.blocks else np.array(val, dtype=A.dtype)
    return out


# ------------------------------------------------------------------ networks (ncon)

def ncon(tensors, labels):
    """Contraction of a network of tensors (Sec. II.B: general networks are contracted
    through pairwise tensordot by the einsum/ncon convenience functions; the labelling
    is the ncon convention of Pfeifer, Evenbly, Singh and Vidal, 2015).

    ``labels[i][k]`` labels leg k of tensor i. A positive label is summed and appears
    on exactly two legs; the negative labels -1, -2, ... name the output legs, in that
    order. The order of evaluation: while positive labels remain, take the smallest;
    if both its legs are on one tensor, trace every label that tensor carries twice;
    else contract the two tensors that carry it over every label they share, as
    tensordot(first in list order, second) with the shared labels in ascending order,
    the result taking the first tensor's place. Tensors left with only negative labels
    are then joined by outer products in list order. Last, the legs are permuted into
    the order -1, -2, ...; a network of one tensor is copied."""
    if len(tensors) != len(labels) or not tensors:
        raise InvalidError("one label list per tensor, at least one tensor")
    items = []
    for T, lab in zip(tensors, labels):
        lab = [int(x) for x in lab]
        if len(lab) != T.rank or 0 in lab:
            raise InvalidError("one nonzero label per leg")
        items.append((T, lab))
    flat = [x for _, lab in items for x in lab]
    pos = sorted(x for x in set(flat) if x > 0)
    neg = sorted((x for x in set(flat) if x < 0), reverse=True)
    if any(flat.count(x) != 2 for x in pos) or any(flat.count(x) != 1 for x in neg):
        raise InvalidError("a positive label must appear twice, a negative label once")
    if neg and neg != list(range(-1, -len(neg) - 1, -1)):
        raise InvalidError("negative labels must be -1, -2, ... without gaps")
    while True:
        rest = sorted({x for _, lab in items for x in lab if x > 0})
        if not rest:
            break
        x = rest[0]
        where = [i for i, (_, lab) in enumerate(items) if x in lab]
        if len(where) == 1:
            T, lab = items[where[0]]
            twice = sorted({y for y in lab if y > 0 and lab.count(y) == 2})
            ax1 = [lab.index(y) for y in twice]
            ax2 = [len(lab) - 1 - lab[::-1].index(y) for y in twice]
            out = trace(T, ax1, ax2)
            items[where[0]] = (out, [y for k, y in enumerate(lab) if k not in ax1 + ax2])
            continue
        i, j = where
        (A, la), (B, lb) = items[i], items[j]
        shared = sorted(set(la) & set(lb))
        C = tensordot(A, B, [la.index(y) for y in shared], [lb.index(y) for y in shared])
        lc = [y for y in la if y not in shared] + [y for y in lb if y not in shared]
        items[i] = (C, lc)
        del items[j]
    while len(items) > 1:
        (A, la), (B, lb) = items[0], items[1]
        items[0:2] = [(tensordot(A, B, (), ()), la + lb)]
    T, lab = items[0]
    order = [lab.index(-k) for k in range(1, len(lab) + 1)]
    return fuse(T, [(a,) for a in order]) if T.rank else OTensor(T.mods, (), T.n, dict(T.blocks), dtype=T.dtype)


def einsum(subscripts, *tensors):
    """einsum front end (Sec. II.B: einsum and ncon differ only by syntax).

    ``subscripts`` like "abc,cd->adb": one letter per leg. A letter on two legs is
    summed (twice on one tensor: a trace); a letter on one leg is an output leg. The
    output order is the part after "->", or, without it, the once-used letters in
    alphabetical order. Translation to ncon labels: summed letters get 1, 2, ... in
    the order of their first appearance, output letters -1, -2, ... in output order."""
    s = subscripts.replace(" ", "")
    lhs, arrow, rhs = s.partition("->")
    ins = lhs.split(",")
    if len(ins) != len(tensors) or not all(x.isalpha() for x in "".join(ins)):
        raise InvalidError("one letter group per tensor")
    count = {}
    for grp in ins:
        for c in grp:
            count[c] = count.get(c, 0) + 1
    if any(v > 2 for v in count.values()):
        raise InvalidError("a letter on more than two legs")
    out = rhs if arrow else "".join(sorted(c for c, v in count.items() if v == 1))
    if sorted(out) != sorted(c for c, v in count.items() if v == 1) or len(set(out)) != len(out):
        raise InvalidError("the output must list every once-used letter once")
    lab = {c: -(k + 1) for k, c in enumerate(out)}
    nxt = 1
    for grp in ins:
        for c in grp:
            if c not in lab:
                lab[c] = nxt
                nxt += 1
    return ncon(list(tensors), [[lab[c] for c in grp] for grp in ins])


# ------------------------------------------------------------------ random data

def philox4x32(ctr, key, rounds=10):
    """Philox4x32 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
    random numbers: as easy as 1, 2, 3", SC'11): ``rounds`` rounds of two 32x32 ->
    64-bit multiplications (multipliers 0xD2511F53, 0xCD9E8D57) with the key added
    by XOR, the key bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85) between
    rounds. ctr: four uint32, key: two uint32; returns four uint32."""
    c = [int(x) & 0xFFFFFFFF for x in ctr]
    k = [int(x) & 0xFFFFFFFF for x in key]
    for r in range(rounds):
        if r:
            k = [(k[0] + 0x9E3779B9) & 0xFFFFFFFF, (k[1] + 0xBB67AE85) & 0xFFFFFFFF]
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k[0]) & 0xFFFFFFFF, p1 & 0xFFFFFFFF,
             ((p0 >> 32) ^ c[3] ^ k[1]) & 0xFFFFFFFF, p0 & 0xFFFFFFFF]
    return c


def normal_fill(seed, size):
    """N(0, 1) numbers of a random tensor's data (the paper's rand, Sec. II.A): element
    i takes word i mod 4 of Philox4x32-10 at counter (i div 4 low 32 bits, high 32
    bits, 0, 0) and key (seed low, seed high); each pair of words (x, y) gives, by
    the Box-Muller transform with u = (x + 1) 2^-32 in (0, 1] and v = y 2^-32,
    sqrt(-2 ln u) cos(2 pi v) and sqrt(-2 ln u) sin(2 pi v)."""
    out = np.zeros(size)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    for q in range((size + 3) // 4):
        w = philox4x32((q & 0xFFFFFFFF, q >> 32, 0, 0), key)
        for h in range(2):
            u = (w[2 * h] + 1.0) * 2.0 ** -32
            v = w[2 * h + 1] * 2.0 ** -32
            r = np.sqrt(-2.0 * np.log(u))
            for j, z in enumerate((r * np.cos(2 * np.pi * v), r * np.sin(2 * np.pi * v))):
                i = 4 * q + 2 * h + j
                if i < size:
                    out[i] = z
    return out


# ------------------------------------------------------------------ block-diagonal SVD

def svd(A, row_legs, col_legs):
    """Block-diagonal singular value decomposition (Sec. III, CTM: the SVD of a fused
    enlarged corner is block diagonal in the charge sectors, one dense SVD per
    block; the paper leaves it to the backend's linear algebra).

    The legs of A are split into rows and columns; rows whose charges sum (with
    signatures) to c meet only columns that complete the total charge, so A is
    block diagonal with one matrix M_c per c: rows are the row-charge tuples with
    sum c in ascending order (each row-major over its legs), columns likewise.
    M_c = U_c diag(S_c) V_c with k_c = min(rows, cols) and S_c descending (numpy's
    SVD). Returns (U, S, V): U on (row legs, new leg of signature -1), S on (new leg
    +1, new leg -1) with a diagonal k_c x k_c block per sector, V on (new leg +1, col
    legs); the new leg carries charge c with dimension k_c. tensordot(tensordot(U, S,
    (last,), (0,)), V, (last,), (0,)) == A (the legs in order rows, cols)."""
    row_legs, col_legs = tuple(int(a) for a in row_legs), tuple(int(b) for b in col_legs)
    if sorted(row_legs + col_legs) != list(range(A.rank)) or not row_legs or not col_legs:
        raise InvalidError("rows and columns must split the legs into two nonempty groups")
    mods = A.mods
    rows, cols, sect = {}, {}, {}
    for key, blk in A.blocks.items():
        rk, ck = tuple(key[a] for a in row_legs), tuple(key[b] for b in col_legs)
        c = tuple([0] * A.nsym)
        for a in row_legs:
            c = _add(c, _scale(A.sig[a], key[a], mods), mods)
        rows.setdefault(c, {})[rk] = int(np.prod([blk.shape[a] for a in row_legs]))
        cols.setdefault(c, {})[ck] = int(np.prod([blk.shape[b] for b in col_legs]))
        sect.setdefault(c, []).append(key)
    U = OTensor(mods, tuple(A.sig[a] for a in row_legs) + (-1,), tuple([0] * A.nsym),
                fus=[A.fus[a] for a in row_legs] + [None], dtype=A.dtype)
    S = OTensor(mods, (1, -1), tuple([0] * A.nsym), dtype=np.float64)
    V = OTensor(mods, (1,) + tuple(A.sig[b] for b in col_legs), A.n,
                fus=[None] + [A.fus[b] for b in col_legs], dtype=A.dtype)
    for c in sorted(sect):
        roff, coff, m, n = {}, {}, 0, 0
        for rk in sorted(rows[c]):
            roff[rk] = m
            m += rows[c][rk]
        for ck in sorted(cols[c]):
            coff[ck] = n
            n += cols[c][ck]
        M = np.zeros((m, n), dtype=A.dtype)
        rshape, cshape = {}, {}
        for key in sect[c]:
            blk = A.blocks[key]
            rk, ck = tuple(key[a] for a in row_legs), tuple(key[b] for b in col_legs)
            sub = np.transpose(blk, row_legs + col_legs).reshape(rows[c][rk], cols[c][ck])
            M[roff[rk]:roff[rk] + sub.shape[0], coff[ck]:coff[ck] + sub.shape[1]] = sub
            rshape[rk] = tuple(blk.shape[a] for a in row_legs)
            cshape[ck] = tuple(blk.shape[b] for b in col_legs)
        u, sv, vh = np.linalg.svd(M, full_matrices=False)
        k = sv.size
        for rk, o in roff.items():
            U.blocks[rk + (c,)] = u[o:o + rows[c][rk], :].reshape(rshape[rk] + (k,))
        S.blocks[(c, c)] = np.diag(sv)
        for ck, o in coff.items():
            V.blocks[(c,) + ck] = vh[:, o:o + cols[c][ck]].reshape((k,) + cshape[ck])
    return U, S, V


def eigh(A, row_legs, col_legs):
    """Block-diagonal eigendecomposition of a Hermitian matrix-shaped tensor (the
    eigen-variant of the CTM's decompositions, Sec. III; the paper leaves it to the
    backend's linear algebra). The column legs must be the duals of the row legs,
    in the same order, and n = 0, so that every sector matrix M_c is square with
    columns ordered as its rows; M_c = U_c diag(w_c) U_c^H with w_c ascending
    (numpy's eigh on the lower triangle). Returns (U, S): U on (row legs, new leg of
    signature -1), S on (new leg +1, new leg -1) with diag(w_c) per sector."""
    row_legs, col_legs = tuple(int(a) for a in row_legs), tuple(int(b) for b in col_legs)
    if len(row_legs) != len(col_legs) or sorted(row_legs + col_legs) != list(range(A.rank)):
        raise InvalidError("rows and columns must split the legs into two groups of equal size")
    if any(A.sig[a] != -A.sig[b] for a, b in zip(row_legs, col_legs)) or any(A.n):
        raise SignatureError("eigh needs dual row and column legs and n = 0")
    U, S, _ = svd(A, row_legs, col_legs)   # structure only: rows, sectors, offsets
    mods = A.mods
    Uo = OTensor(mods, U.sig, U.n, fus=list(U.fus), dtype=A.dtype)
    So = OTensor(mods, S.sig, S.n, dtype=np.float64)
    rows, sect = {}, {}
    for key, blk in A.blocks.items():
        rk, ck = tuple(key[a] for a in row_legs), tuple(key[b] for b in col_legs)
        c = tuple([0] * A.nsym)
        for a in row_legs:
            c = _add(c, _scale(A.sig[a], key[a], mods), mods)
        rows.setdefault(c, {})[rk] = tuple(blk.shape[a] for a in row_legs)
        rows[c].setdefault(ck, tuple(blk.shape[b] for b in col_legs))
        sect.setdefault(c, []).append(key)
    for c in sorted(sect):
        off, m = {}, 0
        for rk in sorted(rows[c]):
            off[rk] = m
            m += int(np.prod(rows[c][rk]))
        M = np.zeros((m, m), dtype=A.dtype)
        for key in sect[c]:
            blk = A.blocks[key]
            rk, ck = tuple(key[a] for a in row_legs), tuple(key[b] for b in col_legs)
            sub = np.transpose(blk, row_legs + col_legs).reshape(int(np.prod(rows[c][rk])), int(np.prod(rows[c][ck])))
            M[off[rk]:off[rk] + sub.shape[0], off[ck]:off[ck] + sub.shape[1]] = sub
        w, u = np.linalg.eigh(M)
        for rk, o in off.items():
            if rk + (c,) in U.blocks:
                Uo.blocks[rk + (c,)] = u[o:o + int(np.prod(rows[c][rk])), :].reshape(rows[c][rk] + (m,))
        So.blocks[(c, c)] = np.diag(w)
    return Uo, So


def truncation(S, D_total, tol=0.0):
    """Kept singular values per sector: the D_total largest over all sectors among
    those >= tol times the largest (ties kept in sector order); returns {c: kept}."""
    vals = []
    for (c, _), blk in sorted(S.blocks.items()):
        for i, v in enumerate(np.diag(blk)):
            vals.append((-float(v), c, i))
    if not vals:
        return {}
    smax = -min(v for v, _, _ in vals)
    vals = sorted(x for x in vals if -x[0] >= tol * smax)[:int(D_total)]
    keep = {c: 0 for (c, _) in S.blocks}
    for _, c, _ in vals:
        keep[c] += 1
    return keep


def slice_leg(T, legs, keep):
    """The first keep[c] indices of every sector c of the given legs (all other legs
    whole): the truncation of U, S and V to the kept singular values. Sectors kept
    at 0 drop their blocks."""
    out = OTensor(T.mods, T.sig, T.n, fus=list(T.fus), dtype=T.dtype)
    for key, blk in T.blocks.items():
        sl = [slice(None)] * T.rank
        ok = True
        for a in legs:
            k = keep.get(key[a], 0)
            if k == 0:
                ok = False
            sl[a] = slice(0, k)
        if ok:
            out.blocks[key] = np.array(blk[tuple(sl)])
    return out


# ------------------------------------------------------------------ fermionic swap gate

def charge_parity(q, mods, fermionic=None):
    """Fermionic parity (0 or 1) of one leg charge: the sum of its fermionic components
    modulo 2. ``fermionic``: one flag per symmetry component (default: all). A fermionic
    component must be U(1) (a particle number) or Z_m with m even (Z_2 parity), so
    that the parity is well defined on its charges."""
    fm = tuple(bool(x) for x in fermionic) if fermionic is not None else (True,) * len(mods)
    if len(fm) != len(mods):
        raise InvalidError("one fermionic flag per symmetry component")
    p = 0
    for c, m, f in zip(q, mods, fm):
        if f:
            if m % 2:
                raise InvalidError("a fermionic component must be U(1) or Z_m with m even")
            p += int(c)
    return p % 2


def swap_gate(A, axes1, axes2, fermionic=None):
    """Fermionic swap gate between two groups of legs (Sec. IV, use case 3): the lattice
    is projected onto a plane in a canonical fermionic order and a swap gate acts at
    every crossing of two lines; it changes the sign of the blocks whose charges have
    odd parity on both crossing lines.

    A group's parity is the parity of the sum of its legs' charges (the sum of their
    parities modulo 2; a leg signature does not change a parity). A block is multiplied
    by -1 when both groups are odd, else kept; the structure and fusion records are
    unchanged. Groups must be disjoint lists of distinct legs."""
    axes1, axes2 = tuple(int(a) for a in axes1), tuple(int(b) for b in axes2)
    allax = axes1 + axes2
    if len(set(allax)) != len(allax):
        raise InvalidError("swap-gate groups must be disjoint lists of distinct legs")
    if any(a < 0 or a >= A.rank for a in allax):
        raise InvalidError("axis out of range")
    charge_parity((0,) * A.nsym, A.mods, fermionic)   # validates the flags, also with no blocks
    out = OTensor(A.mods, A.sig, A.n, fus=list(A.fus), dtype=A.dtype)
    for key in A.keys():
        p1 = sum(charge_parity(key[a], A.mods, fermionic) for a in axes1) % 2
        p2 = sum(charge_parity(key[b], A.mods, fermionic) for b in axes2) % 2
        out.blocks[key] = -A.blocks[key] if (p1 and p2) else A.blocks[key].copy()
    return out


# ------------------------------------------------------------------ reductions

def vdot(A, B):
    """Scalar product <A, B> = sum over every element of conj(A) times the same element
    of B (the Frobenius product of the dense embeddings; for real data, A's element
    times B's).

    The paper leaves the scalar reductions of a tensor network (norms, overlaps,
    expectation values) to the backend; they are kept in FP64 here. Two tensors are
    comparable when they have the same symmetry, rank and leg signatures, one
    dimension per charge on each leg and identical fusion records; blocks present in
    only one of them contribute nothing. The sum runs over the common blocks in
    canonical order, each block's products summed with numpy. The norm is
    sqrt(vdot(A, A))."""
    if A.mods != B.mods or A.rank != B.rank:
        raise InvalidError("tensors of different symmetry or rank")
    if A.sig != B.sig:
        raise SignatureError("tensors with different leg signatures")
    for a in range(A.rank):
        da, db = leg_sectors(A, a), leg_sectors(B, a)
        for q in set(da) & set(db):
            if da[q] != db[q]:
                raise DimMismatchError(f"leg {a} charge {q}: dimension {da[q]} vs {db[q]}")
        fa, fb = A.fus[a], B.fus[a]
        if (fa is None) != (fb is None) or (fa is not None and fa.key() != fb.key()):
            raise FusionMismatchError(f"leg {a}: fusion records differ")
    cplx = np.result_type(A.dtype, B.dtype) == np.complex128
    total = 0.0 + 0.0j if cplx else 0.0
    for key in A.keys():
        if key in B.blocks:
            v = np.sum(np.conj(A.blocks[key]) * B.blocks[key])
            total += complex(v) if cplx else float(v)
    return total


# ------------------------------------------------------------------ dense embedding

def to_dense(T, legs=None):
    """Dense embedding: each leg's index runs over its sectors concatenated in ascending
    charge order; a block sits at its sectors' offsets; everything else is zero.

    ``legs``: optional list of charge -> dim maps (one per leg), to embed several tensors
    in a common basis; defaults to ``leg_sectors``."""
    if legs is None:
        legs = [leg_sectors(T, a) for a in range(T.rank)]
    offs, dims = [], []
    for lg in legs:
        o, acc = {}, 0
        for q in sorted(lg):
            o[q] = acc
            acc += lg[q]
        offs.append(o)
        dims.append(acc)
    out = np.zeros(dims, dtype=T.dtype)
    for key, blk in T.blocks.items():
        sl = tuple(slice(offs[a][key[a]], offs[a][key[a]] + blk.shape[a]) for a in range(T.rank))
        out[sl] = blk
    return out
