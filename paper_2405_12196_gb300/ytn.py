"""Python binding of the C ABI in ``include/ytn.h`` (ctypes; argument marshalling only).

Every entry point keeps the C name and forwards to ``libytn.so``; all structure work
happens in the library's planner and all data work in its CUDA kernels. Device
buffers are passed as torch CUDA tensors (or raw integer device pointers); host
block structures as the plain-array tensor records of the ``workloads`` module:
``{"mods", "sig", "n", "t": int32[nb, rank, nsym], "D": int64[nb, rank],
"fus": optional per-leg fusion records}``.

If the shared library has not been built, importing this module raises: there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libytn.so")

MAX_RANK = 16
MAX_SYM = 4

YTN_OK = 0
STATUS = {
    0: "YTN_OK", 1: "YTN_E_INVALID", 2: "YTN_E_SIGNATURE", 3: "YTN_E_DIM_MISMATCH",
    4: "YTN_E_FUSION_MISMATCH", 5: "YTN_E_NOMEM", 6: "YTN_E_CUDA", 7: "YTN_E_TIMEOUT",
    8: "YTN_E_UNSUPPORTED", 9: "YTN_E_TOLERANCE", 10: "YTN_E_CHARGE", 11: "YTN_E_WORKSPACE",
}
YTN_FP64 = 0
YTN_SPLIT_BF16 = 1
YTN_AUTO = 2
YTN_OP_TENSORDOT, YTN_OP_FUSE, YTN_OP_UNFUSE, YTN_OP_TRACE, YTN_OP_VDOT, YTN_OP_SWAP_GATE, YTN_OP_CONJ = \
    1, 2, 3, 4, 5, 6, 7
YTN_OP_SVD, YTN_OP_SLICE, YTN_OP_EIGH = 8, 9, 10
YTN_FERMIONIC_EXPLICIT = 1 << 31
YTN_REAL64, YTN_COMPLEX128 = 0, 1


class YtnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class ytn_sym(C.Structure):
    _fields_ = [("nsym", C.c_int32), ("mod", C.c_int32 * MAX_SYM)]


class ytn_fusion(C.Structure):
    _fields_ = [("nlegs", C.c_int32), ("sig", C.c_int8 * MAX_RANK), ("nentries", C.c_int64),
                ("nu", C.POINTER(C.c_int32)), ("t", C.POINTER(C.c_int32)),
                ("D", C.POINTER(C.c_int64))]


class ytn_struct(C.Structure):
    _fields_ = [("sym", ytn_sym), ("rank", C.c_int32), ("sig", C.c_int8 * MAX_RANK),
                ("n", C.c_int32 * MAX_SYM), ("nblocks", C.c_int64),
                ("t", C.POINTER(C.c_int32)), ("D", C.POINTER(C.c_int64)),
                ("off", C.POINTER(C.c_int64)), ("size", C.c_int64),
                ("fus", C.POINTER(ytn_fusion) * MAX_RANK), ("dtype", C.c_int32)]


class ytn_leg(C.Structure):
    _fields_ = [("sig", C.c_int8), ("ncharges", C.c_int32), ("t", C.POINTER(C.c_int32)), ("D", C.POINTER(C.c_int64))]


class ytn_op(C.Structure):
    _fields_ = [("kind", C.c_int), ("a", C.POINTER(ytn_struct)), ("b", C.POINTER(ytn_struct)),
                ("naxes", C.c_int32), ("axa", C.c_int32 * MAX_RANK), ("axb", C.c_int32 * MAX_RANK),
                ("ngroups", C.c_int32), ("group_size", C.c_int32 * MAX_RANK),
                ("order", C.c_int32 * MAX_RANK), ("fermionic", C.c_uint32), ("nkeep", C.c_int64),
                ("keep_t", C.POINTER(C.c_int32)), ("keep_D", C.POINTER(C.c_int64))]


class ytn_plan_info(C.Structure):
    _fields_ = [("useful_flops", C.c_double), ("nsectors", C.c_int64), ("max_m", C.c_int64),
                ("max_n", C.c_int64), ("max_k", C.c_int64), ("a_elems", C.c_int64),
                ("b_elems", C.c_int64), ("c_elems", C.c_int64), ("moved_elems", C.c_int64),
                ("out_size", C.c_int64), ("njobs", C.c_int64), ("split_fused", C.c_int32),
                ("max_copy_dims", C.c_int32), ("split_pipe_groups", C.c_int32)]


NPHASES = 8
PHASES = {0: "gather_a", 1: "gather_b", 2: "gemm", 3: "scatter", 4: "split", 5: "move", 6: "reduce", 7: "check"}


class ytn_profile(C.Structure):
    _fields_ = [("calls", C.c_int64 * NPHASES), ("ms", C.c_double * NPHASES), ("dropped", C.c_int64)]


class ytn_result(C.Structure):
    _fields_ = [("useful_flops", C.c_double), ("precision", C.c_int32), ("slices", C.c_int32),
                ("err_est", C.c_double), ("split_variant", C.c_int32), ("narrow_tiles", C.c_int32)]


class ytn_error_report(C.Structure):
    _fields_ = [("err_est", C.c_double), ("split_err_est", C.c_double), ("max_sector_est", C.c_double),
                ("fallback_flops", C.c_double), ("rtol", C.c_double), ("nsectors", C.c_int32),
                ("nfallback", C.c_int32), ("within", C.c_int32), ("slices", C.c_int32)]


class ytn_tuning(C.Structure):
    _fields_ = [("slices", C.c_int32), ("auto_choice", C.c_int32), ("split_variant", C.c_int32),
                ("tile_policy", C.c_int32), ("fp64_ms", C.c_float), ("split_ms", C.c_float),
                ("staged_ms", C.c_float), ("fused_ms", C.c_float), ("wide_ms", C.c_float),
                ("narrow_ms", C.c_float), ("pipelined_ms", C.c_float)]


class ytn_request_info(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("slot", C.c_int32), ("t_arrive", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("workspace", C.c_size_t)]


# entry points declared in include/ytn.h
SYMBOLS = {
    "ytn_ctx_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "ytn_ctx_destroy": (None, [C.c_void_p]),
    "ytn_plan": (C.c_int, [C.c_void_p, C.POINTER(ytn_op), C.POINTER(C.c_void_p)]),
    "ytn_plan_shard": (C.c_int, [C.c_void_p, C.POINTER(ytn_op), C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]),
    "ytn_plan_output": (C.POINTER(ytn_struct), [C.c_void_p]),
    "ytn_plan_blocks": (C.c_int, [C.c_void_p, ytn_sym, C.c_int32, C.POINTER(ytn_leg), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_void_p)]),
    "ytn_fill_normal": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]),
    "ytn_plan_output_at": (C.POINTER(ytn_struct), [C.c_void_p, C.c_int32]),
    "ytn_svd": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                          C.c_void_p]),
    "ytn_slice": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ytn_eigh": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "ytn_plan_get_info": (C.c_int, [C.c_void_p, C.POINTER(ytn_plan_info)]),
    "ytn_plan_tuning": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(ytn_tuning)]),
    "ytn_plan_release": (None, [C.c_void_p]),
    "ytn_workspace_size": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_size_t)]),
    "ytn_workspace_size_staged": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_size_t)]),
    "ytn_tensordot": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                C.c_void_p, C.c_size_t, C.POINTER(ytn_result), C.c_void_p]),
    "ytn_tensordot_report": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(ytn_error_report), C.c_void_p]),
    "ytn_tensordot_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ytn_fuse": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ytn_unfuse": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ytn_trace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ytn_swap_gate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ytn_conj": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ytn_ncon_plan": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.POINTER(ytn_struct)), C.POINTER(C.c_int32),
                                C.POINTER(C.c_void_p)]),
    "ytn_einsum_plan": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int32, C.POINTER(C.POINTER(ytn_struct)),
                                  C.POINTER(C.c_void_p)]),
    "ytn_ncon_output": (C.POINTER(ytn_struct), [C.c_void_p]),
    "ytn_ncon_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "ytn_ncon_workspace_size": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_size_t)]),
    "ytn_ncon": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.c_void_p, C.c_int, C.c_double, C.c_void_p,
                           C.c_size_t, C.c_void_p]),
    "ytn_ncon_release": (None, [C.c_void_p]),
    "ytn_vdot": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "ytn_sync": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "ytn_ctx_set_gemm_sms": (C.c_int, [C.c_void_p, C.c_int]),
    "ytn_selftest_timeout": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ytn_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "ytn_profile_read": (C.c_int, [C.c_void_p, C.POINTER(ytn_profile)]),
    "ytn_graph_begin": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ytn_graph_end": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "ytn_graph_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ytn_graph_destroy": (None, [C.c_void_p]),
    "ytn_server_create": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.POINTER(C.c_void_p)]),
    "ytn_server_submit": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_int, C.c_double, C.c_double]),
    "ytn_server_poll": (C.c_int, [C.c_void_p, C.POINTER(ytn_request_info), C.c_int64, C.POINTER(C.c_int64)]),
    "ytn_server_drain": (C.c_int, [C.c_void_p, C.c_int64]),
    "ytn_server_now_ms": (C.c_double, [C.c_void_p]),
    "ytn_server_destroy": (None, [C.c_void_p]),
    "ytn_last_error": (C.c_char_p, []),
    "ytn_version": (C.c_char_p, []),
}


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libytn.so is not built ({path}); run paper_2405_12196_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SYMBOLS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


def _check(status):
    if status != YTN_OK:
        raise YtnError(status, _lib.ytn_last_error().decode())


def _ptr(x):
    """Device (or host) address of a torch tensor, a numpy array or an integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ------------------------------------------------------------------ structures

class Struct:
    """A ytn_struct built from a tensor record; owns the arrays it points to."""

    def __init__(self, rec):
        mods = tuple(rec["mods"])
        t = np.ascontiguousarray(rec["t"], dtype=np.int32)
        D = np.ascontiguousarray(rec["D"], dtype=np.int64)
        nb = t.shape[0]
        rank = len(rec["sig"])
        self._keep = [t, D]
        s = ytn_struct()
        s.sym.nsym = len(mods)
        for c, m in enumerate(mods):
            s.sym.mod[c] = m
        s.rank = rank
        for i, sg in enumerate(rec["sig"]):
            s.sig[i] = sg
        for c, q in enumerate(rec["n"]):
            s.n[c] = q
        s.nblocks = nb
        s.t = t.ctypes.data_as(C.POINTER(C.c_int32))
        s.D = D.ctypes.data_as(C.POINTER(C.c_int64))
        if rec.get("off") is not None:
            off = np.ascontiguousarray(rec["off"], dtype=np.int64)
            self._keep.append(off)
            s.off = off.ctypes.data_as(C.POINTER(C.c_int64))
        sizes = np.prod(D, axis=1) if nb else np.zeros(0, np.int64)
        s.size = int(rec.get("size", int(sizes.sum()) if nb else 0))
        s.dtype = YTN_COMPLEX128 if rec.get("dtype") == "c128" else YTN_REAL64
        fus = rec.get("fus")
        self._fus = []
        if fus is not None:
            for i, f in enumerate(fus):
                if f is None:
                    continue
                nu = np.ascontiguousarray(f["nu"], dtype=np.int32)
                ft = np.ascontiguousarray(f["t"], dtype=np.int32)
                fD = np.ascontiguousarray(f["D"], dtype=np.int64)
                fz = ytn_fusion()
                fz.nlegs = len(f["sig"])
                for j, sg in enumerate(f["sig"]):
                    fz.sig[j] = sg
                fz.nentries = nu.shape[0]
                fz.nu = nu.ctypes.data_as(C.POINTER(C.c_int32))
                fz.t = ft.ctypes.data_as(C.POINTER(C.c_int32))
                fz.D = fD.ctypes.data_as(C.POINTER(C.c_int64))
                self._keep += [nu, ft, fD]
                self._fus.append(fz)
                s.fus[i] = C.pointer(fz)
        self.c = s

    @property
    def size(self):
        return self.c.size


def struct_to_record(p):
    """Copy a library-owned ytn_struct into a tensor record (numpy arrays)."""
    s = p.contents
    nsym, rank, nb = s.sym.nsym, s.rank, s.nblocks
    t = np.ctypeslib.as_array(s.t, shape=(nb * rank * nsym,)).copy().reshape(nb, rank, nsym) \
        if nb and rank else np.zeros((nb, rank, nsym), np.int32)
    D = np.ctypeslib.as_array(s.D, shape=(nb * rank,)).copy().reshape(nb, rank) \
        if nb and rank else np.zeros((nb, rank), np.int64)
    off = np.ctypeslib.as_array(s.off, shape=(nb,)).copy() if nb else np.zeros(0, np.int64)
    fus = []
    for i in range(rank):
        if not s.fus[i]:
            fus.append(None)
            continue
        f = s.fus[i].contents
        m, ne = f.nlegs, f.nentries
        if ne == 0:   # the fusion of a tensor without blocks
            fus.append({"sig": tuple(int(f.sig[j]) for j in range(m)), "nu": np.zeros((0, nsym), np.int32),
                        "t": np.zeros((0, m, nsym), np.int32), "D": np.zeros((0, m), np.int64)})
            continue
        fus.append({
            "sig": tuple(int(f.sig[j]) for j in range(m)),
            "nu": np.ctypeslib.as_array(f.nu, shape=(ne * nsym,)).copy().reshape(ne, nsym),
            "t": np.ctypeslib.as_array(f.t, shape=(ne * m * nsym,)).copy().reshape(ne, m, nsym),
            "D": np.ctypeslib.as_array(f.D, shape=(ne * m,)).copy().reshape(ne, m),
        })
    return {"mods": tuple(int(s.sym.mod[c]) for c in range(nsym)),
            "sig": tuple(int(s.sig[i]) for i in range(rank)),
            "n": tuple(int(s.n[c]) for c in range(nsym)), "t": t, "D": D, "off": off,
            "size": int(s.size), "fus": fus if any(f is not None for f in fus) else None,
            **({"dtype": "c128"} if s.dtype == YTN_COMPLEX128 else {})}


# ------------------------------------------------------------------ entry points

class Ctx:
    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        h, self.handle = self.handle, None
        if h:
            _lib.ytn_ctx_destroy(h)


class Plan:
    def __init__(self, ctx, handle, keep):
        self.ctx = ctx
        self.handle = handle
        self._keep = keep
        self.out = struct_to_record(_lib.ytn_plan_output(handle))
        self.outs = [self.out]
        i = 1
        while True:   # further outputs (SVD: U, S, V)
            ptr = _lib.ytn_plan_output_at(handle, i)
            if not ptr:
                break
            self.outs.append(struct_to_record(ptr))
            i += 1
        info = ytn_plan_info()
        _check(_lib.ytn_plan_get_info(handle, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in ytn_plan_info._fields_}

    def release(self):
        h, self.handle = self.handle, None
        if h and self.ctx.handle:
            _lib.ytn_plan_release(h)

    def __del__(self):
        self.release()


class Ncon:
    """A planned network (ytn_ncon_plan): output record, useful FLOPs, call count."""

    def __init__(self, ctx, handle, keep):
        self.ctx = ctx
        self.handle = handle
        self._keep = keep
        self.out = struct_to_record(_lib.ytn_ncon_output(handle))
        fl, nc = C.c_double(), C.c_int32()
        _check(_lib.ytn_ncon_info(handle, C.byref(fl), C.byref(nc)))
        self.info = {"useful_flops": fl.value, "ncalls": nc.value}

    def release(self):
        h, self.handle = self.handle, None
        if h and self.ctx.handle:
            _lib.ytn_ncon_release(h)

    def __del__(self):
        self.release()


def ytn_version():
    return _lib.ytn_version().decode()


def ytn_ctx_create(device=0):
    h = C.c_void_p()
    _check(_lib.ytn_ctx_create(C.byref(h), int(device)))
    return Ctx(h.value)


def ytn_plan(ctx, kind, a, b=None, axa=(), axb=(), groups=None, fermionic=None, keep=None, shard=None):
    """Plan an operation. ``a``/``b``: tensor records. ``kind``: one of YTN_OP_*.
    TENSORDOT: pairs (axa[k], axb[k]); FUSE: ``groups`` (list of leg tuples);
    UNFUSE: legs ``axa``; TRACE: pairs (axa[k], axb[k]) of ``a``; SWAP_GATE: two
    ``groups`` and ``fermionic`` (one flag per symmetry component; None = all).
    ``shard=(rank, world)``: this rank's part of a TENSORDOT (ytn_plan_shard)."""
    sa = Struct(a)
    sb = Struct(b) if b is not None else None
    op = ytn_op()
    op.kind = kind
    op.a = C.pointer(sa.c)
    op.b = C.pointer(sb.c) if sb is not None else None
    op.naxes = len(axa)
    for k, x in enumerate(axa):
        op.axa[k] = x
    for k, x in enumerate(axb):
        op.axb[k] = x
    if groups is not None:
        gs = [tuple(g) if isinstance(g, (tuple, list)) else (g,) for g in groups]
        op.ngroups = len(gs)
        flat = [x for g in gs for x in g]
        for k, g in enumerate(gs):
            op.group_size[k] = len(g)
        for k, x in enumerate(flat):
            op.order[k] = x
    if fermionic is not None:
        op.fermionic = YTN_FERMIONIC_EXPLICIT | sum(1 << c for c, f in enumerate(fermionic) if f)
    keep_arrays = ()
    if keep is not None:   # SLICE: {charge tuple: kept dimension}
        kt = np.ascontiguousarray([list(q) for q in keep] or [[0]], dtype=np.int32)
        kd = np.ascontiguousarray(list(keep.values()) or [0], dtype=np.int64)
        op.nkeep = len(keep)
        op.keep_t = kt.ctypes.data_as(C.POINTER(C.c_int32))
        op.keep_D = kd.ctypes.data_as(C.POINTER(C.c_int64))
        keep_arrays = (kt, kd)
    h = C.c_void_p()
    if shard is None:
        _check(_lib.ytn_plan(ctx.handle, C.byref(op), C.byref(h)))
    else:
        _check(_lib.ytn_plan_shard(ctx.handle, C.byref(op), int(shard[0]), int(shard[1]), C.byref(h)))
    return Plan(ctx, h.value, (sa, sb, keep_arrays))


def ytn_plan_blocks(ctx, mods, legs, n):
    """The structure of a tensor on ``legs`` (objects with ``s``, ``t``, ``D``: sig,
    charge tuples, dims) with total charge ``n``: every allowed block."""
    sym = ytn_sym()
    sym.nsym = len(mods)
    for c, m in enumerate(mods):
        sym.mod[c] = m
    arrs, cl = [], (ytn_leg * len(legs))()
    for i, l in enumerate(legs):
        t = np.ascontiguousarray(np.asarray(l.t, dtype=np.int32).reshape(-1, len(mods)))
        d = np.ascontiguousarray(l.D, dtype=np.int64)
        arrs += [t, d]
        cl[i].sig, cl[i].ncharges = int(l.s), len(d)
        cl[i].t = t.ctypes.data_as(C.POINTER(C.c_int32))
        cl[i].D = d.ctypes.data_as(C.POINTER(C.c_int64))
    nn = (C.c_int32 * MAX_SYM)(*[int(x) for x in n])
    h = C.c_void_p()
    _check(_lib.ytn_plan_blocks(ctx.handle, sym, len(legs), cl, nn, C.byref(h)))
    return Plan(ctx, h.value, (arrs, cl))


def ytn_fill_normal(plan, seed, out, stream=None):
    """N(0, 1) numbers (Philox4x32-10, Box-Muller) into ``out`` (the plan's output size)."""
    _check(_lib.ytn_fill_normal(plan.handle, int(seed), _ptr(out), _stream(stream)))


def ytn_workspace_size(plan, prec=YTN_FP64, rtol=0.0):
    n = C.c_size_t()
    _check(_lib.ytn_workspace_size(plan.handle, prec, float(rtol), C.byref(n)))
    return n.value


def ytn_workspace_size_staged(plan, prec=YTN_FP64, rtol=0.0):
    """Workspace with which host operands are staged by the copy engines."""
    n = C.c_size_t()
    _check(_lib.ytn_workspace_size_staged(plan.handle, prec, float(rtol), C.byref(n)))
    return n.value


def ytn_tensordot(plan, a, b, c, prec=YTN_FP64, rtol=0.0, workspace=None, workspace_bytes=None,
                  stream=None):
    res = ytn_result()
    if workspace_bytes is None:
        workspace_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(_lib.ytn_tensordot(plan.handle, _ptr(a), _ptr(b), _ptr(c), prec, float(rtol),
                              _ptr(workspace), int(workspace_bytes), C.byref(res), _stream(stream)))
    return {"useful_flops": res.useful_flops, "precision": res.precision, "slices": res.slices,
            "err_est": res.err_est, "split_variant": res.split_variant, "narrow_tiles": res.narrow_tiles}


def ytn_ncon_plan(ctx, records, labels):
    """Plan the network of tensor ``records`` with ncon ``labels`` (one list per tensor)."""
    structs = [Struct(r) for r in records]
    arr = (C.POINTER(ytn_struct) * len(structs))(*[C.pointer(x.c) for x in structs])
    flat = np.ascontiguousarray([int(x) for lab in labels for x in lab] or [0], dtype=np.int32)
    h = C.c_void_p()
    _check(_lib.ytn_ncon_plan(ctx.handle, len(structs), arr, flat.ctypes.data_as(C.POINTER(C.c_int32)),
                              C.byref(h)))
    return Ncon(ctx, h.value, (structs, arr, flat))


def ytn_einsum_plan(ctx, subscripts, records):
    """Plan the network of tensor ``records`` given by einsum ``subscripts``."""
    structs = [Struct(r) for r in records]
    arr = (C.POINTER(ytn_struct) * len(structs))(*[C.pointer(x.c) for x in structs])
    h = C.c_void_p()
    _check(_lib.ytn_einsum_plan(ctx.handle, subscripts.encode(), len(structs), arr, C.byref(h)))
    return Ncon(ctx, h.value, (structs, arr))


def ytn_ncon_workspace_size(nc, prec=YTN_FP64, rtol=0.0):
    n = C.c_size_t()
    _check(_lib.ytn_ncon_workspace_size(nc.handle, prec, float(rtol), C.byref(n)))
    return n.value


def ytn_ncon(nc, data, out, prec=YTN_FP64, rtol=0.0, workspace=None, workspace_bytes=None, stream=None):
    """Run a planned network: ``data`` one buffer per tensor, ``out`` the output buffer."""
    if workspace_bytes is None:
        workspace_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    ptrs = (C.c_void_p * len(data))(*[_ptr(d) for d in data])
    _check(_lib.ytn_ncon(nc.handle, ptrs, _ptr(out), prec, float(rtol), _ptr(workspace), int(workspace_bytes),
                         _stream(stream)))


def ytn_tensordot_report(plan, workspace, stream=None):
    """Accuracy record of the last split-precision call of ``plan`` in ``workspace``
    (waits for ``stream``): data-aware error estimate after the FP64 fallback, the
    split products' estimate, recomputed sectors."""
    r = ytn_error_report()
    _check(_lib.ytn_tensordot_report(plan.handle, _ptr(workspace), C.byref(r), _stream(stream)))
    return {k: getattr(r, k) for k, _ in ytn_error_report._fields_}


def ytn_plan_tuning(plan, slices):
    """The split-precision choices the plan's first calls made with ``slices`` slices
    (-1: undecided) and the candidates' timings in ms (0: not timed)."""
    t = ytn_tuning()
    _check(_lib.ytn_plan_tuning(plan.handle, int(slices), C.byref(t)))
    return {k: getattr(t, k) for k, _ in ytn_tuning._fields_}


def ytn_tensordot_noalloc(plan, a, b, c, stream=None):
    """FP64 contraction with the library's static scratch instead of a caller
    workspace (for callers that cannot allocate device memory)."""
    _check(_lib.ytn_tensordot_noalloc(plan.handle, _ptr(a), _ptr(b), _ptr(c), _stream(stream)))


def ytn_fuse(plan, a, out, stream=None):
    _check(_lib.ytn_fuse(plan.handle, _ptr(a), _ptr(out), _stream(stream)))


def ytn_unfuse(plan, a, out, stream=None):
    _check(_lib.ytn_unfuse(plan.handle, _ptr(a), _ptr(out), _stream(stream)))


def ytn_trace(plan, a, out, stream=None):
    _check(_lib.ytn_trace(plan.handle, _ptr(a), _ptr(out), _stream(stream)))


def ytn_swap_gate(plan, a, out, stream=None):
    """out = swap_gate(a) for a SWAP_GATE plan; ``out`` may be ``a`` (in place)."""
    _check(_lib.ytn_swap_gate(plan.handle, _ptr(a), _ptr(out), _stream(stream)))


def ytn_svd(plan, a, u, s, v, workspace=None, workspace_bytes=None, stream=None):
    """U, S, V of an SVD plan into ``u``, ``s``, ``v`` (sizes of ``plan.outs``)."""
    if workspace_bytes is None:
        workspace_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(_lib.ytn_svd(plan.handle, _ptr(a), _ptr(u), _ptr(s), _ptr(v), _ptr(workspace), int(workspace_bytes),
                        _stream(stream)))


def ytn_eigh(plan, a, u, s, workspace=None, workspace_bytes=None, stream=None):
    """U, S of an EIGH plan into ``u``, ``s`` (sizes of ``plan.outs``)."""
    if workspace_bytes is None:
        workspace_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(_lib.ytn_eigh(plan.handle, _ptr(a), _ptr(u), _ptr(s), _ptr(workspace), int(workspace_bytes),
                         _stream(stream)))


def ytn_slice(plan, a, out, stream=None):
    _check(_lib.ytn_slice(plan.handle, _ptr(a), _ptr(out), _stream(stream)))


def ytn_conj(plan, a, out, stream=None):
    """out = conj(a) for a CONJ plan; ``out`` may be ``a`` (in place)."""
    _check(_lib.ytn_conj(plan.handle, _ptr(a), _ptr(out), _stream(stream)))


def ytn_vdot(plan, a, b, out, workspace=None, workspace_bytes=None, stream=None):
    """out[0] = <A, B> (a VDOT plan); `out` holds one double."""
    if workspace_bytes is None:
        workspace_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(_lib.ytn_vdot(plan.handle, _ptr(a), _ptr(b), _ptr(out), _ptr(workspace), int(workspace_bytes),
                         _stream(stream)))


def ytn_sync(ctx, stream=None, timeout_ms=-1):
    _check(_lib.ytn_sync(ctx.handle, _stream(stream), int(timeout_ms)))


def ytn_selftest_timeout(ctx, stream=None):
    _check(_lib.ytn_selftest_timeout(ctx.handle, _stream(stream)))


def ytn_ctx_set_gemm_sms(ctx, nsms):
    _check(_lib.ytn_ctx_set_gemm_sms(ctx.handle, int(nsms)))


def ytn_profile_enable(ctx, enable=True):
    _check(_lib.ytn_profile_enable(ctx.handle, 1 if enable else 0))


def ytn_profile_read(ctx):
    """Per-phase {name: (calls, total ms)} recorded since the last read, plus 'dropped'."""
    p = ytn_profile()
    _check(_lib.ytn_profile_read(ctx.handle, C.byref(p)))
    out = {PHASES.get(i, str(i)): (int(p.calls[i]), float(p.ms[i])) for i in range(NPHASES) if p.calls[i]}
    out["dropped"] = int(p.dropped)
    return out


def available_precisions():
    """Precisions this build of the library executes."""
    return [YTN_FP64, YTN_SPLIT_BF16, YTN_AUTO]


# ------------------------------------------------------------------ graphs

class Graph:
    """A recorded sequence of library calls (ytn_graph_*), replayed by launch()."""

    def __init__(self, handle):
        self.handle = handle

    def launch(self, stream):
        _check(_lib.ytn_graph_launch(self.handle, _stream(stream)))

    def close(self):
        h, self.handle = self.handle, None
        if h:
            _lib.ytn_graph_destroy(h)

    def __del__(self):
        self.close()


def ytn_graph_begin(ctx, stream):
    _check(_lib.ytn_graph_begin(ctx.handle, _stream(stream)))


def ytn_graph_end(ctx, stream):
    h = C.c_void_p()
    _check(_lib.ytn_graph_end(ctx.handle, _stream(stream), C.byref(h)))
    return Graph(h.value)


# ------------------------------------------------------------------ serving

class Server:
    """Continuous-batching server (ytn_server_*): `arena` is a device buffer (torch
    uint8 tensor) that bounds the workspace of admitted requests."""

    def __init__(self, ctx, nslots, arena):
        self.ctx = ctx
        self.arena = arena
        h = C.c_void_p()
        _check(_lib.ytn_server_create(ctx.handle, int(nslots), _ptr(arena),
                                      arena.numel() * arena.element_size(), C.byref(h)))
        self.handle = h.value

    def submit(self, rid, plan, a, b, c, prec=YTN_FP64, rtol=0.0, t_arrive=-1.0):
        _check(_lib.ytn_server_submit(self.handle, int(rid), plan.handle, _ptr(a), _ptr(b), _ptr(c), prec,
                                      float(rtol), float(t_arrive)))

    def poll(self, max_n=4096):
        buf = (ytn_request_info * max_n)()
        n = C.c_int64()
        _check(_lib.ytn_server_poll(self.handle, buf, max_n, C.byref(n)))
        return [{k: getattr(buf[i], k) for k, _ in ytn_request_info._fields_} for i in range(n.value)]

    def drain(self, timeout_ms=-1):
        _check(_lib.ytn_server_drain(self.handle, int(timeout_ms)))

    def now_ms(self):
        return _lib.ytn_server_now_ms(self.handle)

    def close(self):
        h, self.handle = self.handle, None
        if h:
            _lib.ytn_server_destroy(h)

    def __del__(self):
        self.close()


def ytn_server_create(ctx, nslots, arena):
    return Server(ctx, nslots, arena)
