"""ctypes binding of the C ABI in include/dh2.h (argument marshalling only).

Every compute step runs in the CUDA library `libdh2.so`; this module only
converts numpy arrays / torch tensors into pointers, sizes and the current
CUDA stream, and turns status codes into exceptions.  There is no fallback:
if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_float, c_int32, c_int64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdh2.so")

DH2_C64 = 0
DH2_C128 = 1
MODE_FP64 = 0
MODE_FP32 = 1
MODE_MIXED_BF16X3 = 2
SIDE_ROW = 0
SIDE_COL = 1
# kernel classes of Matrix.class_launches (DH2_KC_* in include/dh2.h)
KC_LEAF_FACTOR = 0
KC_LEAF_R = 5
KC_LEVEL_FACTOR = 10
KC_LEVEL_R = 14
KC_NORMS = 15
KC_COLW = 16
KC_CLASSIFY = 17
KC_EXPAND = 18
KC_PROJECT = 19
KC_LEAF_GRAM = 20
KC_GRAM_SCALES = 24
KC_LEAF_JACOBI = 25
KC_LEAF_R_TC = 29
KC_GRAM_SCALES = 24
KC_COUNT = 32


class TreeParams(ctypes.Structure):
    _fields_ = [("leaf_size", c_int32), ("dir_rule", c_int32), ("kappa", c_double),
                ("eta1", c_double), ("eta2", c_double)]


class CompressParams(ctypes.Structure):
    _fields_ = [("eps", c_double), ("zeta", c_double), ("err_mode", c_int32), ("mode", c_int32),
                ("nearfield", c_int32), ("max_sweeps", c_int32), ("rank_override", c_void_p * 2),
                ("spin_limit", c_int64), ("keep_gram", c_int32), ("reserved", c_int32)]


def _params(eps, zeta, err_mode, mode, nearfield, max_sweeps, rank_override=None, spin_limit=0, keep_gram=0):
    """dh2_compress_params; rank_override: None or (row ranks, column ranks), each None or int32 per pair
    (kept alive on the returned structure until the call returns)."""
    p = CompressParams(float(eps), float(zeta), int(err_mode), int(mode), int(nearfield), int(max_sweeps))
    p.spin_limit = int(spin_limit)
    p.keep_gram = int(keep_gram)
    keep = []
    if rank_override is not None:
        for sd in (0, 1):
            r = rank_override[sd]
            if r is not None:
                a = np.ascontiguousarray(r, dtype=np.int32)
                keep.append(a)
                p.rank_override[sd] = a.ctypes.data
    p._keep = keep
    return p


class TreeStats(ctypes.Structure):
    _fields_ = [("n", c_int64), ("depth", c_int32), ("nclusters", c_int32), ("nblocks", c_int64),
                ("nadmissible", c_int64), ("adm_fraction", c_double), ("npairs", c_int64 * 2),
                ("nleafpairs", c_int64 * 2), ("ncolumns", c_int64 * 2), ("nleafcolumns", c_int64 * 2),
                ("max_leaf", c_int32), ("ndirs_max", c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("jacobi_tpp", c_int32 * 5), ("jacobi_narrow", c_int32 * 4), ("rq_ctas_per_sm", c_int32),
                ("rq_tensor", c_int32), ("level_seg_cols", c_int32)]


class TuneRecord(ctypes.Structure):
    _fields_ = [("knob", c_int32), ("cls", c_int32), ("value", c_int32), ("ms", ctypes.c_float)]


TUNE_KNOBS = ("rq_ctas_per_sm", "jacobi_narrow", "jacobi_tpp", "rq_tensor", "level_seg_cols")


def _tuning_dict(t: Tuning) -> dict:
    return {"jacobi_tpp": list(t.jacobi_tpp), "jacobi_narrow": list(t.jacobi_narrow),
            "rq_ctas_per_sm": int(t.rq_ctas_per_sm), "rq_tensor": int(t.rq_tensor),
            "level_seg_cols": int(t.level_seg_cols)}


class DH2Error(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_lib().dh2_status_string(status).decode()} (status {status})")


_LIB = None

# (name, restype, argtypes) of every entry point declared in include/dh2.h
SIGNATURES = [
    ("dh2_tree_build", c_int32, [c_void_p, c_int64, POINTER(TreeParams), POINTER(c_void_p)]),
    ("dh2_tree_free", None, [c_void_p]),
    ("dh2_tree_stats_get", c_int32, [c_void_p, POINTER(TreeStats)]),
    ("dh2_tree_perm", c_int32, [c_void_p, c_void_p]),
    ("dh2_tree_clusters", c_int32, [c_void_p] + [c_void_p] * 8),
    ("dh2_tree_ndirs", c_int32, [c_void_p, c_int32, POINTER(c_int32)]),
    ("dh2_tree_directions", c_int32, [c_void_p, c_int32, c_void_p, c_void_p]),
    ("dh2_tree_blocks", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("dh2_tree_pairs", c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("dh2_tree_pair_blocks", c_int32, [c_void_p, c_int32, c_void_p, c_void_p]),
    ("dh2_tree_panels", c_int32, [c_void_p, POINTER(c_int32), c_void_p, c_void_p]),
    ("dh2_compress", c_int32, [c_void_p, c_void_p, c_int32, c_int64, POINTER(CompressParams), c_void_p,
                               POINTER(c_void_p)]),
    ("dh2_compress_host", c_int32, [c_void_p, c_void_p, c_int32, c_int64, POINTER(CompressParams), c_void_p,
                                    POINTER(c_void_p)]),
    ("dh2_compress_batched", c_int32, [c_int32, c_void_p, c_void_p, c_void_p, c_int32, POINTER(CompressParams),
                                       c_void_p, c_void_p]),
    ("dh2_compress_kernel", c_int32, [c_void_p, c_void_p, c_double, c_double, POINTER(CompressParams), c_void_p,
                                      POINTER(c_void_p)]),
    ("dh2_compress_kernel_dlp", c_int32, [c_void_p, c_void_p, c_void_p, c_double, POINTER(CompressParams),
                                          c_void_p, POINTER(c_void_p)]),
    ("dh2_matrix_free", None, [c_void_p]),
    ("dh2_plan_create", c_int32, [c_int32, c_void_p, c_void_p, c_void_p, c_int32, POINTER(CompressParams), c_void_p,
                                  POINTER(c_void_p)]),
    ("dh2_plan_run", c_int32, [c_void_p, c_void_p, c_void_p]),
    ("dh2_plan_wait", c_int32, [c_void_p, c_void_p]),
    ("dh2_plan_matrix", c_int32, [c_void_p, c_int32, POINTER(c_void_p)]),
    ("dh2_plan_free", None, [c_void_p]),
    ("dh2_tuning_get", c_int32, [POINTER(Tuning)]),
    ("dh2_tuning_set", c_int32, [POINTER(Tuning)]),
    ("dh2_autotune", c_int32, [c_void_p, c_void_p, c_int32, c_int64, POINTER(CompressParams), c_void_p, c_int32,
                               POINTER(Tuning), c_void_p, c_int32, POINTER(c_int32)]),
    ("dh2_matvec", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    ("dh2_matvec_noalloc", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    ("dh2_matvec_adjoint", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    ("dh2_error", c_int32, [c_void_p, c_void_p, c_int32, c_int64, c_int32, c_void_p, POINTER(c_double)]),
    ("dh2_matrix_ranks", c_int32, [c_void_p, c_int32, c_void_p]),
    ("dh2_matrix_sigma", c_int32, [c_void_p, c_int32, c_int64, c_void_p, c_int32, POINTER(c_int32)]),
    ("dh2_matrix_sigma_rest", c_int32, [c_void_p, c_int32, c_int64, POINTER(c_double)]),
    ("dh2_matrix_pair_basis", c_int32, [c_void_p, c_int32, c_int64, c_void_p, c_int64, POINTER(c_int32),
                                        POINTER(c_int32)]),
    ("dh2_matrix_coupling", c_int32, [c_void_p, c_int64, c_void_p, c_int64, POINTER(c_int32), POINTER(c_int32)]),
    ("dh2_storage", c_int32, [c_void_p, POINTER(c_double), c_void_p]),
    ("dh2_matrix_phase_ms", c_int32, [c_void_p, c_void_p]),
    ("dh2_matrix_leaf_split_ms", c_int32, [c_void_p, c_void_p]),
    ("dh2_matrix_launch_count", c_int32, [c_void_p, c_void_p]),
    ("dh2_matrix_class_launches", c_int32, [c_void_p, c_void_p]),
    ("dh2_matrix_block_weights", c_int32, [c_void_p, c_void_p]),
    ("dh2_matrix_leaf_gram", c_int32, [c_void_p, c_int32, c_int64, c_void_p, c_int64, POINTER(c_int32)]),
    ("dh2_debug_fail_alloc", c_int32, [c_int32]),
    ("dh2_status_string", ctypes.c_char_p, [c_int32]),
    ("dh2_version", ctypes.c_char_p, []),
]


def _lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libdh2.so is not built ({LIB_PATH}); run `python -m paper_1510_07087_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def _check(status: int, what: str) -> None:
    if status != 0:
        raise DH2Error(status, what)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ------------------------------------------------------------------ tree

class Tree:
    """Owner of a dh2_tree handle."""

    def __init__(self, handle: int, n: int):
        self.handle = c_void_p(handle)
        self.n = n

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value:
            _lib().dh2_tree_free(self.handle)
            self.handle = c_void_p()

    # queries
    def stats(self) -> TreeStats:
        st = TreeStats()
        _check(_lib().dh2_tree_stats_get(self.handle, byref(st)), "dh2_tree_stats_get")
        return st

    def perm(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int64)
        _check(_lib().dh2_tree_perm(self.handle, _ptr(out)), "dh2_tree_perm")
        return out

    def clusters(self) -> dict:
        nc = self.stats().nclusters
        d = {k: np.empty(nc, dtype=np.int32) for k in ("start", "size", "level", "parent", "son0", "son1")}
        lo = np.empty((nc, 3))
        hi = np.empty((nc, 3))
        _check(_lib().dh2_tree_clusters(self.handle, *[_ptr(d[k]) for k in ("start", "size", "level", "parent",
                                                                             "son0", "son1")], _ptr(lo), _ptr(hi)),
               "dh2_tree_clusters")
        d["lo"], d["hi"] = lo, hi
        return d

    def directions(self, level: int):
        nd = c_int32()
        _check(_lib().dh2_tree_ndirs(self.handle, level, byref(nd)), "dh2_tree_ndirs")
        D = np.empty((nd.value, 3))
        sd = np.empty(nd.value, dtype=np.int32)
        _check(_lib().dh2_tree_directions(self.handle, level, _ptr(D), _ptr(sd)), "dh2_tree_directions")
        return D, sd

    def blocks(self) -> np.ndarray:
        nb = self.stats().nblocks
        arr = [np.empty(nb, dtype=np.int32) for _ in range(4)]
        _check(_lib().dh2_tree_blocks(self.handle, *[_ptr(a) for a in arr]), "dh2_tree_blocks")
        return np.stack(arr, axis=1)

    def pairs(self, side: int) -> dict:
        np_ = self.stats().npairs[side]
        cl = np.empty(np_, dtype=np.int32)
        di = np.empty(np_, dtype=np.int32)
        nc = np.empty(np_, dtype=np.int64)
        lf = np.empty(np_, dtype=np.int32)
        _check(_lib().dh2_tree_pairs(self.handle, side, _ptr(cl), _ptr(di), _ptr(nc), _ptr(lf)), "dh2_tree_pairs")
        return {"cluster": cl, "dir": di, "ncols": nc, "leaf": lf}

    def pair_blocks(self, side: int):
        np_ = self.stats().npairs[side]
        off = np.empty(np_ + 1, dtype=np.int64)
        _check(_lib().dh2_tree_pair_blocks(self.handle, side, _ptr(off), None), "dh2_tree_pair_blocks")
        ids = np.empty(max(1, int(off[-1])), dtype=np.int32)
        _check(_lib().dh2_tree_pair_blocks(self.handle, side, _ptr(off), _ptr(ids)), "dh2_tree_pair_blocks")
        return off, ids[:int(off[-1])]

    def panels(self):
        """Column panels of the host-input compression: boundaries and, per row-basis pair, the
        panel after which its leaf factor runs (-1 for non-leaf pairs)."""
        k = c_int32()
        _check(_lib().dh2_tree_panels(self.handle, byref(k), None, None), "dh2_tree_panels")
        col = np.empty(k.value + 1, dtype=np.int64)
        rp = np.empty(self.stats().npairs[0], dtype=np.int32)
        _check(_lib().dh2_tree_panels(self.handle, byref(k), _ptr(col), _ptr(rp)), "dh2_tree_panels")
        return col, rp


def dh2_tree_build(points: np.ndarray, leaf_size: int = 32, kappa: float = 4.0,
                   eta1: float = 2.0 * np.sqrt(2.0), eta2: float = 1.0, dir_rule: int = 0) -> Tree:
    pts = np.ascontiguousarray(points, dtype=np.float64)
    if pts.ndim != 2 or pts.shape[1] != 3:
        raise ValueError("points must be (n, 3)")
    p = TreeParams(int(leaf_size), int(dir_rule), float(kappa), float(eta1), float(eta2))
    h = c_void_p()
    _check(_lib().dh2_tree_build(_ptr(pts), pts.shape[0], byref(p), byref(h)), "dh2_tree_build")
    return Tree(h.value, pts.shape[0])


# ------------------------------------------------------------------ matrix

def _stream_handle(stream) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dtype_code(t) -> int:
    import torch

    if t.dtype == torch.complex64:
        return DH2_C64
    if t.dtype == torch.complex128:
        return DH2_C128
    raise TypeError(f"unsupported dtype {t.dtype}")


def _colmajor_ld(G) -> int:
    if G.dim() != 2 or G.stride(0) != 1 or G.stride(1) < G.shape[0]:
        raise ValueError("G must be a column-major (n, n) view: stride (1, ld) with ld >= n")
    return int(G.stride(1))


class Matrix:
    """Owner of a dh2_matrix handle (device-resident DH^2 representation)."""

    def __init__(self, handle: int, tree: Tree, mode: int, G, owner=None):
        self.handle = c_void_p(handle)
        self.tree = tree
        self.mode = mode
        self._G = G  # keeps a viewed nearfield alive
        self._owner = owner  # a Plan that owns the handle (None: this object owns it)

    def __del__(self):
        if self._owner is None and getattr(self, "handle", None) and self.handle.value:
            _lib().dh2_matrix_free(self.handle)
        self.handle = c_void_p()

    def ranks(self, side: int) -> np.ndarray:
        out = np.empty(self.tree.stats().npairs[side], dtype=np.int32)
        _check(_lib().dh2_matrix_ranks(self.handle, side, _ptr(out)), "dh2_matrix_ranks")
        return out

    def sigma(self, side: int, pair: int) -> np.ndarray:
        """Singular values resolved individually (descending)."""
        out = np.empty(128)
        cnt = c_int32()
        _check(_lib().dh2_matrix_sigma(self.handle, side, pair, _ptr(out), 128, byref(cnt)), "dh2_matrix_sigma")
        return out[:min(cnt.value, 128)].copy()

    def sigma_rest(self, side: int, pair: int) -> float:
        """Sum of squares of the singular values not resolved individually."""
        e = c_double()
        _check(_lib().dh2_matrix_sigma_rest(self.handle, side, pair, byref(e)), "dh2_matrix_sigma_rest")
        return float(e.value)

    def pair_basis(self, side: int, pair: int) -> np.ndarray:
        cap = 128 * 128
        out = np.empty(2 * cap)
        rows, k = c_int32(), c_int32()
        _check(_lib().dh2_matrix_pair_basis(self.handle, side, pair, _ptr(out), cap, byref(rows), byref(k)),
               "dh2_matrix_pair_basis")
        r, kk = rows.value, k.value
        return out[:2 * r * kk].view(np.complex128).reshape(kk, r).T.copy()

    def coupling(self, block: int) -> np.ndarray:
        cap = 128 * 128
        out = np.empty(2 * cap)
        kt, ks = c_int32(), c_int32()
        _check(_lib().dh2_matrix_coupling(self.handle, block, _ptr(out), cap, byref(kt), byref(ks)),
               "dh2_matrix_coupling")
        a, b = kt.value, ks.value
        return out[:2 * a * b].view(np.complex128).reshape(b, a).T.copy()

    def storage(self) -> dict:
        tot = c_double()
        parts = np.zeros(6)
        _check(_lib().dh2_storage(self.handle, byref(tot), _ptr(parts)), "dh2_storage")
        keys = ["V", "W", "E_V", "E_W", "S", "near"]
        d = {k: float(v) for k, v in zip(keys, parts)}
        d["total"] = float(tot.value)
        return d

    def launch_count(self) -> int:
        out = c_int32(0)
        _check(_lib().dh2_matrix_launch_count(self.handle, byref(out)), "dh2_matrix_launch_count")
        return int(out.value)

    def block_weights(self) -> np.ndarray:
        """1/omega_b per block (Remark "Error control")."""
        out = np.empty(max(1, int(self.tree.stats().nblocks)))
        _check(_lib().dh2_matrix_block_weights(self.handle, _ptr(out)), "dh2_matrix_block_weights")
        return out[:int(self.tree.stats().nblocks)]

    def leaf_gram(self, side: int, pair: int) -> np.ndarray:
        """The tensor-core Gram matrix of a leaf pair (compressed with keep_gram=1), complex128."""
        cap = 64 * 64
        out = np.empty(2 * cap)
        m = c_int32()
        _check(_lib().dh2_matrix_leaf_gram(self.handle, side, pair, _ptr(out), cap, byref(m)), "dh2_matrix_leaf_gram")
        k = m.value
        return out[:2 * k * k].view(np.complex128).reshape(k, k).T.copy()

    def class_launches(self) -> np.ndarray:
        """Launches of the last compression by kernel class (KC_* indices)."""
        out = np.zeros(KC_COUNT, dtype=np.int32)
        _check(_lib().dh2_matrix_class_launches(self.handle, _ptr(out)), "dh2_matrix_class_launches")
        return out

    def phase_ms(self) -> np.ndarray:
        out = np.zeros(6, dtype=np.float32)
        _check(_lib().dh2_matrix_phase_ms(self.handle, _ptr(out)), "dh2_matrix_phase_ms")
        return out

    def leaf_split_ms(self) -> np.ndarray:
        """Mixed modes, device input: the leaf phase as [Gram launches, factor launches] in ms."""
        out = np.zeros(2, dtype=np.float32)
        _check(_lib().dh2_matrix_leaf_split_ms(self.handle, _ptr(out)), "dh2_matrix_leaf_split_ms")
        return out


def dh2_compress(tree: Tree, G, eps: float = 1e-4, zeta: float = 2.0 / 3.0, err_mode: int = 0,
                 mode: int | None = None, nearfield: int = 0, max_sweeps: int = 0, stream=None,
                 rank_override=None, spin_limit: int = 0, keep_gram: int = 0) -> Matrix:
    """Compress a device matrix G (torch, column-major view, tree's permuted order).

    rank_override: None or (row ranks, column ranks) per used pair (dh2_tree_pairs order), entries < 0
    keep the truncation rule; spin_limit, keep_gram: see dh2_compress_params in include/dh2.h."""
    dt = _dtype_code(G)
    if mode is None:
        mode = MODE_FP32 if dt == DH2_C64 else MODE_FP64
    ld = _colmajor_ld(G)
    p = _params(eps, zeta, err_mode, mode, nearfield, max_sweeps, rank_override, spin_limit, keep_gram)
    h = c_void_p()
    _check(_lib().dh2_compress(tree.handle, c_void_p(G.data_ptr()), dt, ld, byref(p),
                               c_void_p(_stream_handle(stream)), byref(h)), "dh2_compress")
    return Matrix(h.value, tree, mode, G)


def tuning() -> dict:
    """The process's tuning table (dh2_tuning_get)."""
    t = Tuning()
    _check(_lib().dh2_tuning_get(byref(t)), "dh2_tuning_get")
    return _tuning_dict(t)


def set_tuning(d: dict) -> None:
    """Install a tuning table (dh2_tuning_set); keys as returned by tuning()."""
    t = Tuning()
    for c, v in enumerate(d["jacobi_tpp"]):
        t.jacobi_tpp[c] = int(v)
    for c, v in enumerate(d["jacobi_narrow"]):
        t.jacobi_narrow[c] = int(v)
    t.rq_ctas_per_sm = int(d["rq_ctas_per_sm"])
    t.rq_tensor = int(d.get("rq_tensor", 0))
    t.level_seg_cols = int(d.get("level_seg_cols", 1024))
    _check(_lib().dh2_tuning_set(byref(t)), "dh2_tuning_set")


def autotune(tree: Tree, G, eps: float = 1e-4, zeta: float = 2.0 / 3.0, err_mode: int = 0,
             mode: int | None = None, nearfield: int = 0, reps: int = 3, stream=None):
    """dh2_autotune on one problem: returns (installed table, timed candidates as
    [{"knob", "cls", "value", "ms"}])."""
    dt = _dtype_code(G)
    if mode is None:
        mode = MODE_FP32 if dt == DH2_C64 else MODE_FP64
    p = _params(eps, zeta, err_mode, mode, nearfield, 0)
    t = Tuning()
    cap = 64
    recs = (TuneRecord * cap)()
    nrec = c_int32(0)
    _check(_lib().dh2_autotune(tree.handle, c_void_p(G.data_ptr()), dt, _colmajor_ld(G), byref(p),
                               c_void_p(_stream_handle(stream)), int(reps), byref(t), ctypes.cast(recs, c_void_p),
                               cap, byref(nrec)), "dh2_autotune")
    log = [{"knob": TUNE_KNOBS[r.knob], "cls": int(r.cls), "value": int(r.value), "ms": float(r.ms)}
           for r in recs[:nrec.value]]
    return _tuning_dict(t), log


def dh2_compress_host(tree: Tree, G, eps: float = 1e-4, zeta: float = 2.0 / 3.0, err_mode: int = 0,
                      mode: int | None = None, max_sweeps: int = 0, stream=None) -> Matrix:
    """Compress a host matrix G (torch CPU tensor, column-major view, tree's permuted order;
    pinned memory for the full copy rate).  The library copies it to the device itself."""
    if G.device.type != "cpu":
        raise ValueError("G must be in host memory")
    dt = _dtype_code(G)
    if mode is None:
        mode = MODE_FP32 if dt == DH2_C64 else MODE_FP64
    ld = _colmajor_ld(G)
    p = _params(eps, zeta, err_mode, mode, 0, max_sweeps)
    h = c_void_p()
    _check(_lib().dh2_compress_host(tree.handle, c_void_p(G.data_ptr()), dt, ld, byref(p),
                                    c_void_p(_stream_handle(stream)), byref(h)), "dh2_compress_host")
    return Matrix(h.value, tree, mode, None)


def dh2_compress_batched(trees, Gs, eps: float = 1e-4, zeta: float = 2.0 / 3.0, err_mode: int = 0,
                         mode: int | None = None, nearfield: int = 0, max_sweeps: int = 0, stream=None) -> list:
    """Compress several independent device matrices (column-major views) in one schedule."""
    n = len(trees)
    if n != len(Gs) or n == 0:
        raise ValueError("need one matrix per tree")
    dt = _dtype_code(Gs[0])
    if any(_dtype_code(g) != dt for g in Gs):
        raise TypeError("all matrices must have the same dtype")
    if mode is None:
        mode = MODE_FP32 if dt == DH2_C64 else MODE_FP64
    th = (c_void_p * n)(*[t.handle for t in trees])
    gp = (c_void_p * n)(*[g.data_ptr() for g in Gs])
    lds = (c_int64 * n)(*[_colmajor_ld(g) for g in Gs])
    outs = (c_void_p * n)()
    p = _params(eps, zeta, err_mode, mode, nearfield, max_sweeps)
    _check(_lib().dh2_compress_batched(n, th, gp, lds, dt, byref(p), c_void_p(_stream_handle(stream)), outs),
           "dh2_compress_batched")
    return [Matrix(outs[i], trees[i], mode, Gs[i]) for i in range(n)]


class Plan:
    """Owner of a dh2_plan handle: the compression of one or several problems captured once into a CUDA
    graph (include/dh2.h, dh2_plan_create) and replayed by run() on new matrices of the same shapes."""

    def __init__(self, trees, Gs, eps: float = 1e-4, zeta: float = 2.0 / 3.0, err_mode: int = 0,
                 mode: int | None = None, nearfield: int = 0, max_sweeps: int = 0, stream=None):
        n = len(trees)
        if n != len(Gs) or n == 0:
            raise ValueError("need one matrix per tree")
        dt = _dtype_code(Gs[0])
        if any(_dtype_code(g) != dt for g in Gs):
            raise TypeError("all matrices must have the same dtype")
        if mode is None:
            mode = MODE_FP32 if dt == DH2_C64 else MODE_FP64
        self.handle = c_void_p()
        self.trees = list(trees)
        self.mode = mode
        self.lds = [_colmajor_ld(g) for g in Gs]
        self._dt = dt
        th = (c_void_p * n)(*[t.handle for t in trees])
        gp = (c_void_p * n)(*[g.data_ptr() for g in Gs])
        lds = (c_int64 * n)(*self.lds)
        p = _params(eps, zeta, err_mode, mode, nearfield, max_sweeps)
        h = c_void_p()
        _check(_lib().dh2_plan_create(n, th, gp, lds, dt, byref(p), c_void_p(_stream_handle(stream)), byref(h)),
               "dh2_plan_create")
        self.handle = h
        self._Gs = list(Gs)

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value:
            _lib().dh2_plan_free(self.handle)
            self.handle = c_void_p()

    def run(self, Gs=None, stream=None) -> None:
        """Replay the captured schedule on Gs (same dtypes, shapes and leading dimensions), or on the
        matrices of the previous run; stream-ordered, no host synchronisation."""
        if Gs is None:
            gp = None
        else:
            if len(Gs) != len(self.trees):
                raise ValueError("need one matrix per tree")
            for g, ld in zip(Gs, self.lds):
                if _dtype_code(g) != self._dt or _colmajor_ld(g) != ld:
                    raise ValueError("a plan runs on matrices of its own dtype and leading dimension")
            self._Gs = list(Gs)
            gp = (c_void_p * len(Gs))(*[g.data_ptr() for g in Gs])
        _check(_lib().dh2_plan_run(self.handle, gp, c_void_p(_stream_handle(stream))), "dh2_plan_run")

    def wait(self, stream=None) -> None:
        """Synchronise the stream and raise the last run's device status, if any."""
        _check(_lib().dh2_plan_wait(self.handle, c_void_p(_stream_handle(stream))), "dh2_plan_wait")

    def matrices(self) -> list:
        out = []
        for i, t in enumerate(self.trees):
            h = c_void_p()
            _check(_lib().dh2_plan_matrix(self.handle, i, byref(h)), "dh2_plan_matrix")
            out.append(Matrix(h.value, t, self.mode, self._Gs[i], owner=self))
        return out


def dh2_compress_kernel(tree: Tree, points: np.ndarray, kappa: float, diag: float, eps: float = 1e-4,
                        zeta: float = 2.0 / 3.0, err_mode: int = 0, mode: int = MODE_FP32, max_sweeps: int = 0,
                        stream=None) -> Matrix:
    """Matrix-free compression of the Helmholtz collocation matrix of `points` (caller order)."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    p = _params(eps, zeta, err_mode, mode, 0, max_sweeps)
    h = c_void_p()
    _check(_lib().dh2_compress_kernel(tree.handle, _ptr(pts), float(kappa), float(diag), byref(p),
                                      c_void_p(_stream_handle(stream)), byref(h)), "dh2_compress_kernel")
    return Matrix(h.value, tree, mode, None)


def dh2_compress_kernel_dlp(tree: Tree, points: np.ndarray, normals: np.ndarray, kappa: float, eps: float = 1e-4,
                            zeta: float = 2.0 / 3.0, err_mode: int = 0, mode: int = MODE_FP32, max_sweeps: int = 0,
                            stream=None) -> Matrix:
    """Matrix-free compression of 1/2 I + the double-layer collocation matrix of `points` with unit
    `normals` (both caller order)."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    nrm = np.ascontiguousarray(normals, dtype=np.float64)
    if nrm.shape != pts.shape:
        raise ValueError("normals must have the shape of points")
    p = _params(eps, zeta, err_mode, mode, 0, max_sweeps)
    h = c_void_p()
    _check(_lib().dh2_compress_kernel_dlp(tree.handle, _ptr(pts), _ptr(nrm), float(kappa), byref(p),
                                          c_void_p(_stream_handle(stream)), byref(h)), "dh2_compress_kernel_dlp")
    return Matrix(h.value, tree, mode, None)


def _matvec_operands(M: Matrix, x, y) -> int:
    """Check x and y against M before any C call (the kernels trust their sizes): CUDA tensors on the
    current device, the matrix's complex dtype, n rows, column-major (n,) or (n, nrhs) with the same
    shape.  Returns nrhs."""
    import torch

    want = torch.complex128 if M.mode == MODE_FP64 else torch.complex64
    dev = torch.cuda.current_device()
    for name, v in (("x", x), ("y", y)):
        if not isinstance(v, torch.Tensor) or v.device.type != "cuda" or v.device.index != dev:
            raise ValueError(f"{name} must be a CUDA tensor on the current device (cuda:{dev})")
        if v.dtype != want:
            raise TypeError(f"{name} must be {want} for this matrix, got {v.dtype}")
        if v.dim() not in (1, 2) or v.shape[0] != M.tree.n:
            raise ValueError(f"{name} must have {M.tree.n} rows")
        if v.dim() == 2 and (v.stride(0) != 1 or v.stride(1) != v.shape[0]):
            raise ValueError(f"{name} must be column-major (n, nrhs)")
        if v.dim() == 1 and v.stride(0) != 1:
            raise ValueError(f"{name} must be contiguous")
    if tuple(x.shape) != tuple(y.shape):
        raise ValueError("x and y must have the same shape")
    nrhs = 1 if x.dim() == 1 else x.shape[1]
    if nrhs < 1:
        raise ValueError("nrhs must be at least 1")
    return nrhs


def dh2_matvec(M: Matrix, x, y, stream=None) -> None:
    """y = G~ x; x, y torch device tensors (n,) or (n, nrhs) column-major, matrix dtype."""
    nrhs = _matvec_operands(M, x, y)
    _check(_lib().dh2_matvec(M.handle, c_void_p(x.data_ptr()), c_void_p(y.data_ptr()), nrhs,
                             c_void_p(_stream_handle(stream))), "dh2_matvec")


def dh2_matvec_noalloc(M: Matrix, x, y, stream=None) -> None:
    """y = G~ x without any device allocation (fixed 8 MiB library scratch array)."""
    nrhs = _matvec_operands(M, x, y)
    _check(_lib().dh2_matvec_noalloc(M.handle, c_void_p(x.data_ptr()), c_void_p(y.data_ptr()), nrhs,
                                     c_void_p(_stream_handle(stream))), "dh2_matvec_noalloc")


def dh2_debug_fail_alloc(nth: int) -> None:
    """Refuse the nth device allocation the library makes from now on (0 disarms); test instrumentation."""
    _check(_lib().dh2_debug_fail_alloc(int(nth)), "dh2_debug_fail_alloc")


ERR_FRO_BLOCKWISE = 0
ERR_FRO_CLOSED = 1
ERR_SPECTRAL = 2


def dh2_error(M: Matrix, Gref=None, stream=None, which: int = ERR_FRO_BLOCKWISE) -> float:
    """Relative error against Gref by `which` (ERR_FRO_BLOCKWISE |G - G~|_F/|G|_F, ERR_FRO_CLOSED its
    closed form from the block norms, ERR_SPECTRAL |G - G~|_2/|G|_2 by power iteration); Gref=None for a
    matrix-free compression (reference generated in FP64)."""
    out = c_double()
    if Gref is None:
        _check(_lib().dh2_error(M.handle, None, 0, 0, int(which), c_void_p(_stream_handle(stream)), byref(out)),
               "dh2_error")
    else:
        _check(_lib().dh2_error(M.handle, c_void_p(Gref.data_ptr()), _dtype_code(Gref), _colmajor_ld(Gref),
                                int(which), c_void_p(_stream_handle(stream)), byref(out)), "dh2_error")
    return float(out.value)


def dh2_matvec_adjoint(M: Matrix, x, y, stream=None) -> None:
    """y = G~^* x (adjoint product); operands as dh2_matvec."""
    nrhs = _matvec_operands(M, x, y)
    _check(_lib().dh2_matvec_adjoint(M.handle, c_void_p(x.data_ptr()), c_void_p(y.data_ptr()), nrhs,
                                     c_void_p(_stream_handle(stream))), "dh2_matvec_adjoint")


def dh2_version() -> str:
    return _lib().dh2_version().decode()


def exported_symbols() -> list:
    return [name for name, _, _ in SIGNATURES]
