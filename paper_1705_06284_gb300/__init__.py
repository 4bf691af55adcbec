"""GB300-native FFT polyspectrum estimator (arXiv 1705.06284).

A thin ctypes binding over the C ABI in ``include/fbs.h`` (argument
marshalling only: every step of the estimator runs in the hand-written
sm_103a kernels of ``libfbs.so``).  The functions below carry the C names;
:class:`Plan` is a small convenience wrapper over them.

PyTorch is used only for device memory and streams: pass CUDA float32
tensors to keep everything on the device, or NumPy arrays to let the
library stage host buffers.

There is no CPU fallback.  Loading fails loudly if ``libfbs.so`` has not
been built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from ._build import LIB as _LIB_PATH

__all__ = [
    "FBS_PREC_FP32", "FBS_PREC_BF16X3", "FBS_PREC_BF16",
    "FBS_FLAG_TRISPECTRUM", "FBS_FLAG_ALLOW_ALIASED", "FBS_FLAG_TIMING",
    "FbsError", "Plan", "lib", "kernel_class_names",
    "fbs_plan_create", "fbs_plan_free", "fbs_bispectrum", "fbs_trispectrum",
]

FBS_PREC_FP32 = 0
FBS_PREC_BF16X3 = 1
FBS_PREC_BF16 = 2
FBS_FLAG_TRISPECTRUM = 1
FBS_FLAG_ALLOW_ALIASED = 2
FBS_FLAG_TIMING = 4
FBS_FLAG_FULL_GRID = 8
FBS_FLAG_SINGLE_GRID = 16
FBS_OPT_TC_WIDE = 1
FBS_OPT_TC_ROLES = 2
FBS_OPT_TC_CHUNK = 3
FBS_OPT_TC_PAIRS = 4
FBS_OPT_TC_WAIT_LIMIT = 5
FBS_OPT_SLAB_PLANES = 6
FBS_OPT_TC_MERGE = 7
FBS_OPT_TC_BSTAGES = 8
FBS_OPT_TC_BFROMA = 9
FBS_OPT_TC_STACK = 10

_PREC = {"fp32": FBS_PREC_FP32, "bf16x3": FBS_PREC_BF16X3, "bf16": FBS_PREC_BF16}

_STATUS = {0: "FBS_OK", -1: "FBS_ERR_ARG", -2: "FBS_ERR_UNSUPPORTED_N", -3: "FBS_ERR_OOM",
           -4: "FBS_ERR_CUDA", -5: "FBS_ERR_TIMEOUT", -6: "FBS_ERR_STATE", -7: "FBS_ERR_NUMERIC"}


class FbsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (_STATUS.get(status, "?"), status, msg))
        self.status = status


_lib = None

# (name, restype, argtypes) of every entry point declared in include/fbs.h
_vp = ctypes.c_void_p
_SIGS = [
    ("fbs_plan_create", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                       ctypes.c_uint, _vp]),
    ("fbs_plan_free", None, [_vp]),
    ("fbs_plan_export_counts", ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_int64)]),
    ("fbs_plan_create_from_counts", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_double,
                                                   ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_uint, _vp, _vp, ctypes.c_int64]),
    ("fbs_plan_num_triplets", ctypes.c_int, [_vp]),
    ("fbs_plan_num_quads", ctypes.c_int, [_vp]),
    ("fbs_plan_triplets", ctypes.c_int, [_vp, _vp, _vp]),
    ("fbs_plan_quads", ctypes.c_int, [_vp, _vp, _vp]),
    ("fbs_plan_shells", ctypes.c_int, [_vp, _vp, _vp]),
    ("fbs_plan_set_precision", ctypes.c_int, [_vp, ctypes.c_int]),
    ("fbs_plan_set_stream", ctypes.c_int, [_vp, _vp]),
    ("fbs_plan_set_option", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    ("fbs_bispectrum", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("fbs_trispectrum", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    ("fbs_plan_sums", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("fbs_trispectrum_connected", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("fbs_plan_set_diagonal", ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    ("fbs_plan_follow", ctypes.c_int, [_vp, _vp]),
    ("fbs_plan_tc_info", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp]),
    ("fbs_plan_num_diagonal_bins", ctypes.c_int, [_vp]),
    ("fbs_plan_diagonal_counts", ctypes.c_int, [_vp, _vp, _vp]),
    ("fbs_trispectrum_diagonal", ctypes.c_int, [_vp, _vp, _vp]),
    ("fbs_bispectrum_batch", ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp]),
    ("fbs_plan_quads_connected", ctypes.c_int, [_vp, _vp]),
    ("fbs_plan_shell_average", ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp]),
    ("fbs_plan_triangle_average", ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int64, _vp, _vp,
                                                  ctypes.c_int, _vp]),
    ("fbs_num_kernel_classes", ctypes.c_int, []),
    ("fbs_kernel_class_name", ctypes.c_char_p, [ctypes.c_int]),
    ("fbs_plan_kernel_times", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
    ("fbs_plan_create_ms", ctypes.c_double, [_vp]),
    ("fbs_plan_device_bytes", ctypes.c_int64, [_vp]),
    ("fbs_plan_count_margin", ctypes.c_double, [_vp]),
    ("fbs_plan_quad_counts_exact", ctypes.c_int, [_vp]),
    ("fbs_plan_quad_counts_u128", ctypes.c_int, [_vp, _vp]),
    ("fbs_plan_eval_grid", ctypes.c_int, [_vp]),
    ("fbs_plan_slab_planes", ctypes.c_int, [_vp]),
    ("fbs_plan_num_slabs", ctypes.c_int, [_vp]),
    ("fbs_plan_num_levels", ctypes.c_int, [_vp]),
    ("fbs_plan_level", ctypes.c_int, [_vp, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 6),
    ("fbs_plan_item_levels", ctypes.c_int, [_vp, _vp, _vp]),
    ("fbs_plan_check", ctypes.c_int, [_vp]),
    ("fbs_rebin_create", ctypes.c_int, [ctypes.POINTER(_vp), _vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int]),
    ("fbs_rebin_bispectrum", ctypes.c_int, [_vp, _vp, _vp]),
    ("fbs_rebin_counts", ctypes.c_int, [_vp, _vp]),
    ("fbs_rebin_free", None, [_vp]),
    ("fbs_gplan_create", ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_uint32]),
    ("fbs_gplan_num_triplets", ctypes.c_int, [_vp]),
    ("fbs_gplan_triplets", ctypes.c_int, [_vp, _vp, _vp]),
    ("fbs_gplan_shells", ctypes.c_int, [_vp, _vp]),
    ("fbs_gplan_bispectrum", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("fbs_gplan_free", None, [_vp]),
    ("fbs_set_device_budget", ctypes.c_int, [ctypes.c_int64]),
    ("fbs_set_slab_budget", ctypes.c_int, [ctypes.c_int64]),
    ("fbs_device_bytes_in_use", ctypes.c_int64, []),
    ("fbs_triple_sums_noalloc", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong,
                                                _vp, ctypes.c_int, _vp, _vp]),
    ("fbs_last_error", ctypes.c_char_p, []),
    ("fbs_version", ctypes.c_int, []),
]


def lib():
    """Load ``libfbs.so`` (built in-tree).  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libfbs.so is not built (%s); run __graft_entry__.build()" % _LIB_PATH)
        L = ctypes.CDLL(_LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        msg = lib().fbs_last_error().decode(errors="replace")
        raise FbsError(status, msg)


def kernel_class_names():
    L = lib()
    return [L.fbs_kernel_class_name(i).decode() for i in range(L.fbs_num_kernel_classes())]


# ---------------------------------------------------------------- C-named calls
def fbs_plan_create(N, L, edges, precision=FBS_PREC_FP32, flags=0, stream=None, counts=None):
    """Returns an opaque plan handle (int).  ``counts``: bytes from
    fbs_plan_export_counts of an equal plan (skips the plan-time count pass)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    h = _vp()
    ep = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if counts is None:
        _check(lib().fbs_plan_create(ctypes.byref(h), int(N), float(L), ep, len(e) - 1,
                                     int(precision), int(flags), _vp(stream or 0)))
    else:
        buf = ctypes.create_string_buffer(bytes(counts), len(counts))
        _check(lib().fbs_plan_create_from_counts(ctypes.byref(h), int(N), float(L), ep, len(e) - 1,
                                                 int(precision), int(flags), _vp(stream or 0),
                                                 ctypes.cast(buf, _vp), len(counts)))
    return h.value


def fbs_plan_export_counts(h):
    """The plan's closed items and exact counts, serialised (bytes)."""
    n = ctypes.c_int64(0)
    _check(lib().fbs_plan_export_counts(_vp(h), None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().fbs_plan_export_counts(_vp(h), ctypes.cast(buf, _vp), ctypes.byref(n)))
    return buf.raw[:n.value]


def fbs_plan_free(h):
    lib().fbs_plan_free(_vp(h))


def fbs_bispectrum(h, field_ptr, B_ptr, P_ptr):
    _check(lib().fbs_bispectrum(_vp(h), _vp(field_ptr), _vp(B_ptr or 0), _vp(P_ptr or 0)))


def fbs_trispectrum(h, field_ptr, T_ptr, B_ptr, P_ptr):
    _check(lib().fbs_trispectrum(_vp(h), _vp(field_ptr), _vp(T_ptr or 0), _vp(B_ptr or 0),
                                 _vp(P_ptr or 0)))


def fbs_plan_check(h):
    """Wait for the plan's stream; raise FbsError(FBS_ERR_TIMEOUT) if an
    evaluation since the last report gave up a tensor-core wait."""
    _check(lib().fbs_plan_check(_vp(h)))


def fbs_set_device_budget(nbytes):
    """Process-wide cap on the device bytes all plans may hold (0: none)."""
    _check(lib().fbs_set_device_budget(int(nbytes)))


def fbs_set_slab_budget(nbytes):
    """Process-wide default slab buffer of plans created afterwards (0: 8 GiB)."""
    _check(lib().fbs_set_slab_budget(int(nbytes)))


def fbs_device_bytes_in_use():
    return int(lib().fbs_device_bytes_in_use())


def fbs_triple_sums_noalloc(fields_ptr, nfields, bin_stride, npts, abc_ptr, ntrip, num_ptr, stream=None):
    """sum_p f_a f_b f_c per triplet with no device allocation (see fbs.h)."""
    _check(lib().fbs_triple_sums_noalloc(_vp(fields_ptr), int(nfields), int(bin_stride), int(npts),
                                         _vp(abc_ptr), int(ntrip), _vp(num_ptr), _vp(stream or 0)))


# ---------------------------------------------------------------- convenience
def _ptr(a):
    """(pointer, keepalive) for a torch tensor or NumPy array (NULL for None)."""
    if a is None:
        return 0, None
    if isinstance(a, np.ndarray):
        return a.ctypes.data, a
    return a.data_ptr(), a


class Plan:
    """Plan for N^3 fields in a box of side L with the given bin edges.

    ``precision``: "fp32" | "bf16x3" | "bf16".  ``stream``: a torch CUDA
    stream (default: torch's current stream, or the legacy default stream
    without torch).
    """

    def __init__(self, N, L, edges, precision="fp32", trispectrum=False, allow_aliased=False,
                 timing=False, stream=None, full_grid=False, single_grid=False, counts=None):
        flags = (FBS_FLAG_TRISPECTRUM if trispectrum else 0) | \
                (FBS_FLAG_ALLOW_ALIASED if allow_aliased else 0) | (FBS_FLAG_TIMING if timing else 0) | \
                (FBS_FLAG_FULL_GRID if full_grid else 0) | (FBS_FLAG_SINGLE_GRID if single_grid else 0)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream()
            except Exception:
                stream = None
        sp = getattr(stream, "cuda_stream", stream) if stream is not None else 0
        self.N, self.L = int(N), float(L)
        self.edges = np.ascontiguousarray(edges, dtype=np.float64)
        self.nbins = len(self.edges) - 1
        self._h = fbs_plan_create(N, L, self.edges, _PREC[precision], flags, sp, counts=counts)
        self.precision = precision
        Lb = lib()
        self.ntrip = Lb.fbs_plan_num_triplets(_vp(self._h))
        self.nquad = Lb.fbs_plan_num_quads(_vp(self._h))
        self.triplets = np.zeros((self.ntrip, 3), dtype=np.int32)
        self.N_tri = np.zeros(self.ntrip, dtype=np.int64)
        _check(Lb.fbs_plan_triplets(_vp(self._h), self.triplets.ctypes.data, self.N_tri.ctypes.data))
        self.quads = np.zeros((self.nquad, 4), dtype=np.int32)
        self.N_quad = np.zeros(self.nquad, dtype=np.float64)
        _check(Lb.fbs_plan_quads(_vp(self._h), self.quads.ctypes.data, self.N_quad.ctypes.data))
        self.shell = np.zeros(self.nbins, dtype=np.int64)
        self.thresholds = np.zeros(self.nbins + 1, dtype=np.int64)
        _check(Lb.fbs_plan_shells(_vp(self._h), self.shell.ctypes.data, self.thresholds.ctypes.data))
        self.create_ms = Lb.fbs_plan_create_ms(_vp(self._h))
        self.device_bytes = int(Lb.fbs_plan_device_bytes(_vp(self._h)))
        self.count_margin = float(Lb.fbs_plan_count_margin(_vp(self._h)))
        self.quad_counts_exact = bool(Lb.fbs_plan_quad_counts_exact(_vp(self._h)) == 1)
        w = np.zeros(2 * max(self.nquad, 1), dtype=np.uint64)
        _check(Lb.fbs_plan_quad_counts_u128(_vp(self._h), w.ctypes.data))
        # exact ordered quadruple counts as Python integers (past 2^63 for wide shells)
        self.N_quad_exact = [int(w[2 * i]) | (int(w[2 * i + 1]) << 64) for i in range(self.nquad)]
        self.eval_grid = int(Lb.fbs_plan_eval_grid(_vp(self._h)))
        self.slab_planes = int(Lb.fbs_plan_slab_planes(_vp(self._h)))
        self.num_slabs = int(Lb.fbs_plan_num_slabs(_vp(self._h)))
        self.levels = []
        for i in range(Lb.fbs_plan_num_levels(_vp(self._h))):
            v = [ctypes.c_int() for _ in range(6)]
            _check(Lb.fbs_plan_level(_vp(self._h), i, *[ctypes.byref(x) for x in v]))
            self.levels.append(dict(zip(("M", "nbins", "ntrip", "nquad", "slab_planes", "nslabs"),
                                        (x.value for x in v))))
        self.N_conn = np.zeros(self.nquad, dtype=np.float64)
        _check(Lb.fbs_plan_quads_connected(_vp(self._h), self.N_conn.ctypes.data))
        self.trip_level = np.zeros(self.ntrip, dtype=np.int32)
        self.quad_level = np.zeros(self.nquad, dtype=np.int32)
        _check(Lb.fbs_plan_item_levels(_vp(self._h), self.trip_level.ctypes.data, self.quad_level.ctypes.data))

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            fbs_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_precision(self, precision):
        _check(lib().fbs_plan_set_precision(_vp(self._h), _PREC[precision]))
        self.precision = precision

    def set_option(self, option, value):
        _check(lib().fbs_plan_set_option(_vp(self._h), int(option), int(value)))

    def set_tc_wide(self, wide: bool):
        """Tensor-core orientation: False = pair products as operand A
        (default), True = the wide orientation (see FBS_OPT_TC_WIDE)."""
        self.set_option(FBS_OPT_TC_WIDE, 1 if wide else 0)

    def set_stream(self, stream):
        sp = getattr(stream, "cuda_stream", stream) or 0
        _check(lib().fbs_plan_set_stream(_vp(self._h), _vp(sp)))

    # -- estimators
    def _outputs(self, like, n):
        if isinstance(like, np.ndarray):
            return np.empty(n, dtype=np.float64)
        import torch
        dev = like.device if like is not None else torch.device("cuda", torch.cuda.current_device())
        return torch.empty(n, dtype=torch.float64, device=dev)

    def tc_info(self):
        """Tensor-core job shapes per level (after an evaluation): a list of
        {job: dict(tiles, inner, Npad, merged, ka, stages)} for the built jobs
        (stages: operand-A, operand-B and field pipeline depths; b_from_a:
        the inner pair rows stored by the operand-A warps)."""
        out = []
        for lvl in range(len(self.levels)):
            d = {}
            for which, name in enumerate(("triplets", "quadruplets", "fused")):
                a = (ctypes.c_int32 * 11)()
                _check(lib().fbs_plan_tc_info(_vp(self._h), lvl, which, ctypes.cast(a, _vp)))
                if a[0] and a[1]:
                    d[name] = {"tiles": a[2], "inner": a[3], "Npad": a[4], "merged": a[5], "ka": a[6],
                               "stages": [a[7], a[8], a[9]], "b_from_a": a[10]}
            out.append(d)
        return out

    def follow(self, leader):
        """Evaluate ``leader``'s spectrum (its last evaluation on the shared
        stream) instead of a field of this plan's own: pass ``None`` as the
        field afterwards (see fbs_plan_follow).  ``leader=None`` detaches."""
        _check(lib().fbs_plan_follow(_vp(self._h), _vp(leader._h if leader is not None else 0)))
        self.leader = leader

    def bispectrum(self, field, B=None, P=None):
        """B[ntrip], P[nbins] for an N^3 float32 field (torch CUDA tensor or
        NumPy array; None for a following plan).  Outputs live where the
        field lives unless given (on the current CUDA device for None)."""
        self._check_field(field)
        B = self._outputs(field, self.ntrip) if B is None else B
        P = self._outputs(field, self.nbins) if P is None else P
        fp, _k0 = _ptr(field)
        bp, _k1 = _ptr(B)
        pp, _k2 = _ptr(P)
        fbs_bispectrum(self._h, fp, bp, pp)
        return B, P

    def trispectrum(self, field, T=None, B=None, P=None):
        self._check_field(field)
        T = self._outputs(field, self.nquad) if T is None else T
        B = self._outputs(field, self.ntrip) if B is None else B
        P = self._outputs(field, self.nbins) if P is None else P
        fp, _k0 = _ptr(field)
        tp, _k1 = _ptr(T)
        bp, _k2 = _ptr(B)
        pp, _k3 = _ptr(P)
        fbs_trispectrum(self._h, fp, tp, bp, pp)
        return T, B, P

    def bispectrum_batch(self, fields, B=None, P=None):
        """B[nf, ntrip], P[nf, nbins] of a list of N^3 float32 CUDA tensors in
        one set of launches (see fbs_bispectrum_batch)."""
        import torch
        nf = len(fields)
        for f in fields:
            self._check_field(f)
        dev = fields[0].device
        B = torch.empty((nf, self.ntrip), dtype=torch.float64, device=dev) if B is None else B
        P = torch.empty((nf, self.nbins), dtype=torch.float64, device=dev) if P is None else P
        ptrs = (ctypes.c_void_p * nf)(*[f.data_ptr() for f in fields])
        _check(lib().fbs_bispectrum_batch(_vp(self._h), ctypes.cast(ptrs, _vp), nf, _vp(B.data_ptr()),
                                          _vp(P.data_ptr())))
        return B, P

    def triangle_average(self, tables, terms, coef):
        """Average of sum_k coef[k] f_i(|m1|) f_j(|m2|) f_l(|m3|) over each closed
        triplet's ordered triangles (see fbs_plan_triangle_average).
        tables: (nfunc, nw) FP64 values at integer |m|^2; terms: (nterms, 3)."""
        w = np.ascontiguousarray(tables, dtype=np.float64)
        t = np.ascontiguousarray(terms, dtype=np.int32).reshape(-1, 3)
        c = np.ascontiguousarray(coef, dtype=np.float64).ravel()
        out = np.zeros(self.ntrip)
        _check(lib().fbs_plan_triangle_average(_vp(self._h), w.ctypes.data, w.shape[0], w.shape[1], t.ctypes.data,
                                               c.ctypes.data, len(c), out.ctypes.data))
        return out

    def shell_average(self, table):
        """Average of table[|m|^2] over the modes of each bin (NaN if empty)."""
        w = np.ascontiguousarray(table, dtype=np.float64)
        out = np.zeros(self.nbins)
        _check(lib().fbs_plan_shell_average(_vp(self._h), w.ctypes.data, len(w), out.ctypes.data))
        return out

    def trispectrum_connected(self, field, Tc=None, T=None, B=None, P=None):
        """(Tc, T, B, P): the connected trispectrum (paired quadruples left
        out) with the raw T, B and P of the same evaluation."""
        self._check_field(field)
        Tc = self._outputs(field, self.nquad) if Tc is None else Tc
        T = self._outputs(field, self.nquad) if T is None else T
        B = self._outputs(field, self.ntrip) if B is None else B
        P = self._outputs(field, self.nbins) if P is None else P
        ptrs = [_ptr(x) for x in (field, Tc, T, B, P)]
        _check(lib().fbs_trispectrum_connected(_vp(self._h), *[_vp(p) for p, _ in ptrs]))
        return Tc, T, B, P

    def set_diagonal(self, diag_edges):
        """Diagonal bins of the quadrilateral diagonal |k1 + k2| (see
        fbs_plan_set_diagonal); sets ``N_D`` (nquad, ndiag) FP64 and
        ``N_D_exact`` (Python integers) from the exact plan-time counts."""
        e = np.ascontiguousarray(diag_edges, dtype=np.float64)
        nd = len(e) - 1
        _check(lib().fbs_plan_set_diagonal(_vp(self._h), e.ctypes.data, nd))
        self.ndiag = nd
        self.N_D = np.zeros((self.nquad, nd), dtype=np.float64)
        w = np.zeros(2 * max(1, self.nquad * nd), dtype=np.uint64)
        _check(lib().fbs_plan_diagonal_counts(_vp(self._h), self.N_D.ctypes.data, w.ctypes.data))
        self.N_D_exact = [[int(w[2 * (q * nd + d)]) | (int(w[2 * (q * nd + d) + 1]) << 64) for d in range(nd)]
                          for q in range(self.nquad)]

    def trispectrum_diagonal(self, field, TD=None):
        """TD (nquad, ndiag): the trispectrum of every closed quadruplet split
        by the diagonal bin of k1 + k2 (see fbs_trispectrum_diagonal)."""
        self._check_field(field)
        n = self.nquad * getattr(self, "ndiag", 0)
        TD = self._outputs(field, n) if TD is None else TD
        ptrs = [_ptr(x) for x in (field, TD)]
        _check(lib().fbs_trispectrum_diagonal(_vp(self._h), *[_vp(p) for p, _ in ptrs]))
        return TD.reshape(self.nquad, -1) if n else TD

    def _check_field(self, f):
        if f is None:
            if getattr(self, "leader", None) is None:
                raise ValueError("field is None but the plan follows no other plan")
            return
        n = self.N
        if tuple(f.shape) != (n, n, n):
            raise ValueError("field must have shape (%d, %d, %d)" % (n, n, n))
        if isinstance(f, np.ndarray):
            if f.dtype != np.float32 or not f.flags["C_CONTIGUOUS"]:
                raise ValueError("field must be C-contiguous float32")
        else:
            import torch
            if f.dtype != torch.float32 or not f.is_contiguous():
                raise ValueError("field must be a contiguous float32 tensor")

    def export_counts(self):
        """Serialised closed items and exact counts (see fbs_plan_export_counts)."""
        return fbs_plan_export_counts(self._h)

    def check(self):
        """Wait for the plan's stream; raise on a timed-out evaluation."""
        fbs_plan_check(self._h)

    def sums(self):
        """Raw FP64 sums of the last call: (num_trip, num_quad, sumsq)."""
        a = np.zeros(self.ntrip)
        q = np.zeros(self.nquad)
        s = np.zeros(self.nbins)
        _check(lib().fbs_plan_sums(_vp(self._h), a.ctypes.data, q.ctypes.data, s.ctypes.data))
        return a, q, s

    def kernel_times(self, reset=False):
        """{class: (ms, launches)} accumulated with timing=True."""
        n = lib().fbs_num_kernel_classes()
        ms = np.zeros(n)
        cnt = np.zeros(n, dtype=np.int64)
        _check(lib().fbs_plan_kernel_times(_vp(self._h), ms.ctypes.data, cnt.ctypes.data,
                                           1 if reset else 0))
        return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(kernel_class_names())}


class GeneralPlan:
    """Bispectrum and power spectrum on a non-cubic grid of a real or complex
    field (fbs_gplan_*): shape (N_x, N_y, N_z), box (L_x, L_y, L_z), edges in
    physical k.  ``bispectrum`` returns complex B[ntrip] and P[nbins]."""

    def __init__(self, shape, Ls, edges, allow_aliased=False):
        e = np.ascontiguousarray(edges, dtype=np.float64)
        self.shape = tuple(int(v) for v in shape)
        self.Ls = tuple(float(v) for v in Ls)
        self.nbins = len(e) - 1
        n = (ctypes.c_int32 * 3)(*self.shape)
        L = (ctypes.c_double * 3)(*self.Ls)
        h = ctypes.c_void_p()
        Lb = lib()
        _check(Lb.fbs_gplan_create(ctypes.byref(h), ctypes.cast(n, _vp), ctypes.cast(L, _vp), e.ctypes.data,
                                   self.nbins, FBS_FLAG_ALLOW_ALIASED if allow_aliased else 0))
        self._h = h = h.value
        self.ntrip = int(Lb.fbs_gplan_num_triplets(_vp(h)))
        self.triplets = np.zeros((self.ntrip, 3), dtype=np.int32)
        self.N_tri = np.zeros(self.ntrip, dtype=np.int64)
        _check(Lb.fbs_gplan_triplets(_vp(h), self.triplets.ctypes.data, self.N_tri.ctypes.data))
        self.shell = np.zeros(self.nbins, dtype=np.int64)
        _check(Lb.fbs_gplan_shells(_vp(h), self.shell.ctypes.data))

    def bispectrum(self, field):
        """field: NumPy array (real or complex) or a CUDA tensor (real or
        complex) of the plan's shape; returns (B, P) as complex128 NumPy arrays."""
        if tuple(field.shape) != self.shape:
            raise ValueError("field must have shape %s" % (self.shape,))
        if isinstance(field, np.ndarray):
            buf = np.ascontiguousarray(field, dtype=np.complex64)
            fp = buf.ctypes.data
        else:
            import torch
            buf = field.to(torch.complex64).contiguous()
            fp = buf.data_ptr()
        B = np.zeros(2 * max(1, self.ntrip))
        P = np.zeros(2 * self.nbins)
        _check(lib().fbs_gplan_bispectrum(_vp(self._h), _vp(fp), B.ctypes.data, P.ctypes.data))
        return B[: 2 * self.ntrip].view(np.complex128), P.view(np.complex128)

    def close(self):
        if getattr(self, "_h", None):
            lib().fbs_gplan_free(_vp(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Rebin:
    """Cells (k1 bin, k2 bin, cos theta bin) over a fine-bin plan's triplets
    (see fbs_rebin_create).  ``k_rep``: the k of each fine bin (default: the
    midpoint of its edges)."""

    def __init__(self, plan, k_edges, mu_edges, k_rep=None):
        ke = np.ascontiguousarray(k_edges, dtype=np.float64)
        me = np.ascontiguousarray(mu_edges, dtype=np.float64)
        kr = None if k_rep is None else np.ascontiguousarray(k_rep, dtype=np.float64)
        self.nk, self.nmu = len(ke) - 1, len(me) - 1
        self.plan = plan
        h = _vp()
        _check(lib().fbs_rebin_create(ctypes.byref(h), _vp(plan.handle), _vp(kr.ctypes.data if kr is not None else 0),
                                      _vp(ke.ctypes.data), self.nk, _vp(me.ctypes.data), self.nmu))
        self._h = h.value
        self.counts = np.zeros(self.nk * self.nk * self.nmu, dtype=np.int64)
        _check(lib().fbs_rebin_counts(_vp(self._h), self.counts.ctypes.data))
        self.counts = self.counts.reshape(self.nk, self.nk, self.nmu)

    def bispectrum(self, out=None):
        """B of every cell from the plan's last evaluation, shape (nk, nk, nmu)."""
        if out is None:
            out = np.empty(self.nk * self.nk * self.nmu)
        p, _k = _ptr(out)
        _check(lib().fbs_rebin_bispectrum(_vp(self._h), _vp(self.plan.handle), _vp(p)))
        return out.reshape(self.nk, self.nk, self.nmu)

    def close(self):
        if getattr(self, "_h", None):
            lib().fbs_rebin_free(_vp(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
