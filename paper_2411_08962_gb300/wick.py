"""Thin ctypes binding of libwick (include/wick.h): argument marshalling only.

The function names mirror the C ABI.  Device buffers are passed as torch CUDA
tensors (or raw integer device pointers); operator tables as the dataclasses
of `operators`.  Every computation runs in the CUDA library; if libwick.so is
missing this module raises on first use -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import operators as _ops

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwick.so")

WICK_OK, WICK_EINVAL, WICK_ENOMEM, WICK_ECUDA = 0, -1, -2, -3
WICK_ECAPACITY, WICK_EOVERFLOW, WICK_ETIMEOUT, WICK_EIO, WICK_ESCRATCH = -4, -5, -6, -7, -8
WICK_C128, WICK_C64 = 0, 1
WICK_FP64, WICK_MIXED, WICK_MIXED_SIMT = 0, 1, 2
WICK_UPLOAD_AUTO, WICK_UPLOAD_DMA, WICK_UPLOAD_KERNEL = 0, 1, 2
WICK_U, WICK_D = 0, 1

EXPORTS = ("wick_block_count", "wick_build_blocks", "wick_upload_rows", "wick_reduce_terms", "wick_terms_count",
           "wick_terms_nucleons", "wick_terms_block_count", "wick_terms_copy", "wick_terms_stats", "wick_terms_select",
           "wick_terms_magnitudes", "wick_terms_top", "wick_terms_save", "wick_terms_load", "wick_terms_free", "wick_contract", "wick_contract_noalloc",
           "wick_status", "wick_batch_create", "wick_batch_run", "wick_batch_launches", "wick_batch_free",
           "wick_synth_propagator", "wick_cluster_product", "wick_det_reduce", "wick_det_reduce_matrix", "wick_det_stats",
           "wick_det_element_offsets", "wick_det_copy", "wick_det_contract", "wick_det_contract_3pt", "wick_det_free", "wick_set_tuning", "wick_get_tuning",
           "wick_build_blocks_3pt", "wick_contract_3pt", "wick_reduce_terms_matrix", "wick_terms_elements",
           "wick_terms_copy_matrix", "wick_inject_alloc_failure", "wick_selftest_wait", "wick_strerror",
           "wick_version")


class WickError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class wick_prop(C.Structure):
    _fields_ = [("data", C.c_void_p), ("L", C.c_int), ("T", C.c_int), ("n_src", C.c_int), ("dtype", C.c_int)]


class wick_nucleon_op(C.Structure):
    _fields_ = [("n_entries", C.c_int), ("entries", C.POINTER(C.c_int8)), ("w", C.POINTER(C.c_int32)),
                ("flav_pair", C.c_int)]


class wick_block_layout(C.Structure):
    _fields_ = [("n_ops", C.c_int), ("n_spin", C.c_int), ("n_chi", C.c_int), ("chi", C.c_int8 * 12)]


class wick_nucleus(C.Structure):
    _fields_ = [("A", C.c_int), ("n_sink", C.c_int), ("sink_type", C.POINTER(C.c_int8)),
                ("sink_spin", C.POINTER(C.c_int8)), ("sink_w", C.POINTER(C.c_int64)), ("n_src", C.c_int),
                ("src_chi", C.POINTER(C.c_int8)), ("src_w", C.POINTER(C.c_int64)),
                ("src_flav", C.POINTER(C.c_int8)), ("scale", C.c_double)]


class wick_tuning(C.Structure):
    _fields_ = [("range_sites", C.c_int), ("contract_threads", C.c_int), ("contract_ctas_per_sm", C.c_int),
                ("contract_chunk_terms", C.c_int), ("hash_log2_start", C.c_int), ("hash_log2_max", C.c_int),
                ("no_pair_kernel", C.c_int)]


class wick_quark_operator(C.Structure):
    _fields_ = [("n_u", C.c_int), ("n_d", C.c_int), ("n_terms", C.c_int), ("chi", C.POINTER(C.c_int8)),
                ("w", C.POINTER(C.c_int64))]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libwick.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libwick.so not found at {path}: run paper_2411_08962_gb300.build")
            L = C.CDLL(path)
            vp, P = C.c_void_p, C.POINTER
            L.wick_block_count.argtypes = [P(wick_block_layout)]
            L.wick_block_count.restype = C.c_size_t
            L.wick_build_blocks.argtypes = [P(wick_prop), P(wick_prop), P(wick_nucleon_op), P(wick_block_layout),
                                            C.c_int, vp, vp]
            L.wick_upload_rows.argtypes = [P(wick_prop), P(wick_prop), P(wick_prop), P(wick_prop),
                                           P(wick_nucleon_op), P(wick_block_layout), C.c_int, P(C.c_size_t), vp]
            L.wick_reduce_terms.argtypes = [P(wick_nucleus), P(wick_nucleon_op), P(wick_block_layout), C.c_uint64,
                                            C.c_int, C.c_int, P(vp), vp]
            L.wick_terms_count.argtypes = [vp]
            L.wick_terms_count.restype = C.c_int64
            L.wick_terms_nucleons.argtypes = [vp]
            L.wick_terms_block_count.argtypes = [vp]
            L.wick_terms_block_count.restype = C.c_int64
            L.wick_terms_copy.argtypes = [vp, vp, vp, vp]
            L.wick_terms_stats.argtypes = [vp, P(C.c_int64), P(C.c_double)]
            L.wick_terms_select.argtypes = [vp, P(C.c_int64), C.c_int64]
            L.wick_terms_magnitudes.argtypes = [vp, C.c_int, vp, P(C.c_double), vp]
            L.wick_terms_top.argtypes = [vp, P(C.c_double), C.c_double]
            L.wick_terms_save.argtypes = [vp, C.c_char_p]
            L.wick_terms_load.argtypes = [C.c_char_p, P(vp)]
            L.wick_terms_free.argtypes = [vp]
            L.wick_terms_free.restype = None
            L.wick_contract.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, vp, vp]
            L.wick_contract_noalloc.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, vp, vp]
            L.wick_status.argtypes = [vp]
            L.wick_batch_create.argtypes = [P(wick_prop), P(wick_prop), C.c_int, P(wick_nucleon_op),
                                            P(wick_block_layout), P(vp), C.c_int, C.c_int, vp, vp, P(vp)]
            L.wick_batch_run.argtypes = [vp, vp]
            L.wick_batch_launches.argtypes = [vp]
            L.wick_batch_free.argtypes = [vp]
            L.wick_batch_free.restype = None
            L.wick_synth_propagator.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp]
            L.wick_cluster_product.argtypes = [vp, vp, C.c_int64, vp, vp]
            L.wick_det_reduce.argtypes = [P(wick_quark_operator), P(wick_quark_operator), C.c_uint64, C.c_int, P(vp)]
            L.wick_det_reduce_matrix.argtypes = [P(wick_quark_operator), C.c_int, C.c_uint64, C.c_int, P(vp)]
            L.wick_det_stats.argtypes = [vp, P(C.c_int64)]
            L.wick_det_element_offsets.argtypes = [vp, P(C.c_int64)]
            L.wick_det_copy.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
            L.wick_det_contract.argtypes = [P(wick_prop), P(wick_prop), vp, C.c_double, C.c_int, vp, vp]
            L.wick_det_contract_3pt.argtypes = [P(wick_prop), P(wick_prop), P(wick_prop), C.c_int, vp, C.c_double,
                                                C.c_int, vp, vp]
            L.wick_det_free.argtypes = [vp]
            L.wick_det_free.restype = None
            L.wick_build_blocks_3pt.argtypes = [P(wick_prop), P(wick_prop), P(wick_prop), C.c_int, P(wick_nucleon_op),
                                                P(wick_block_layout), C.c_int, vp, vp]
            L.wick_contract_3pt.argtypes = [vp, vp, C.c_int, C.c_int, vp, C.c_int, vp, vp]
            L.wick_reduce_terms_matrix.argtypes = [P(wick_nucleus), C.c_int, P(wick_nucleon_op), P(wick_block_layout),
                                                   C.c_uint64, C.c_int, C.c_int, P(vp), vp]
            L.wick_terms_elements.argtypes = [vp]
            L.wick_terms_copy_matrix.argtypes = [vp, vp, vp, vp]
            L.wick_set_tuning.argtypes = [P(wick_tuning)]
            L.wick_get_tuning.argtypes = [P(wick_tuning)]
            L.wick_inject_alloc_failure.argtypes = [C.c_int]
            L.wick_selftest_wait.argtypes = [C.c_int, C.c_int, vp]
            L.wick_strerror.argtypes = [C.c_int]
            L.wick_strerror.restype = C.c_char_p
            L.wick_version.restype = C.c_char_p
            for f in ("wick_build_blocks", "wick_reduce_terms", "wick_terms_nucleons", "wick_terms_copy",
                      "wick_terms_stats", "wick_terms_select", "wick_terms_magnitudes", "wick_terms_top", "wick_terms_save",
                      "wick_terms_load",
                      "wick_contract", "wick_contract_noalloc", "wick_status", "wick_batch_create",
                      "wick_batch_run", "wick_batch_launches", "wick_synth_propagator", "wick_cluster_product",
                      "wick_det_reduce", "wick_det_reduce_matrix", "wick_det_stats", "wick_det_element_offsets",
                      "wick_det_copy", "wick_det_contract", "wick_det_contract_3pt", "wick_set_tuning",
                      "wick_get_tuning", "wick_build_blocks_3pt", "wick_contract_3pt", "wick_reduce_terms_matrix",
                      "wick_terms_elements", "wick_terms_copy_matrix", "wick_inject_alloc_failure",
                      "wick_selftest_wait"):
                getattr(L, f).restype = C.c_int
            _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return load().wick_strerror(code).decode()
    except RuntimeError:
        return f"error {code}"


def _check(rc, what):
    if rc != WICK_OK:
        raise WickError(rc, what)


_C128 = ("torch.complex128",)
_CPLX = ("torch.complex64", "torch.complex128")


def _buf(x, what: str, dtypes, numel: int, where: str = "cuda", exact: bool = False):
    """Pointer of a torch tensor that the library will read or write, after the checks the C side
    cannot make: dtype, contiguity, size (at least `numel` elements, exactly with `exact`) and
    placement ("cuda": device memory; "pinned": page-locked host memory).  Raw integer pointers pass
    through unchecked.  A bad tensor raises ValueError before anything reaches libwick."""
    if isinstance(x, int):
        return x
    if x is None:
        raise ValueError(f"{what}: a tensor is required")
    if str(x.dtype) not in dtypes:
        raise ValueError(f"{what}: dtype {x.dtype}, expected {' or '.join(dtypes)}")
    if not x.is_contiguous():
        raise ValueError(f"{what}: tensor is not contiguous")
    if x.numel() < numel or (exact and x.numel() != numel):
        raise ValueError(f"{what}: {x.numel()} elements, {'exactly' if exact else 'at least'} {numel} needed")
    if where == "cuda" and not x.is_cuda:
        raise ValueError(f"{what}: tensor is not in CUDA device memory")
    if where == "pinned" and (x.is_cuda or not x.is_pinned()):
        raise ValueError(f"{what}: tensor is not in page-locked host memory")
    return x.data_ptr()


def _dtype_code(S) -> int:
    return WICK_C64 if str(getattr(S, "dtype", "")) == "torch.complex64" else WICK_C128


def _prop(S, L: int, T: int, n_src: int, what: str, where: str = "cuda") -> "wick_prop":
    """wick_prop of a propagator tensor [n_src][T][L^3][3][4][3][4] (complex64 or complex128)."""
    n = n_src * T * L ** 3 * 144
    return wick_prop(_buf(S, what, _CPLX, n, where, exact=True), L, T, n_src, _dtype_code(S))


def _stream(stream):
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _np_ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class Tables:
    """ctypes views of a `operators.Nucleus` (keeps the numpy arrays alive)."""

    def __init__(self, nuc: _ops.Nucleus):
        self.nuc = nuc
        self._keep = []
        n_ops = len(nuc.ops)
        self.ops = (wick_nucleon_op * n_ops)()
        for o, op in enumerate(nuc.ops):
            ent = np.array([e[:4] for e in op.entries], dtype=np.int8).reshape(-1)
            w = np.array([e[4] for e in op.entries], dtype=np.int32)
            self._keep += [ent, w]
            self.ops[o] = wick_nucleon_op(len(op.entries), _np_ptr(ent, C.c_int8), _np_ptr(w, C.c_int32),
                                          op.flav_pair)
        chi = (C.c_int8 * 12)(*(list(nuc.chi) + [0] * (12 - len(nuc.chi))))
        self.layout = wick_block_layout(n_ops, nuc.n_spin, len(nuc.chi), chi)
        A = nuc.A
        st = np.array([t for t, _, _ in nuc.sink], dtype=np.int8).reshape(-1)
        ss = np.array([s for _, s, _ in nuc.sink], dtype=np.int8).reshape(-1)
        sw = np.array([w for _, _, w in nuc.sink], dtype=np.int64)
        sc = np.array([c for c, _ in nuc.src], dtype=np.int8).reshape(-1)
        cw = np.array([w for _, w in nuc.src], dtype=np.int64)
        fl = np.array(nuc.src_flav, dtype=np.int8)
        self._keep += [st, ss, sw, sc, cw, fl]
        self.nucleus = wick_nucleus(A, len(nuc.sink), _np_ptr(st, C.c_int8), _np_ptr(ss, C.c_int8),
                                    _np_ptr(sw, C.c_int64), len(nuc.src), _np_ptr(sc, C.c_int8),
                                    _np_ptr(cw, C.c_int64), _np_ptr(fl, C.c_int8), float(nuc.scale))


def wick_block_count(tables: Tables) -> int:
    return int(load().wick_block_count(C.byref(tables.layout)))


def wick_build_blocks(Su, Sd, tables: Tables, precision: int, blocks, L: int, T: int, n_src: int, stream=None):
    """Blocks[src][t][n_blk] complex128 (torch.complex128 CUDA tensor) from Su, Sd."""
    pu, pd = _prop(Su, L, T, n_src, "Su"), _prop(Sd, L, T, n_src, "Sd")
    pb = _buf(blocks, "blocks", _C128, n_src * T * tables.nuc.n_blk)
    _check(load().wick_build_blocks(C.byref(pu), C.byref(pd), tables.ops, C.byref(tables.layout), precision,
                                    pb, _stream(stream)), "wick_build_blocks")


def wick_upload_rows(Su_host, Sd_host, Su_dev, Sd_dev, tables: Tables, L: int, T: int, n_src: int,
                     stream=None, mode: int = 0) -> int:
    """Copy the rows of S the block build of `tables` reads from pinned host tensors to device tensors of
    the same shape (mode WICK_UPLOAD_AUTO / _DMA / _KERNEL); returns the bytes copied."""
    hu, hd = _prop(Su_host, L, T, n_src, "Su_host", "pinned"), _prop(Sd_host, L, T, n_src, "Sd_host", "pinned")
    du, dd = _prop(Su_dev, L, T, n_src, "Su_dev"), _prop(Sd_dev, L, T, n_src, "Sd_dev")
    n = C.c_size_t(0)
    _check(load().wick_upload_rows(C.byref(hu), C.byref(hd), C.byref(du), C.byref(dd), tables.ops,
                                   C.byref(tables.layout), mode, C.byref(n), _stream(stream)), "wick_upload_rows")
    return int(n.value)


class Terms:
    """Library-owned reduced term table."""

    def __init__(self, handle):
        self.h = C.c_void_p(handle)

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "h", None) and self.h.value:
            load().wick_terms_free(self.h)
            self.h = C.c_void_p(None)

    @property
    def count(self) -> int:
        return int(load().wick_terms_count(self.h))

    @property
    def nucleons(self) -> int:
        return int(load().wick_terms_nucleons(self.h))

    @property
    def elements(self) -> int:
        """Weight columns: 1, or N * N for a correlation-matrix table."""
        return int(load().wick_terms_elements(self.h))

    def copy_matrix(self):
        U, A, E = self.count, self.nucleons, self.elements
        ids = np.zeros((max(U, 1), A), dtype=np.uint16)
        w = np.zeros((max(U, 1), E), dtype=np.int64)
        sc = np.zeros(E, dtype=np.float64)
        _check(load().wick_terms_copy_matrix(self.h, ids.ctypes.data, w.ctypes.data, sc.ctypes.data),
               "wick_terms_copy_matrix")
        return dict(ids=ids[:U], w=w[:U], scale=sc)

    @property
    def block_count(self) -> int:
        """Block entries per (source, time slice) of the layout the table was reduced for."""
        n = int(load().wick_terms_block_count(self.h))
        if n < 0:
            raise WickError(n, "wick_terms_block_count")
        return n

    def copy(self):
        U, A = self.count, self.nucleons
        ids = np.zeros((U, A), dtype=np.uint16)
        w = np.zeros(U, dtype=np.int64)
        rep = np.zeros(U, dtype=np.int64)
        _check(load().wick_terms_copy(self.h, ids.ctypes.data, w.ctypes.data, rep.ctypes.data), "wick_terms_copy")
        return dict(ids=ids, w=w, rep=rep)

    def stats(self):
        st = np.zeros(4, dtype=np.int64)
        b = C.c_double(0)
        _check(load().wick_terms_stats(self.h, _np_ptr(st, C.c_int64), C.byref(b)), "wick_terms_stats")
        return tuple(int(x) for x in st), float(b.value)

    def select(self, perm):
        p = np.ascontiguousarray(perm, dtype=np.int64)
        _check(load().wick_terms_select(self.h, _np_ptr(p, C.c_int64), len(p)), "wick_terms_select")

    def magnitudes(self, blocks, n_slices: int, stream=None) -> np.ndarray:
        """Each term's |contribution| summed over the n_slices slices of `blocks` (Sec. V.C)."""
        pb = _buf(blocks, "blocks", _C128, n_slices * self.block_count)
        mag = np.zeros(max(self.count, 1), dtype=np.float64)
        _check(load().wick_terms_magnitudes(pb, n_slices, self.h, _np_ptr(mag, C.c_double), _stream(stream)),
               "wick_terms_magnitudes")
        return mag[:self.count]

    def top(self, mag, fraction: float):
        """Keep the ceil(fraction * U) terms of largest magnitude (wick_terms_top)."""
        m = np.ascontiguousarray(mag, dtype=np.float64)
        if len(m) != self.count:
            raise ValueError("one magnitude per term is needed")
        _check(load().wick_terms_top(self.h, _np_ptr(m, C.c_double), float(fraction)), "wick_terms_top")

    def save(self, path: str):
        _check(load().wick_terms_save(self.h, path.encode()), "wick_terms_save")

    @classmethod
    def load_file(cls, path: str) -> "Terms":
        h = C.c_void_p(None)
        _check(load().wick_terms_load(path.encode(), C.byref(h)), "wick_terms_load")
        return cls(h.value)


def wick_reduce_terms(tables: Tables, seed: int = 0x2411, trials: int = 2, sites: int = 1, stream=None) -> Terms:
    h = C.c_void_p(None)
    _check(load().wick_reduce_terms(C.byref(tables.nucleus), tables.ops, C.byref(tables.layout), seed, trials, sites,
                                    C.byref(h), _stream(stream)), "wick_reduce_terms")
    return Terms(h.value)


def _contract_args(blocks, n_src, T, terms, C_out):
    nb = terms.block_count
    n_el = getattr(terms, "elements", 1)
    return (_buf(blocks, "blocks", _C128, n_src * T * nb), _buf(C_out, "C_out", _C128, n_el * n_src * T))


def wick_contract(blocks, n_src: int, T: int, terms: Terms, precision: int, C_out, stream=None):
    pb, pc = _contract_args(blocks, n_src, T, terms, C_out)
    _check(load().wick_contract(pb, n_src, T, terms.h, precision, pc, _stream(stream)), "wick_contract")


def wick_contract_noalloc(blocks, n_src: int, T: int, terms: Terms, precision: int, C_out, stream=None):
    """wick_contract for callers that cannot allocate device memory: its scratch
    is a fixed 1 MiB device array inside the library (see include/wick.h)."""
    pb, pc = _contract_args(blocks, n_src, T, terms, C_out)
    _check(load().wick_contract_noalloc(pb, n_src, T, terms.h, precision, pc, _stream(stream)),
           "wick_contract_noalloc")


def wick_reduce_terms_matrix(tables_list, seed: int = 0x2411, trials: int = 2, sites: int = 1, stream=None) -> Terms:
    """Correlation-matrix table of N operators (`Tables` of nuclei with the same nucleon operators and
    quark content; element i * N + j: sink of operator i, source of operator j)."""
    n = len(tables_list)
    arr = (wick_nucleus * n)(*[t.nucleus for t in tables_list])
    h = C.c_void_p(None)
    t0 = tables_list[0]
    _check(load().wick_reduce_terms_matrix(arr, n, t0.ops, C.byref(t0.layout), seed, trials, sites, C.byref(h),
                                           _stream(stream)), "wick_reduce_terms_matrix")
    return Terms(h.value)


def wick_build_blocks_3pt(Su, Sd, Sig, flavour: int, tables: Tables, precision: int, dblocks, L: int, T: int,
                          n_src: int, stream=None):
    """Derivative blocks D[src][t][n_blk] (complex128) of a current on `flavour` through Sig."""
    pu, pd = _prop(Su, L, T, n_src, "Su"), _prop(Sd, L, T, n_src, "Sd")
    pg = _prop(Sig, L, T, n_src, "Sig")
    pb = _buf(dblocks, "dblocks", _C128, n_src * T * tables.nuc.n_blk)
    _check(load().wick_build_blocks_3pt(C.byref(pu), C.byref(pd), C.byref(pg), flavour, tables.ops,
                                        C.byref(tables.layout), precision, pb, _stream(stream)),
           "wick_build_blocks_3pt")


def wick_contract_3pt(blocks, dblocks, n_src: int, T: int, terms: Terms, precision: int, C_out, stream=None):
    """Three-point function C3[src][t] from the blocks, the derivative blocks and the two-point table."""
    pb, pc = _contract_args(blocks, n_src, T, terms, C_out)
    pdb = _buf(dblocks, "dblocks", _C128, n_src * T * terms.block_count)
    _check(load().wick_contract_3pt(pb, pdb, n_src, T, terms.h, precision, pc, _stream(stream)), "wick_contract_3pt")


class Batch:
    """A captured batch (wick_batch_create); keeps its inputs alive."""

    def __init__(self, Su_list, Sd_list, tables: Tables, terms_list, precision, blocks, C_out, L, T, n_src):
        n = len(Su_list)

        def props(lst, what):
            arr = (wick_prop * n)()
            for i, S in enumerate(lst):
                arr[i] = _prop(S, L, T, n_src, f"{what}[{i}]")
            return arr
        self._keep = (Su_list, Sd_list, tables, terms_list, blocks, C_out)
        if len(Sd_list) != n:
            raise ValueError("Su_list and Sd_list differ in length")
        self.su, self.sd = props(Su_list, "Su_list"), props(Sd_list, "Sd_list")
        pb = _buf(blocks, "blocks", _C128, n * n_src * T * tables.nuc.n_blk)
        pc = _buf(C_out, "C_out", _C128, n * len(terms_list) * n_src * T)
        handles = (C.c_void_p * len(terms_list))(*[t.h.value for t in terms_list])
        h = C.c_void_p(None)
        _check(load().wick_batch_create(self.su, self.sd, n, tables.ops, C.byref(tables.layout), handles,
                                        len(terms_list), precision, pb, pc, C.byref(h)),
               "wick_batch_create")
        self.h = h

    def run(self, stream=None):
        _check(load().wick_batch_run(self.h, _stream(stream)), "wick_batch_run")

    @property
    def launches(self) -> int:
        return int(load().wick_batch_launches(self.h))

    def free(self):
        if getattr(self, "h", None) and self.h.value:
            load().wick_batch_free(self.h)
            self.h = C.c_void_p(None)

    def __del__(self):
        self.free()


def wick_synth_propagator(seed: int, flavour: int, src: int, L: int, T: int, out, stream=None):
    """Device-generated synthetic propagator of one (flavour, source) into `out`."""
    po = _buf(out, "out", _CPLX, T * L ** 3 * 144, exact=True)
    _check(load().wick_synth_propagator(seed, flavour, src, L, T, _dtype_code(out), po, _stream(stream)),
           "wick_synth_propagator")


def wick_cluster_product(Ca, Cb, out, stream=None):
    """out = Ca * Cb elementwise (complex128 device tensors of equal size)."""
    n = Ca.numel()
    pa, pb = _buf(Ca, "Ca", _C128, n, exact=True), _buf(Cb, "Cb", _C128, n, exact=True)
    po = _buf(out, "out", _C128, n, exact=True)
    _check(load().wick_cluster_product(pa, pb, n, po, _stream(stream)),
           "wick_cluster_product")


TUNING_FIELDS = ("range_sites", "contract_threads", "contract_ctas_per_sm", "contract_chunk_terms",
                 "hash_log2_start", "hash_log2_max", "no_pair_kernel")


def wick_set_tuning(tuning=None):
    """Process-wide launch tuning (a dict with any of TUNING_FIELDS, 0 = default; None = all defaults)."""
    t = wick_tuning(*[int((tuning or {}).get(f, 0)) for f in TUNING_FIELDS])
    _check(load().wick_set_tuning(C.byref(t)), "wick_set_tuning")


def wick_get_tuning() -> dict:
    t = wick_tuning()
    _check(load().wick_get_tuning(C.byref(t)), "wick_get_tuning")
    return {f: int(getattr(t, f)) for f in TUNING_FIELDS}


def wick_status(stream=None) -> int:
    return int(load().wick_status(_stream(stream)))


def wick_inject_alloc_failure(k: int) -> int:
    """Make the library's k-th device allocation from now report failure (host-side fault injection;
    0 cancels); returns the allocations that were still to go before a pending injected failure."""
    r = int(load().wick_inject_alloc_failure(int(k)))
    if r < 0:
        raise WickError(r, "wick_inject_alloc_failure")
    return r


def wick_selftest_wait(which: int, limit: int, stream=None) -> int:
    """Run a bounded device wait (0 hash-slot, 1 mbarrier) on a flag nothing sets; returns the status the
    kernel recorded (WICK_ETIMEOUT when the wait ran out)."""
    r = int(load().wick_selftest_wait(int(which), int(limit), _stream(stream)))
    if r in (WICK_EINVAL, WICK_ENOMEM, WICK_ECUDA):
        raise WickError(r, "wick_selftest_wait")
    return r


def wick_version() -> str:
    return load().wick_version().decode()


# ---------------------------------------------------------------------------
# point-sink determinant algorithm
# ---------------------------------------------------------------------------
def _quark_op(q):
    chi = np.ascontiguousarray(q.chi, dtype=np.int8)
    w = np.ascontiguousarray(q.w, dtype=np.int64)
    s = wick_quark_operator(int(q.n_u), int(q.n_d), len(w), chi.ctypes.data_as(C.POINTER(C.c_int8)),
                            w.ctypes.data_as(C.POINTER(C.c_int64)))
    return s, (chi, w)


class DetPlan:
    """Library-owned minimal sets zeta_u, zeta_d and Theta of a point-sink operator pair (wick_det_reduce)."""

    def __init__(self, sink, source=None, seed: int = 0x2411D7, trials: int = 2, matrix=None):
        """One correlator (sink, source), or with `matrix` = [O_1 .. O_N] the N x N correlation matrix."""
        h = C.c_void_p()
        if matrix is not None:
            ops = [_quark_op(q) for q in matrix]
            arr = (wick_quark_operator * len(ops))(*[o[0] for o in ops])
            _check(load().wick_det_reduce_matrix(arr, len(ops), seed, trials, C.byref(h)), "wick_det_reduce_matrix")
            self.scale = float(getattr(matrix[0], "scale", 1.0))
        else:
            source = sink if source is None else source
            a, keep_a = _quark_op(sink)
            b, keep_b = _quark_op(source)
            _check(load().wick_det_reduce(C.byref(a), C.byref(b), seed, trials, C.byref(h)), "wick_det_reduce")
            self.scale = float(getattr(sink, "scale", 1.0))
        self.h = h

    def stats(self) -> dict:
        out = (C.c_int64 * 7)()
        _check(load().wick_det_stats(self.h, out), "wick_det_stats")
        return dict(n_sink=out[0], n_source=out[1], zeta_u=out[2], zeta_d=out[3], theta=out[4],
                    n_u=out[5] // 8, n_d=out[5] % 8, n_el=out[6])

    def element_offsets(self) -> np.ndarray:
        off = np.zeros(self.stats()["n_el"] + 1, np.int64)
        _check(load().wick_det_element_offsets(self.h, off.ctypes.data_as(C.POINTER(C.c_int64))),
               "wick_det_element_offsets")
        return off

    def copy(self) -> dict:
        st = self.stats()
        k = np.zeros(max(st["theta"], 1), np.int32)
        l = np.zeros_like(k)
        w = np.zeros(max(st["theta"], 1), np.int64)
        zu = [np.zeros((max(st["zeta_u"], 1), max(st["n_u"], 1)), np.int8) for _ in range(2)]
        zd = [np.zeros((max(st["zeta_d"], 1), max(st["n_d"], 1)), np.int8) for _ in range(2)]
        _check(load().wick_det_copy(self.h, k.ctypes.data, l.ctypes.data, w.ctypes.data, zu[0].ctypes.data,
                                    zu[1].ctypes.data, zd[0].ctypes.data, zd[1].ctypes.data), "wick_det_copy")
        n = st["theta"]
        return dict(k=k[:n], l=l[:n], w=w[:n], zu_rows=zu[0][:st["zeta_u"], :st["n_u"]],
                    zu_cols=zu[1][:st["zeta_u"], :st["n_u"]], zd_rows=zd[0][:st["zeta_d"], :st["n_d"]],
                    zd_cols=zd[1][:st["zeta_d"], :st["n_d"]])

    def free(self):
        if self.h:
            load().wick_det_free(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def wick_det_contract(Su, Sd, plan: DetPlan, C_out, L: int, T: int, n_src: int, scale=None,
                      precision: int = WICK_FP64, stream=None):
    """C_out[el][src][t] (torch complex128 CUDA tensor; el = i * N + j for a matrix plan, one element
    otherwise) = point-sink correlators of the plan."""
    pu, pd = _prop(Su, L, T, n_src, "Su"), _prop(Sd, L, T, n_src, "Sd")
    pc = _buf(C_out, "C_out", _C128, plan.stats()["n_el"] * n_src * T)
    sc = plan.scale if scale is None else float(scale)
    _check(load().wick_det_contract(C.byref(pu), C.byref(pd), plan.h, sc, precision, pc, _stream(stream)),
           "wick_det_contract")


def wick_det_contract_3pt(Su, Sd, Sig, flavour: int, plan: DetPlan, C_out, L: int, T: int, n_src: int, scale=None,
                          precision: int = WICK_FP64, stream=None):
    """Three-point function: the current on `flavour` (WICK_U / WICK_D) through the sequential propagator Sig."""
    pu, pd = _prop(Su, L, T, n_src, "Su"), _prop(Sd, L, T, n_src, "Sd")
    pq = _prop(Sig, L, T, n_src, "Sig")
    pc = _buf(C_out, "C_out", _C128, plan.stats()["n_el"] * n_src * T)
    sc = plan.scale if scale is None else float(scale)
    _check(load().wick_det_contract_3pt(C.byref(pu), C.byref(pd), C.byref(pq), flavour, plan.h, sc, precision,
                                        pc, _stream(stream)), "wick_det_contract_3pt")
