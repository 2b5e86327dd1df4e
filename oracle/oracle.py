"""Python face of the CPU reference (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this module.  It compiles `wick_oracle.c` with gcc (OpenMP) into
`liboracle.so` next to this file and marshals arguments; all arithmetic is in
that C file (FP64, compensated sums) or, for the operator tables, in
`operators.py`.  Nothing here is shared with the CUDA product library.

Block-id convention of the reduced tables (the same arithmetic the product
library documents for its block layout):
    id = (((op * n_spin + s) * n_chi + i1) * n_chi + i2) * n_chi + i3
with i1..i3 the positions of the source indices chi' in the layout's list.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "wick_oracle.c")
SRC_DET = os.path.join(HERE, "det_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C reference (gcc -O2 -fopenmp); returns the .so path."""
    newest = max(os.path.getmtime(SRC), os.path.getmtime(SRC_DET))
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-o", LIB + ".tmp", SRC, SRC_DET, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


class Problem(C.Structure):
    _fields_ = [
        ("n_ops", C.c_int), ("op_f1", C.POINTER(C.c_int32)), ("op_off", C.POINTER(C.c_int32)),
        ("ent", C.POINTER(C.c_int8)), ("ent_w", C.POINTER(C.c_int32)),
        ("n_spin", C.c_int), ("n_chi", C.c_int), ("chi", C.POINTER(C.c_int8)),
        ("A", C.c_int), ("n_sink", C.c_int), ("sink_type", C.POINTER(C.c_int8)),
        ("sink_spin", C.POINTER(C.c_int8)), ("sink_w", C.POINTER(C.c_int64)),
        ("n_src", C.c_int), ("src_chi", C.POINTER(C.c_int8)), ("src_w", C.POINTER(C.c_int64)),
        ("src_flav", C.POINTER(C.c_int8)),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            P = C.POINTER(Problem)
            dp, i64p, u16p, u64p = (C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_uint16), C.POINTER(C.c_uint64))
            L.oracle_blocks.argtypes = [dp, dp, C.c_int, C.c_int, C.c_int, P, dp]
            L.oracle_raw_correlator.argtypes = [P, dp, C.c_int, C.c_double, dp]
            L.oracle_table_correlator.argtypes = [P, dp, C.c_int, C.c_double, C.c_int64, u16p, i64p, dp]
            L.oracle_dedup.argtypes = [P, C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int64, i64p, i64p, u16p, i64p]
            L.oracle_modp_raw.argtypes = [P, C.c_uint64, u64p]
            L.oracle_modp_table.argtypes = [P, C.c_uint64, C.c_int64, u16p, i64p, u64p]
            i8p = C.POINTER(C.c_int8)
            L.oracle_source_multisets.argtypes = [P, C.c_int64, i8p, i8p, i64p, i64p]
            L.oracle_point_correlator.argtypes = [dp, dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, i8p, i8p,
                                                  C.c_int64, i8p, i8p, C.c_int64, i64p, i64p, dp, dp]
            L.oracle_point_3pt.argtypes = [dp, dp, dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, i8p,
                                           i8p, C.c_int64, i8p, i8p, C.c_int64, i64p, i64p, dp, dp]
            L.oracle_det_modp.argtypes = [u64p, C.c_int, C.c_int64, i8p, i8p, u64p]
            for f in ("oracle_point_correlator", "oracle_point_3pt", "oracle_det_modp",
                      "oracle_blocks", "oracle_raw_correlator", "oracle_table_correlator", "oracle_dedup",
                      "oracle_modp_raw", "oracle_modp_table", "oracle_num_threads", "oracle_source_multisets"):
                getattr(L, f).restype = C.c_int
            _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class _Packed:
    """Keeps the numpy arrays behind a Problem struct alive."""

    def __init__(self, nuc):
        ops = nuc["ops"]
        self.op_f1 = np.array([f for f, _ in ops], dtype=np.int32)
        off = [0]
        ent, ent_w = [], []
        for _, tab in ops:
            for (s, r1, r2, r3, w) in tab:
                ent += [s, r1, r2, r3]
                ent_w.append(w)
            off.append(len(ent_w))
        self.op_off = np.array(off, dtype=np.int32)
        self.ent = np.array(ent, dtype=np.int8)
        self.ent_w = np.array(ent_w, dtype=np.int32)
        self.chi = np.array(nuc["chi"], dtype=np.int8)
        A = nuc["A"]
        self.sink_type = np.array([t for t, _, _ in nuc["sink"]], dtype=np.int8).reshape(-1, A)
        self.sink_spin = np.array([s for _, s, _ in nuc["sink"]], dtype=np.int8).reshape(-1, A)
        self.sink_w = np.array([w for _, _, w in nuc["sink"]], dtype=np.int64)
        self.src_chi = np.array([c for c, _ in nuc["src"]], dtype=np.int8).reshape(-1, 3 * A)
        self.src_w = np.array([w for _, w in nuc["src"]], dtype=np.int64)
        self.src_flav = np.array(nuc["src_flav"], dtype=np.int8)
        self.p = Problem(
            len(ops), _ptr(self.op_f1, C.c_int32), _ptr(self.op_off, C.c_int32),
            _ptr(self.ent, C.c_int8), _ptr(self.ent_w, C.c_int32),
            nuc["n_spin"], len(nuc["chi"]), _ptr(self.chi, C.c_int8),
            A, len(nuc["sink"]), _ptr(self.sink_type, C.c_int8), _ptr(self.sink_spin, C.c_int8),
            _ptr(self.sink_w, C.c_int64), len(nuc["src"]), _ptr(self.src_chi, C.c_int8),
            _ptr(self.src_w, C.c_int64), _ptr(self.src_flav, C.c_int8))
        self.n_blk = len(ops) * nuc["n_spin"] * len(nuc["chi"]) ** 3


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def num_threads() -> int:
    return lib().oracle_num_threads()


def blocks_single(Su: np.ndarray, Sd: np.ndarray, nuc) -> np.ndarray:
    """Single-product blocks Bhat[src][t][n_blk] (complex128), FP64 site sums."""
    Su = np.ascontiguousarray(Su, dtype=np.complex128)
    Sd = np.ascontiguousarray(Sd, dtype=np.complex128)
    n_src, T, V = Su.shape[:3]
    pk = _Packed(nuc)
    out = np.zeros((n_src, T, pk.n_blk), dtype=np.complex128)
    _check(lib().oracle_blocks(_ptr(Su.view(np.float64), C.c_double), _ptr(Sd.view(np.float64), C.c_double),
                               n_src, T, V, C.byref(pk.p), _ptr(out.view(np.float64), C.c_double)), "blocks")
    return out


def antisymmetric_blocks(Bhat: np.ndarray, nuc) -> np.ndarray:
    """B(c1,c2,c3) = Bhat(c1,c2,c3) - Bhat(c2,c1,c3) (Eq. 2.4)."""
    nc = len(nuc["chi"])
    b = Bhat.reshape(Bhat.shape[:-1] + (-1, nc, nc, nc))
    return (b - b.swapaxes(-3, -2)).reshape(Bhat.shape)


def raw_correlator(nuc, Bhat: np.ndarray) -> np.ndarray:
    """Plain Wick sum over every raw term; C[src][t] complex128."""
    pk = _Packed(nuc)
    shp = Bhat.shape[:-1]
    Bh = np.ascontiguousarray(Bhat.reshape(-1, pk.n_blk))
    out = np.zeros(Bh.shape[0], dtype=np.complex128)
    _check(lib().oracle_raw_correlator(C.byref(pk.p), _ptr(Bh.view(np.float64), C.c_double), Bh.shape[0],
                                       float(nuc["scale"]), _ptr(out.view(np.float64), C.c_double)), "raw")
    return out.reshape(shp)


def table_correlator(nuc, Bhat: np.ndarray, table) -> np.ndarray:
    """C[src][t] from a reduced table with antisymmetric blocks."""
    pk = _Packed(nuc)
    shp = Bhat.shape[:-1]
    Bh = np.ascontiguousarray(Bhat.reshape(-1, pk.n_blk))
    ids = np.ascontiguousarray(table["ids"], dtype=np.uint16)
    w = np.ascontiguousarray(table["w"], dtype=np.int64)
    out = np.zeros(Bh.shape[0], dtype=np.complex128)
    _check(lib().oracle_table_correlator(C.byref(pk.p), _ptr(Bh.view(np.float64), C.c_double), Bh.shape[0],
                                         float(nuc["scale"]), len(w), _ptr(ids, C.c_uint16), _ptr(w, C.c_int64),
                                         _ptr(out.view(np.float64), C.c_double)), "table")
    return out.reshape(shp)


def term_contributions(nuc, Bhat: np.ndarray, table) -> np.ndarray:
    """Each reduced term's contribution to C (Sec. V.C): c[u][slice] = scale w_u prod_k B[slice][id_{u,k}]
    with the antisymmetric blocks, slices = the flattened leading axes of Bhat.  Their sum over u is
    table_correlator (written separately, in numpy)."""
    B = antisymmetric_blocks(np.asarray(Bhat, dtype=np.complex128), nuc)
    B = B.reshape(-1, B.shape[-1])
    ids = np.asarray(table["ids"], dtype=np.int64)
    w = np.asarray(table["w"], dtype=np.float64)
    prod = np.ones((len(w), B.shape[0]), dtype=np.complex128)
    for k in range(ids.shape[1]):
        prod = prod * B[:, ids[:, k]].T
    return float(nuc["scale"]) * w[:, None] * prod


def top_terms(mag: np.ndarray, fraction: float) -> np.ndarray:
    """Indices of the ceil(fraction * U) largest magnitudes, ties to the smaller index (Sec. V.C),
    in ascending index order."""
    U = len(mag)
    n = max(1, min(U, int(np.ceil(fraction * U - 1e-9)))) if U else 0
    order = sorted(range(U), key=lambda u: (-mag[u], u))
    return np.array(sorted(order[:n]), dtype=np.int64)


def three_point_planewave(Su, Sd, Sig, flavour: int, nuc, table=None) -> np.ndarray:
    """Three-point function with the plane-wave sink (Sec. IV.A, Eq. Proton3pt_seq generalised):
    the connected term of a current on `flavour` (0 = u, 1 = d) through the sequential propagator
    Sig, i.e. every Wick term with one line of that flavour replaced by Sig, summed over the lines:
    the linear coefficient of C(S_f + e Sig) in e.  C is a polynomial of degree n_f (the quarks of
    that flavour) in e, so the coefficient is extracted exactly by the discrete Fourier transform over
    the m = n_f + 1 roots of unity: c_1 = (1/m) sum_k C(w^k) w^(-k), w = exp(2 pi i / m).  Each C is the
    plain definition (single-product blocks and the raw Wick sum), or the reduced-table sum of
    `table` when given."""
    nu, nd = ops_quark_counts(nuc)
    m = (nu if flavour == 0 else nd) + 1
    acc = 0.0
    for k in range(m):
        e = np.exp(2j * np.pi * k / m)
        su = Su + e * Sig if flavour == 0 else Su
        sd = Sd + e * Sig if flavour == 1 else Sd
        Bh = blocks_single(su, sd, nuc)
        C = table_correlator(nuc, Bh, table) if table is not None else raw_correlator(nuc, Bh)
        acc = acc + C * np.conj(e)
    return acc / m


def ops_quark_counts(nuc):
    nu = sum(1 for f in nuc["src_flav"] if f == 0)
    return nu, len(nuc["src_flav"]) - nu


def matrix_element(nuc_sink, nuc_source):
    """The correlator with the sink of one operator and the source of another (Eq. E1): a nucleus
    dict with the sink half of nuc_sink and the source half of nuc_source, scale sqrt(s_i s_j)."""
    el = dict(nuc_sink)
    el["src"] = nuc_source["src"]
    el["scale"] = float(np.sqrt(nuc_sink["scale"] * nuc_source["scale"]))
    return el


def source_multisets(nuc):
    """Antisymmetrised source: dict(Mu[n_M][n_u], Md[n_M][n_d], CM[n_M], n_red)."""
    pk = _Packed(nuc)
    nu = int(np.sum(pk.src_flav == 0))
    nd = len(pk.src_flav) - nu
    cap = max(1, len(pk.src_w))
    Mu = np.zeros((cap, max(nu, 1)), dtype=np.int8)
    Md = np.zeros((cap, max(nd, 1)), dtype=np.int8)
    CM = np.zeros(cap, dtype=np.int64)
    counts = np.zeros(2, dtype=np.int64)
    _check(lib().oracle_source_multisets(C.byref(pk.p), cap, _ptr(Mu, C.c_int8), _ptr(Md, C.c_int8),
                                         _ptr(CM, C.c_int64), _ptr(counts, C.c_int64)), "source_multisets")
    n = int(counts[0])
    return dict(Mu=Mu[:n, :nu].copy(), Md=Md[:n, :nd].copy(), CM=CM[:n].copy(), n_red=int(counts[1]))


def dedup(nuc, seed: int = 0x0BAC1E, trials: int = 2, V0: int = 1, mode: str = "hash", cap: int | None = None):
    """Reduced term table: dict(rep, w, ids[U][A], stats=(raw terms of the
    reduction, identically zero, classes, kept))."""
    pk = _Packed(nuc)
    n_raw = source_multisets(nuc)["n_red"]
    if cap is None:
        cap = max(1, min(n_raw, 1 << 24))
    rep = np.zeros(cap, dtype=np.int64)
    w = np.zeros(cap, dtype=np.int64)
    ids = np.zeros((cap, nuc["A"]), dtype=np.uint16)
    stats = np.zeros(4, dtype=np.int64)
    _check(lib().oracle_dedup(C.byref(pk.p), seed, trials, V0, 0 if mode == "hash" else 1, cap,
                              _ptr(rep, C.c_int64), _ptr(w, C.c_int64), _ptr(ids, C.c_uint16),
                              _ptr(stats, C.c_int64)), "dedup")
    U = int(stats[3])
    return dict(rep=rep[:U].copy(), w=w[:U].copy(), ids=ids[:U].copy(), stats=tuple(int(x) for x in stats))


def modp_raw(nuc, seed: int) -> int:
    pk = _Packed(nuc)
    out = C.c_uint64(0)
    _check(lib().oracle_modp_raw(C.byref(pk.p), seed, C.byref(out)), "modp_raw")
    return int(out.value)


def modp_table(nuc, table, seed: int) -> int:
    pk = _Packed(nuc)
    ids = np.ascontiguousarray(table["ids"], dtype=np.uint16)
    w = np.ascontiguousarray(table["w"], dtype=np.int64)
    out = C.c_uint64(0)
    _check(lib().oracle_modp_table(C.byref(pk.p), seed, len(w), _ptr(ids, C.c_uint16), _ptr(w, C.c_int64),
                                   C.byref(out)), "modp_table")
    return int(out.value)


def correlator(Su, Sd, nuc) -> np.ndarray:
    """The plain definition end to end: single-product blocks, raw Wick sum."""
    return raw_correlator(nuc, blocks_single(Su, Sd, nuc))
