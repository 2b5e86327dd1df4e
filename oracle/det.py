"""CPU reference of the point-sink determinant algorithm (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this module; the GPU product path never does, and nothing here is
shared with the product library.

Eq. 2.9 (Sec. III.A) with the coefficient tables antisymmetrised within each
flavour (Sec. III.C, method A):

    G(t) = scale * sum_x sum_{M, M'} C[M] C'[M'] det M^u(x; M_u, M'_u) det M^d(x; M_d, M'_d)

M, M' run over flavour-ordered index lists (sorted u indices, sorted d
indices); M^f_ij = S_f(x, t)(chi_i, chi'_j).  The determinants are evaluated
by their definition (Leibniz sum) in `det_oracle.c`, once per distinct
(row set, column set) pair and site.

Three-point functions (Sec. "Three-point functions", Eq. Proton3pt_seq): the
current on flavour f through a sequential propagator Sigma_f replaces one
f-quark line of every Wick term by Sigma_f, summed over the lines, i.e. each
f determinant becomes the sum of the determinants with one row taken from
Sigma_f (the derivative of Eq. 2.9 in the direction Sigma_f).

The minimal set of App. A (Eq. a1): zeta_u, zeta_d = the distinct determinant
index pairs, Theta(k, l) = sum of C[M] C'[M'] over the (M, M') whose u pair is
k and d pair is l.  `minimal_sets` finds them by comparing index lists;
`minimal_sets_modp` by the paper's randomised identity testing (Sec. III.B,
App. C): every determinant evaluated at random integer matrices modulo
p = 2^61 - 1, equal value vectors merged.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import operators as ops
from .oracle import _check, _ptr, lib

P61 = (1 << 61) - 1


def pair_structure(snk_table, src_table, n_u: int):
    """Antisymmetrise both tables and list, for every (M, M') pair with a
    non-zero product of coefficients, its u pair, d pair and weight.

    Returns dict(pu=[(rows, cols)], pd=[(rows, cols)], t_pu, t_pd, t_w,
    n_snk, n_src): the distinct pairs in order of first appearance."""
    snk = ops.antisymmetrised(snk_table, n_u)
    src = ops.antisymmetrised(src_table, n_u)
    pu, pd, iu, idd = [], [], {}, {}
    t_pu, t_pd, t_w = [], [], []
    for (mu, md), w in sorted(snk.items()):
        for (mu2, md2), w2 in sorted(src.items()):
            ku = (mu, mu2)
            kd = (md, md2)
            if ku not in iu:
                iu[ku] = len(pu)
                pu.append(ku)
            if kd not in idd:
                idd[kd] = len(pd)
                pd.append(kd)
            t_pu.append(iu[ku])
            t_pd.append(idd[kd])
            t_w.append(w * w2)
    return dict(pu=pu, pd=pd, t_pu=np.array(t_pu, dtype=np.int64), t_pd=np.array(t_pd, dtype=np.int64),
                t_w=np.array(t_w, dtype=np.int64), n_snk=len(snk), n_src=len(src))


def _index_arrays(pairs, n):
    rows = np.zeros((max(len(pairs), 1), max(n, 1)), dtype=np.int8)
    cols = np.zeros_like(rows)
    for k, (r, c) in enumerate(pairs):
        rows[k, :n] = r
        cols[k, :n] = c
    return rows, cols


def point_correlator(Su, Sd, snk_table, src_table, n_u: int, n_d: int, scale: float = 1.0, structure=None):
    """G[src][t] (complex128) of Eq. 2.9 for propagators S[src][t][x][3][4][3][4]."""
    st = structure or pair_structure(snk_table, src_table, n_u)
    Su = np.ascontiguousarray(Su, dtype=np.complex128)
    Sd = np.ascontiguousarray(Sd, dtype=np.complex128)
    n_src, T, V = Su.shape[:3]
    ur, uc = _index_arrays(st["pu"], n_u)
    dr, dc = _index_arrays(st["pd"], n_d)
    w = st["t_w"].astype(np.float64)
    out = np.zeros(n_src * T, dtype=np.complex128)
    i8, i64, dp = C.c_int8, C.c_int64, C.c_double
    _check(lib().oracle_point_correlator(
        _ptr(Su.view(np.float64), dp), _ptr(Sd.view(np.float64), dp), V, n_src * T, n_u, n_d,
        len(st["pu"]), _ptr(ur, i8), _ptr(uc, i8), len(st["pd"]), _ptr(dr, i8), _ptr(dc, i8),
        len(w), _ptr(st["t_pu"], i64), _ptr(st["t_pd"], i64), _ptr(w, dp),
        _ptr(out.view(np.float64), dp)), "point_correlator")
    return scale * out.reshape(n_src, T)


def point_3pt(Su, Sd, Sig, flavour: int, snk_table, src_table, n_u: int, n_d: int, scale: float = 1.0,
              structure=None):
    """Three-point function G3[src][t] with the current on `flavour` (0 = u, 1 = d) inserted through the
    sequential propagator Sig (same layout as S): the derivative of Eq. 2.9 in the direction Sig."""
    st = structure or pair_structure(snk_table, src_table, n_u)
    Su = np.ascontiguousarray(Su, dtype=np.complex128)
    Sd = np.ascontiguousarray(Sd, dtype=np.complex128)
    Sg = np.ascontiguousarray(Sig, dtype=np.complex128)
    n_src, T, V = Su.shape[:3]
    ur, uc = _index_arrays(st["pu"], n_u)
    dr, dc = _index_arrays(st["pd"], n_d)
    w = st["t_w"].astype(np.float64)
    out = np.zeros(n_src * T, dtype=np.complex128)
    i8, i64, dp = C.c_int8, C.c_int64, C.c_double
    _check(lib().oracle_point_3pt(
        _ptr(Su.view(np.float64), dp), _ptr(Sd.view(np.float64), dp), _ptr(Sg.view(np.float64), dp), flavour, V,
        n_src * T, n_u, n_d, len(st["pu"]), _ptr(ur, i8), _ptr(uc, i8), len(st["pd"]), _ptr(dr, i8), _ptr(dc, i8),
        len(w), _ptr(st["t_pu"], i64), _ptr(st["t_pd"], i64), _ptr(w, dp),
        _ptr(out.view(np.float64), dp)), "point_3pt")
    return scale * out.reshape(n_src, T)


def minimal_sets(snk_table, src_table, n_u: int):
    """zeta_u, zeta_d (lists of (rows, cols)) and Theta {(k, l): weight}, zeros dropped."""
    st = pair_structure(snk_table, src_table, n_u)
    theta = {}
    for k, l, w in zip(st["t_pu"], st["t_pd"], st["t_w"]):
        theta[(int(k), int(l))] = theta.get((int(k), int(l)), 0) + int(w)
    theta = {k: v for k, v in theta.items() if v}
    return st["pu"], st["pd"], theta


def splitmix64(x: int) -> int:
    """SplitMix64 output function (Steele, Lea, Flood 2014)."""
    x &= (1 << 64) - 1
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & ((1 << 64) - 1)
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & ((1 << 64) - 1)
    return x ^ (x >> 31)


def random_matrix_modp(seed: int, trial: int, flavour: int) -> np.ndarray:
    """12 x 12 integers uniform in [0, p): entry e = splitmix64(seed + (key + e + 1) * gamma) mod p."""
    g = 0x9E3779B97F4A7C15
    key = splitmix64(seed ^ (0x1000 * (trial + 1) + flavour))
    vals = [splitmix64((key + (e + 1) * g) & ((1 << 64) - 1)) % P61 for e in range(144)]
    return np.array(vals, dtype=np.uint64).reshape(12, 12)


def det_modp(M: np.ndarray, pairs, n: int) -> np.ndarray:
    rows, cols = _index_arrays(pairs, n)
    out = np.zeros(max(len(pairs), 1), dtype=np.uint64)
    M = np.ascontiguousarray(M, dtype=np.uint64)
    _check(lib().oracle_det_modp(_ptr(M, C.c_uint64), n, len(pairs), _ptr(rows, C.c_int8), _ptr(cols, C.c_int8),
                                 _ptr(out, C.c_uint64)), "det_modp")
    return out[:len(pairs)]


def minimal_sets_modp(snk_table, src_table, n_u: int, n_d: int, seed: int = 0x5EED, trials: int = 2):
    """The same sets by identity testing: candidate determinants (one per
    (M, M') pair and flavour) evaluated mod p at `trials` random matrices; the
    sign is made canonical (first non-zero value <= (p-1)/2) and Theta takes
    each member's sign relative to its class representative (the first member
    met); identically zero determinants (all values 0) drop their terms.
    Returns (zeta_u, zeta_d, Theta) with zeta given as the representative
    index pairs."""
    st = pair_structure(snk_table, src_table, n_u)
    res = []
    for f, (pairs, n) in enumerate(((st["pu"], n_u), (st["pd"], n_d))):
        vals = np.stack([det_modp(random_matrix_modp(seed, t, f), pairs, n) for t in range(trials)], axis=1)
        classes, cls_of, sign_of = {}, [], []
        reps, rep_sign = [], []
        for k in range(len(pairs)):
            v = [int(x) for x in vals[k]]
            nz = next((x for x in v if x), 0)
            s = 1
            if nz > (P61 - 1) // 2:
                v = [(P61 - x) % P61 for x in v]
                s = -1
            key = tuple(v)
            if not any(key):
                cls_of.append(-1)
                sign_of.append(0)
                continue
            if key not in classes:
                classes[key] = len(reps)
                reps.append(pairs[k])
                rep_sign.append(s)
            cls_of.append(classes[key])
            sign_of.append(s * rep_sign[classes[key]])
        res.append((reps, cls_of, sign_of))
    theta = {}
    for k, l, w in zip(st["t_pu"], st["t_pd"], st["t_w"]):
        ku, kd = res[0][1][k], res[1][1][l]
        if ku < 0 or kd < 0:
            continue
        key = (ku, kd)
        theta[key] = theta.get(key, 0) + int(w) * res[0][2][k] * res[1][2][l]
    theta = {k: v for k, v in theta.items() if v}
    return res[0][0], res[1][0], theta


def operator(name: str):
    """(table, n_u, n_d, scale) of a point-sink nucleus: 2H, 3He (J = 0), 4He."""
    if name == "deuteron":
        tab, fl = ops.paper_deuteron()
        scale = 1.0
    elif name == "he3":
        tab, fl = ops.paper_he3(0)
        scale = 1.0
    elif name == "he4":
        tab, fl = ops.paper_he4()
        scale = 1.0 / 96.0
    else:
        raise ValueError(name)
    n_u = sum(1 for f in fl if f == ops.U)
    return tab, n_u, len(fl) - n_u, scale
