"""Integer operator weight tables for the C ABI (host side, no GPU needed).

Builds, from the paper's definitions, the tables `wick_build_blocks` and
`wick_reduce_terms` take:

* nucleon operators p_s = eps_abc u^a_s u^b_beta Gamma_{beta eta} d^c_eta and
  n_s with u <-> d (Eqs. 1000/1001), Gamma = C gamma5 with C = gamma4 gamma2
  (Sec. II) in the Dirac-Pauli basis, optionally times P_pm = (1 pm gamma4)/2
  (Sec. III.C);
* nucleus operators as integer combinations of products of nucleon operators
  (Sec. III.C): the deuteron p(up) n(up), He-3 antisymmetrised in the proton
  spins, He-4 p(up) p(down) n(up) n(down).

"Upper" form: all quark spins restricted to the upper Dirac components
(alpha in {0, 1}); the block layout then keeps the 6 source indices with an
upper spin and 2 nucleon spin labels.

Every table is canonical (sorted, duplicates merged, zeros dropped), so the
raw-term order of the reduction -- and hence the reduced table byte for byte --
is a function of the operator alone.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import permutations
from math import factorial

import numpy as np

U, D = 0, 1
PROTON, NEUTRON = 0, 1

_SX = np.array([[0, 1], [1, 0]], dtype=complex)
_SY = np.array([[0, -1j], [1j, 0]], dtype=complex)
_SZ = np.array([[1, 0], [0, -1]], dtype=complex)
_I2 = np.eye(2, dtype=complex)


def dirac_matrices():
    """(g1, g2, g3, g4, g5) in the Dirac-Pauli basis: g_k = sigma_y (x) sigma_k,
    g4 = sigma_z (x) 1, g5 = g1 g2 g3 g4."""
    g = [np.kron(_SY, s) for s in (_SX, _SY, _SZ)]
    g4 = np.kron(_SZ, _I2)
    return g[0], g[1], g[2], g4, g[0] @ g[1] @ g[2] @ g4


def diquark_matrix(parity: int = 0) -> np.ndarray:
    """C gamma5 (parity 0) or C gamma5 P_pm (parity +1 / -1) as an int matrix."""
    g1, g2, g3, g4, g5 = dirac_matrices()
    m = g4 @ g2 @ g5
    if parity:
        m = m @ (0.5 * (np.eye(4) + parity * g4))
    r = np.round(m.real)
    if np.abs(m - r).max() > 1e-12:
        raise ValueError("diquark matrix is not integral in this basis")
    return r.astype(np.int64)


def _eps_entries():
    out = []
    for p in permutations(range(3)):
        inv = sum(p[i] > p[j] for i in range(3) for j in range(i + 1, 3))
        out.append((p, -1 if inv & 1 else 1))
    return out


@dataclass
class NucleonOp:
    flav_pair: int                                  # flavour of slots 1, 2
    entries: list = field(default_factory=list)     # (s, chi1, chi2, chi3, w), canonical


def nucleon_op(flav_pair: int, gamma: np.ndarray, nucleon_spins, quark_spins) -> NucleonOp:
    acc = {}
    for s in nucleon_spins:
        for (a, b, c), sg in _eps_entries():
            for be in quark_spins:
                for et in quark_spins:
                    w = sg * int(gamma[be, et])
                    if w:
                        k = (s, 4 * a + s, 4 * b + be, 4 * c + et)
                        acc[k] = acc.get(k, 0) + w
    return NucleonOp(flav_pair, sorted(k + (w,) for k, w in acc.items() if w))


@dataclass
class Nucleus:
    name: str
    A: int
    ops: list          # NucleonOp per block type
    n_spin: int
    chi: list          # source indices kept in the block layout
    sink: list         # (types tuple, spins tuple, w)
    src: list          # (chi' tuple of length 3A, w)
    src_flav: list
    scale: float = 1.0

    @property
    def quark_counts(self):
        nu = sum(1 for f in self.src_flav if f == U)
        return nu, len(self.src_flav) - nu

    @property
    def n_raw(self) -> int:
        nu, nd = self.quark_counts
        return len(self.sink) * len(self.src) * factorial(nu) * factorial(nd)

    @property
    def n_blk(self) -> int:
        return len(self.ops) * self.n_spin * len(self.chi) ** 3


def _source_table(ops, types, spin_combos):
    acc = {}
    for spins, coef in spin_combos:
        rows = [[e for e in ops[o].entries if e[0] == s] for o, s in zip(types, spins)]
        # cartesian product of the nucleons' entries
        idx = [0] * len(rows)
        while True:
            chi, w = [], coef
            for r, i in zip(rows, idx):
                chi += list(r[i][1:4])
                w *= r[i][4]
            acc[tuple(chi)] = acc.get(tuple(chi), 0) + w
            k = len(rows) - 1
            while k >= 0:
                idx[k] += 1
                if idx[k] < len(rows[k]):
                    break
                idx[k] = 0
                k -= 1
            if k < 0:
                break
    return sorted((c, w) for c, w in acc.items() if w)


_NUCLEI = {
    "proton": ((PROTON,), [((0,), 1)]),
    "deuteron": ((PROTON, NEUTRON), [((0, 0), 1)]),
    "he3": ((PROTON, PROTON, NEUTRON), [((0, 1, 0), 1), ((1, 0, 0), -1)]),
    "he4": ((PROTON, PROTON, NEUTRON, NEUTRON), [((0, 1, 0, 1), 1)]),
}


def standard_ops(form: str = "upper"):
    G = diquark_matrix()
    if form == "upper":
        sp = (0, 1)
    elif form == "full":
        sp = (0, 1, 2, 3)
    else:
        raise ValueError(form)
    return [nucleon_op(U, G, sp, sp), nucleon_op(D, G, sp, sp)]


def nucleus(name: str, form: str = "upper") -> Nucleus:
    """Standard nucleus operators (same spin combination at sink and source)."""
    types, combos = _NUCLEI[name]
    ops = standard_ops(form)
    n_spin = 2 if form == "upper" else 4
    chi = [c for c in range(12) if c % 4 < n_spin]
    sink = sorted((tuple(types), tuple(s), w) for s, w in combos)
    src = _source_table(ops, types, combos)
    flav = []
    for o in types:
        f = ops[o].flav_pair
        flav += [f, f, 1 - f]
    return Nucleus(name, len(types), ops, n_spin, chi, sink, src, flav)


# ---------------------------------------------------------------------------
# Li-7 clusters (Sec. III.C, Eqs. He4_op and Li7): block types p+, p-, n+, n-
# (C gamma5 P_pm, all four spins, every source index).  The isospin wave
# function moves p and n between nucleon positions, so the source quarks of
# every term are stored flavour-grouped (u first, then d, each in nucleon-slot
# order) and the parity of that reordering is folded into the term's weight.
# ---------------------------------------------------------------------------
P_PLUS, P_MINUS, N_PLUS, N_MINUS = 0, 1, 2, 3


def pm_ops():
    sp = (0, 1, 2, 3)
    gp, gm = diquark_matrix(+1), diquark_matrix(-1)
    return [nucleon_op(U, gp, sp, sp), nucleon_op(U, gm, sp, sp), nucleon_op(D, gp, sp, sp),
            nucleon_op(D, gm, sp, sp)]


def _flavour_grouped(ops, terms):
    acc = {}
    flav_ref = None
    for types, spins, coef in terms:
        flav = []
        for o in types:
            f = ops[o].flav_pair
            flav += [f, f, 1 - f]
        perm = sorted(range(len(flav)), key=lambda q: (flav[q], q))      # stable: u first
        parity = 1
        seen = [False] * len(perm)
        for start in range(len(perm)):                                  # parity from the cycle lengths
            if not seen[start]:
                n, q = 0, start
                while not seen[q]:
                    seen[q] = True
                    q = perm[q]
                    n += 1
                if n % 2 == 0:
                    parity = -parity
        grouped = [flav[q] for q in perm]
        if flav_ref is not None and grouped != flav_ref:
            raise ValueError("terms of one operator must carry the same quarks")
        flav_ref = grouped
        for chi, w in _source_table(ops, types, [(spins, coef * parity)]):
            key = tuple(chi[q] for q in perm)
            acc[key] = acc.get(key, 0) + w
    return sorted((c, w) for c, w in acc.items() if w), flav_ref


def cluster(name: str) -> Nucleus:
    """'he4_cluster': (chibar eta - chi etabar)/sqrt2 with p+, n+ and up/down
    spins (scale 1/96 for sink x source);  'triton': n_-^T C g5 p_+ n_+^(J=up)."""
    ops = pm_ops()
    if name == "he4_cluster":
        pats = [(0, 1, 0, 1), (1, 0, 1, 0), (0, 1, 1, 0), (1, 0, 0, 1), (0, 0, 1, 1), (1, 1, 0, 0)]
        chi_w = [1, 1, -1, -1, 0, 0]       # times 1/2
        chibar_w = [1, 1, 1, 1, -2, -2]    # times 1/sqrt(12)
        terms = []
        for a, spins in enumerate(pats):
            for b, iso in enumerate(pats):
                w = chibar_w[a] * chi_w[b] - chi_w[a] * chibar_w[b]
                if w:
                    terms.append((tuple(P_PLUS if x == 0 else N_PLUS for x in iso), spins, w))
        scale = 1.0 / 96.0
    elif name == "triton":
        G = diquark_matrix()
        terms = [((N_MINUS, P_PLUS, N_PLUS), (a, b, 0), int(G[a, b])) for a in range(4) for b in range(4)
                 if G[a, b]]
        scale = 1.0
    else:
        raise ValueError(name)
    src, flav = _flavour_grouped(ops, terms)
    sink = sorted((tuple(t), tuple(s), w) for t, s, w in terms)
    return Nucleus(name, len(terms[0][0]), ops, 4, list(range(12)), sink, src, flav, scale)


# ---------------------------------------------------------------------------
# Point-sink operators of the determinant algorithm (Sec. III.C, Eqs. NP_op,
# He3_op, He4_op) for wick_det_reduce: flavour-grouped quark index tuples
# (u quarks first, then d, each in nucleon-slot order, regrouping parity in
# the weight).  2H and 4He use the nucleons of Eqs. 1000/1001 with all spins;
# the projected nucleons of 3He take the paper's P+- = (1 -+ gamma4)/2 of this
# basis (its gamma4 has the opposite sign), with which the operators have the
# 356 / 1026 / 2716 terms of the paper's determinant table.
# ---------------------------------------------------------------------------
@dataclass
class QuarkOperator:
    name: str
    n_u: int
    n_d: int
    chi: np.ndarray      # int8 [n_terms][n_u + n_d]
    w: np.ndarray        # int64 [n_terms]
    scale: float = 1.0   # overall factor of sink x source


def point_operator(name: str) -> QuarkOperator:
    sp = (0, 1, 2, 3)
    G = diquark_matrix()
    plain = [nucleon_op(U, G, sp, sp), nucleon_op(D, G, sp, sp)]
    scale = 1.0
    if name == "deuteron":                                 # n^T (C g5 P+) p
        Gp = diquark_matrix(-1)
        ops, terms = plain, [((NEUTRON, PROTON), (a, b), int(Gp[a, b])) for a in range(4) for b in range(4)
                             if Gp[a, b]]
    elif name == "he3":                                    # p-^T (C g5) n+ p+^(J=0)
        ops = [nucleon_op(U, diquark_matrix(+1), sp, sp), nucleon_op(D, diquark_matrix(-1), sp, sp),
               nucleon_op(U, diquark_matrix(-1), sp, sp)]
        terms = [((0, 1, 2), (a, b, 0), int(G[a, b])) for a in range(4) for b in range(4) if G[a, b]]
    elif name == "he4":                                    # (chibar eta - chi etabar)/sqrt2, plain p, n
        pats = [(0, 1, 0, 1), (1, 0, 1, 0), (0, 1, 1, 0), (1, 0, 0, 1), (0, 0, 1, 1), (1, 1, 0, 0)]
        chi_w = [1, 1, -1, -1, 0, 0]
        chibar_w = [1, 1, 1, 1, -2, -2]
        ops, terms = plain, []
        for a, spins in enumerate(pats):
            for b, iso in enumerate(pats):
                w = chibar_w[a] * chi_w[b] - chi_w[a] * chibar_w[b]
                if w:
                    terms.append((tuple(PROTON if x == 0 else NEUTRON for x in iso), spins, w))
        scale = 1.0 / 96.0
    else:
        raise ValueError(name)
    table, flav = _flavour_grouped(ops, terms)
    n_u = sum(1 for f in flav if f == U)
    chi = np.array([c for c, _ in table], dtype=np.int8).reshape(len(table), len(flav))
    w = np.array([x for _, x in table], dtype=np.int64)
    return QuarkOperator(name, n_u, len(flav) - n_u, chi, w, scale)


def deuteron_basis():
    """[n^T (C g5 P+) p, n^T (C g5 P-) p, n+^T (C g5 P+) p+]: three 2H point operators
    (the paper's P+-) for a correlation matrix (Eqs. E1-E3)."""
    sp = (0, 1, 2, 3)
    out = []
    for name, gpar, npar in (("2H P+", -1, 0), ("2H P-", +1, 0), ("2H P+ projected", -1, -1)):
        Gp = diquark_matrix(gpar)
        nuc_gamma = diquark_matrix(npar) if npar else diquark_matrix()
        ops = [nucleon_op(U, nuc_gamma, sp, sp), nucleon_op(D, nuc_gamma, sp, sp)]
        terms = [((NEUTRON, PROTON), (a, b), int(Gp[a, b])) for a in range(4) for b in range(4) if Gp[a, b]]
        table, flav = _flavour_grouped(ops, terms)
        n_u = sum(1 for f in flav if f == U)
        chi = np.array([c for c, _ in table], dtype=np.int8).reshape(len(table), len(flav))
        w = np.array([x for _, x in table], dtype=np.int64)
        out.append(QuarkOperator(name, n_u, len(flav) - n_u, chi, w, 1.0))
    return out


# ---------------------------------------------------------------------------
# Plane-wave operators given as nucleon products: a basis for a correlation
# matrix (Eqs. E1-E3) and the 2H operator of Eq. NP_op with a plane-wave sink.
# ---------------------------------------------------------------------------
def nucleus_from_terms(name: str, types, combos, form: str = "upper", scale: float = 1.0) -> Nucleus:
    """sum_t coef_t prod_k N^{types_k}_{spins_k}, the same combination at sink and source; combos =
    [(spins tuple, coef)]."""
    ops = standard_ops(form)
    n_spin = 2 if form == "upper" else 4
    chi = [c for c in range(12) if c % 4 < n_spin]
    flav = []
    for o in types:
        f = ops[o].flav_pair
        flav += [f, f, 1 - f]
    sink = sorted((tuple(types), tuple(s), w) for s, w in combos)
    return Nucleus(name, len(types), ops, n_spin, chi, sink, _source_table(ops, tuple(types), combos), flav, scale)


def deuteron_pw_basis():
    """Three plane-wave deuteron operators with upper-spin nucleons, one quark content and spin
    projection 0: p(up) n(down), p(down) n(up) and their sum (the triplet) -- a 3 x 3 correlation
    matrix whose elements share terms (the third operator contains the first two)."""
    t = (PROTON, NEUTRON)
    return [nucleus_from_terms("pn ud", t, [((0, 1), 1)]),
            nucleus_from_terms("pn du", t, [((1, 0), 1)]),
            nucleus_from_terms("pn ud+du", t, [((0, 1), 1), ((1, 0), 1)])]


def deuteron_np() -> Nucleus:
    """Eq. NP_op with a plane-wave sink: n^T (C gamma5 P+) p with the plain nucleons of Eqs. 1000/1001
    (all four spins) and the paper's P+ = (1 - gamma4)/2 of this basis."""
    G = diquark_matrix(-1)
    combos = [((a, b), int(G[a, b])) for a in range(4) for b in range(4) if G[a, b]]
    return nucleus_from_terms("2H NP", (NEUTRON, PROTON), combos, form="full")
