"""Oracle-side interpolating operators (test infrastructure only).

This file is part of the independent CPU reference: only the tests, the smoke
check and the benchmark's CPU-baseline leg may import it; the GPU product path
never does.  It shares no code with the product package.

Contents, each following the passage it cites:
  * Euclidean Dirac matrices in the Dirac-Pauli basis, C = gamma4 gamma2
    (Sec. II, below Eq. 1.2) and P_pm = (1 pm gamma4)/2 (Sec. III.C).
  * Nucleon operators p_alpha = eps_abc u^a_alpha u^b_beta (C g5)_{beta eta} d^c_eta
    and the neutron with u <-> d (Eqs. 1000/1001), as integer weight tables
    over combined colour-spin indices chi = 4 * colour + spin (Sec. II.A).
  * Nucleus operators as products of nucleon operators with integer weights
    (Sec. III.C): the deuteron p(up) n(up), He-3 antisymmetrised in the two
    proton spins, He-4 p(up) p(down) n(up) n(down).

The operator "upper components" reading: every quark spin (the nucleon spin
label and the diquark spins) is restricted to the upper Dirac components
alpha in {0, 1}; with C gamma5 block diagonal in this basis that is the same
as using C gamma5 P_+ with an upper nucleon spin.
"""
from __future__ import annotations

from itertools import permutations, product
from math import factorial

import numpy as np

# ----------------------------------------------------------------------------
# Dirac algebra (Euclidean, Dirac-Pauli basis)
# ----------------------------------------------------------------------------

def pauli():
    s1 = np.array([[0, 1], [1, 0]], dtype=complex)
    s2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
    s3 = np.array([[1, 0], [0, -1]], dtype=complex)
    return s1, s2, s3


def gammas():
    """Return (g1, g2, g3, g4, g5) with g_k = [[0, -i s_k], [i s_k, 0]],
    g4 = diag(1, 1, -1, -1), g5 = g1 g2 g3 g4."""
    z = np.zeros((2, 2), dtype=complex)
    gs = []
    for s in pauli():
        gs.append(np.block([[z, -1j * s], [1j * s, z]]))
    g4 = np.diag([1, 1, -1, -1]).astype(complex)
    g5 = gs[0] @ gs[1] @ gs[2] @ g4
    return gs[0], gs[1], gs[2], g4, g5


def charge_conjugation():
    """C = gamma4 gamma2 (Sec. II)."""
    g1, g2, g3, g4, g5 = gammas()
    return g4 @ g2


def cg5():
    """C gamma5, the diquark spin matrix of Eqs. 1000/1001."""
    g5 = gammas()[4]
    return charge_conjugation() @ g5


def parity_projector(sign: int):
    """P_pm = (1 pm gamma4) / 2 (Sec. III.C)."""
    g4 = gammas()[3]
    return 0.5 * (np.eye(4) + sign * g4)


def levi_civita():
    e = np.zeros((3, 3, 3), dtype=int)
    for (a, b, c), sgn in (((0, 1, 2), 1), ((1, 2, 0), 1), ((2, 0, 1), 1),
                           ((0, 2, 1), -1), ((2, 1, 0), -1), ((1, 0, 2), -1)):
        e[a, b, c] = sgn
    return e


def integer_matrix(m: np.ndarray) -> np.ndarray:
    """Return m as an int matrix; fail if it is not real and integral."""
    if np.max(np.abs(m.imag)) > 1e-12 or np.max(np.abs(m.real - np.round(m.real))) > 1e-12:
        raise ValueError("spin matrix is not an integer matrix in this basis")
    return np.round(m.real).astype(int)


# ----------------------------------------------------------------------------
# Nucleon operators as weight tables
# ----------------------------------------------------------------------------

U, D = 0, 1


def nucleon_table(gamma: np.ndarray, spins_nucleon, spins_diquark):
    """Weight table of N_s = eps_abc q1^a_s q1^b_beta Gamma_{beta eta} q2^c_eta.

    Returns a sorted list of (s, chi1, chi2, chi3, w): slot 1 is the quark that
    carries the nucleon spin label s, slots 1 and 2 have the pair flavour q1,
    slot 3 the other flavour q2 (Eq. 1000 for the proton, Eq. 1001 for the
    neutron).  Only Gamma entries with beta, eta in `spins_diquark` are kept.
    """
    G = integer_matrix(gamma)
    eps = levi_civita()
    out = {}
    for s in spins_nucleon:
        for a, b, c in product(range(3), repeat=3):
            if eps[a, b, c] == 0:
                continue
            for be in spins_diquark:
                for et in spins_diquark:
                    w = int(eps[a, b, c] * G[be, et])
                    if w == 0:
                        continue
                    key = (s, 4 * a + s, 4 * b + be, 4 * c + et)
                    out[key] = out.get(key, 0) + w
    return sorted((k + (w,)) for k, w in out.items() if w != 0)


UPPER = (0, 1)
ALL_SPINS = (0, 1, 2, 3)


def nucleon_ops(form: str = "upper"):
    """The two block types (proton, neutron) as (pair_flavour, table) tuples."""
    if form == "upper":
        tab = nucleon_table(cg5(), UPPER, UPPER)
    elif form == "full":
        tab = nucleon_table(cg5(), ALL_SPINS, ALL_SPINS)
    else:
        raise ValueError(form)
    return [(U, tab), (D, tab)]  # op 0 = proton (u u d), op 1 = neutron (d d u)


# ----------------------------------------------------------------------------
# Nucleus operators
# ----------------------------------------------------------------------------

PROTON, NEUTRON = 0, 1


def source_terms(ops, types, spin_terms):
    """Source weight table C'(chi'_1 .. chi'_3A) of a sum of nucleon products.

    spin_terms: list of (spins tuple, integer coefficient); the nucleon types
    `types` (one per nucleon position) are the same in every product.  The
    source tuple lists each nucleon's three quarks in slot order, nucleon by
    nucleon, and its weight is the coefficient times the product of the nucleon
    table weights.  Equal tuples are merged; zeros dropped; sorted.
    """
    acc = {}
    for spins, coef in spin_terms:
        per = []
        for o, s in zip(types, spins):
            per.append([e for e in ops[o][1] if e[0] == s])
        for combo in product(*per):
            chi = tuple(x for e in combo for x in e[1:4])
            w = coef
            for e in combo:
                w *= e[4]
            acc[chi] = acc.get(chi, 0) + w
    return sorted((k, w) for k, w in acc.items() if w != 0)


def source_flavours(ops, types):
    f = []
    for o in types:
        q1 = ops[o][0]
        f += [q1, q1, 1 - q1]
    return f


def nucleus(name: str, form: str = "upper"):
    """Return the nucleus description used by the oracle.

    dict(A, ops, n_spin, chi, sink=[(types, spins, w)], src=[(chi tuple, w)],
    src_flav, scale).  Sink and source use the same spin combination.
    """
    ops = nucleon_ops(form)
    if name == "proton":
        types = (PROTON,)
        spin_terms = [((0,), 1)]
    elif name == "deuteron":
        types = (PROTON, NEUTRON)
        spin_terms = [((0, 0), 1)]
    elif name == "he3":
        types = (PROTON, PROTON, NEUTRON)
        spin_terms = [((0, 1, 0), 1), ((1, 0, 0), -1)]
    elif name == "he4":
        types = (PROTON, PROTON, NEUTRON, NEUTRON)
        spin_terms = [((0, 1, 0, 1), 1)]
    else:
        raise ValueError(name)
    sink = sorted((tuple(types), tuple(sp), w) for sp, w in spin_terms)
    src = source_terms(ops, types, spin_terms)
    n_spin = 2 if form == "upper" else 4
    chi = [c for c in range(12) if (c % 4) < n_spin]
    return dict(A=len(types), ops=ops, n_spin=n_spin, chi=chi, sink=sink, src=src,
                src_flav=source_flavours(ops, types), scale=1.0)


def quark_counts(nuc):
    nu = sum(1 for f in nuc["src_flav"] if f == U)
    return nu, len(nuc["src_flav"]) - nu


def n_raw_terms(nuc) -> int:
    """|W| |C'| n_u! n_d!: the number of Wick terms before any reduction."""
    nu, nd = quark_counts(nuc)
    return len(nuc["sink"]) * len(nuc["src"]) * factorial(nu) * factorial(nd)


def all_permutations(n):
    """Permutations of 0..n-1 in lexicographic order with their signs."""
    out = []
    for p in permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        out.append((p, -1 if inv % 2 else 1))
    return out


# ----------------------------------------------------------------------------
# Cluster operators of the Li-7 reading (Sec. III.C, Eqs. He4_op and Li7):
# nucleon types p+-, n+- with C gamma5 P+- and all four spins; source quarks
# listed flavour-grouped (u first, then d, each in nucleon-slot order) with
# the Grassmann sign of that reordering, since the nucleon types vary between
# the terms of one operator.
# ----------------------------------------------------------------------------
P_PLUS, P_MINUS, N_PLUS, N_MINUS = 0, 1, 2, 3


def pm_ops():
    """[p+, p-, n+, n-]: eps_abc q1^a_s q1^b_beta (C g5 P_pm)_{beta delta} q2^c_delta."""
    cgp = cg5() @ parity_projector(+1)
    cgm = cg5() @ parity_projector(-1)
    tp = nucleon_table(cgp, ALL_SPINS, ALL_SPINS)
    tm = nucleon_table(cgm, ALL_SPINS, ALL_SPINS)
    return [(U, tp), (U, tm), (D, tp), (D, tm)]


def _grouped_source(ops, terms):
    """Source table of sum_t coef_t prod_k N^{type_k}_{spin_k}: each product tuple
    reordered flavour-grouped (u quarks first, then d, stable) with the parity
    of that reordering folded into its weight; equal tuples merged."""
    acc = {}
    flav_out = None
    for types, spins, coef in terms:
        per = [[e for e in ops[o][1] if e[0] == s] for o, s in zip(types, spins)]
        flav = []
        for o in types:
            f = ops[o][0]
            flav += [f, f, 1 - f]
        order = [q for q in range(len(flav)) if flav[q] == U] + [q for q in range(len(flav)) if flav[q] == D]
        inv = sum(1 for a in range(len(order)) for b in range(a + 1, len(order)) if order[a] > order[b])
        sgn = -1 if inv % 2 else 1
        fo = [flav[q] for q in order]
        assert flav_out is None or fo == flav_out
        flav_out = fo
        for combo in product(*per):
            chi = [x for e in combo for x in e[1:4]]
            w = coef * sgn
            for e in combo:
                w *= e[4]
            key = tuple(chi[q] for q in order)
            acc[key] = acc.get(key, 0) + w
    return sorted((k, w) for k, w in acc.items() if w != 0), flav_out


def _cluster(ops, terms, scale):
    sink = sorted((tuple(t), tuple(s), w) for t, s, w in terms)
    src, flav = _grouped_source(ops, terms)
    return dict(A=len(terms[0][0]), ops=ops, n_spin=4, chi=list(range(12)), sink=sink, src=src, src_flav=flav,
                scale=scale)


def he4_cluster():
    """O_He4 = (chibar eta - chi etabar)/sqrt2 with p+, n+ (Eq. He4_op): spin
    patterns chi, chibar and isospin patterns eta, etabar over four nucleons;
    integer weights chibar_s eta_i - chi_s etabar_i and scale 1/96 for
    sink x source."""
    pats = [(0, 1, 0, 1), (1, 0, 1, 0), (0, 1, 1, 0), (1, 0, 0, 1), (0, 0, 1, 1), (1, 1, 0, 0)]
    c = [1, 1, -1, -1, 0, 0]          # chi, times 1/2
    cb = [1, 1, 1, 1, -2, -2]         # chibar, times 1/sqrt(12)
    iso = [tuple(P_PLUS if x == 0 else N_PLUS for x in p) for p in pats]   # up -> p, down -> n
    terms = []
    for a, s in enumerate(pats):
        for b, t in enumerate(iso):
            w = cb[a] * c[b] - c[a] * cb[b]
            if w:
                terms.append((t, s, w))
    return _cluster(pm_ops(), terms, 1.0 / 96.0)


def triton_cluster(J: int = 0):
    """n_-^T C g5 p_+ n_+^J (the three-nucleon factor of Eq. Li7)."""
    G = integer_matrix(cg5())
    terms = [((N_MINUS, P_PLUS, N_PLUS), (a, b, J), int(G[a, b])) for a in range(4) for b in range(4) if G[a, b]]
    return _cluster(pm_ops(), terms, 1.0)


# ----------------------------------------------------------------------------
# Point-sink operators of the determinant algorithm (Sec. III.C, "Implementation
# of the proposed algorithm": Eqs. NP_op, He3_op, He4_op).  Each is a weight
# table over flavour-grouped quark index tuples (u quarks first, then d, each
# in nucleon-slot order, the Grassmann sign of that regrouping folded into the
# weight), the same form for sink and source.  Pinned by the operator term
# counts of the paper's determinant table (2H 356, 3He 1026 per spin
# component, 4He 2716), which count the flavour-ordered index lists with a
# non-zero antisymmetrised coefficient.
#
# Readings: the 2H and 4He operators are built from the nucleons of Eqs.
# 1000/1001 (all four spins, no projection; 4He with the spin and isospin
# wave functions chi, chibar, eta, etabar of Eq. He4_op).  The projected
# nucleons p+-, n+- of the 3He operator carry C gamma5 P with the paper's
# P+- = (1 -+ gamma4)/2 of this Dirac-Pauli basis (the paper's gamma4 has the
# opposite sign): with (1 +- gamma4)/2 the 3He count would be 744, not 1026;
# the 2H and 4He counts are the same under either sign.
# ----------------------------------------------------------------------------

def plain_nucleons():
    """[proton, neutron] of Eqs. 1000/1001 with all four spins."""
    tab = nucleon_table(cg5(), ALL_SPINS, ALL_SPINS)
    return [(U, tab), (D, tab)]


def paper_projector(sign: int) -> np.ndarray:
    """The paper's P_pm in this basis: (1 -+ gamma4)/2 (see the reading above)."""
    return parity_projector(-sign)


def grouped_operator(ops, terms):
    """(table, flavours) of sum_t coef_t prod_k N^{type_k}_{spin_k}, flavour-grouped."""
    return _grouped_source(ops, terms)


def paper_deuteron():
    """O_2H = n^T (C gamma5 P+) p (Eq. NP_op), nucleon spins contracted."""
    G = integer_matrix(cg5() @ paper_projector(+1))
    terms = [((NEUTRON, PROTON), (a, b), int(G[a, b])) for a in range(4) for b in range(4) if G[a, b]]
    return grouped_operator(plain_nucleons(), terms)


def paper_he3(J: int = 0):
    """O_3He^J = p_-^T (C gamma5) n_+ p_+^J (Eq. He3_op)."""
    cgp = cg5() @ paper_projector(+1)
    cgm = cg5() @ paper_projector(-1)
    ops = [(U, nucleon_table(cgm, ALL_SPINS, ALL_SPINS)),   # p-
           (D, nucleon_table(cgp, ALL_SPINS, ALL_SPINS)),   # n+
           (U, nucleon_table(cgp, ALL_SPINS, ALL_SPINS))]   # p+
    G = integer_matrix(cg5())
    terms = [((0, 1, 2), (a, b, J), int(G[a, b])) for a in range(4) for b in range(4) if G[a, b]]
    return grouped_operator(ops, terms)


def paper_he4():
    """O_4He = (chibar eta - chi etabar)/sqrt2 (Eq. He4_op) with the plain p, n:
    integer weights chibar_s eta_i - chi_s etabar_i (overall factor 1/(2 sqrt24)
    per operator, 1/96 for sink x source)."""
    pats = [(0, 1, 0, 1), (1, 0, 1, 0), (0, 1, 1, 0), (1, 0, 0, 1), (0, 0, 1, 1), (1, 1, 0, 0)]
    c = [1, 1, -1, -1, 0, 0]
    cb = [1, 1, 1, 1, -2, -2]
    iso = [tuple(PROTON if x == 0 else NEUTRON for x in p) for p in pats]
    terms = [(iso[b], s, cb[a] * c[b] - c[a] * cb[b]) for a, s in enumerate(pats) for b in range(6)
             if cb[a] * c[b] - c[a] * cb[b]]
    return grouped_operator(plain_nucleons(), terms)


def paper_point_nucleus(name: str):
    """Plane-wave description (for the block oracle) of the same operators:
    dict as `nucleus` with the grouped source and sink = the nucleon products."""
    if name == "deuteron":
        G = integer_matrix(cg5() @ paper_projector(+1))
        ops = plain_nucleons()
        terms = [((NEUTRON, PROTON), (a, b), int(G[a, b])) for a in range(4) for b in range(4) if G[a, b]]
    elif name == "he3":
        cgp = cg5() @ paper_projector(+1)
        cgm = cg5() @ paper_projector(-1)
        ops = [(U, nucleon_table(cgm, ALL_SPINS, ALL_SPINS)), (D, nucleon_table(cgp, ALL_SPINS, ALL_SPINS)),
               (U, nucleon_table(cgp, ALL_SPINS, ALL_SPINS))]
        G = integer_matrix(cg5())
        terms = [((0, 1, 2), (a, b, 0), int(G[a, b])) for a in range(4) for b in range(4) if G[a, b]]
    else:
        raise ValueError(name)
    return _cluster(ops, terms, 1.0)


def antisymmetrised(table, n_u: int):
    """C^[M] over flavour-ordered index lists M = (sorted u indices, sorted d indices):
    sum over the orderings of each flavour's indices with the sign of the ordering;
    zero entries dropped (Sec. III.C, method A)."""
    acc = {}
    for chi, w in table:
        u, d = list(chi[:n_u]), list(chi[n_u:])
        if len(set(u)) < len(u) or len(set(d)) < len(d):
            continue
        key = (tuple(sorted(u)), tuple(sorted(d)))
        acc[key] = acc.get(key, 0) + w * _perm_sign(u) * _perm_sign(d)
    return {k: v for k, v in acc.items() if v != 0}


def _perm_sign(x) -> int:
    inv = sum(1 for i in range(len(x)) for j in range(i + 1, len(x)) if x[i] > x[j])
    return -1 if inv % 2 else 1


def deuteron_basis():
    """Three 2H operators for a correlation matrix (Eqs. E1-E3): n^T (C g5 P+) p,
    n^T (C g5 P-) p and n+^T (C g5 P+) p+ (nucleons projected with the paper's P+)."""
    out = []
    for gpar, npar in ((+1, 0), (-1, 0), (+1, +1)):
        G = integer_matrix(cg5() @ paper_projector(gpar))
        if npar:
            tab = nucleon_table(cg5() @ paper_projector(npar), ALL_SPINS, ALL_SPINS)
            nucs = [(U, tab), (D, tab)]
        else:
            nucs = plain_nucleons()
        terms = [((NEUTRON, PROTON), (a, b), int(G[a, b])) for a in range(4) for b in range(4) if G[a, b]]
        out.append(grouped_operator(nucs, terms))
    return out


# ----------------------------------------------------------------------------
# Plane-wave operators for the correlation matrix and the 2H operator of Eq. NP_op
# (block form, each nucleon projected to zero momentum on its own).
# ----------------------------------------------------------------------------
def nucleus_from_terms(name: str, types, spin_terms, form: str = "upper", ops=None, scale: float = 1.0):
    """A nucleus sum_t coef_t prod_k N^{types_k}_{spins_k} (the same combination at sink and source)."""
    ops = nucleon_ops(form) if ops is None else ops
    n_spin = 2 if form == "upper" else 4
    return dict(A=len(types), ops=ops, n_spin=n_spin, chi=[c for c in range(12) if (c % 4) < n_spin],
                sink=sorted((tuple(types), tuple(sp), w) for sp, w in spin_terms),
                src=source_terms(ops, tuple(types), spin_terms), src_flav=source_flavours(ops, tuple(types)),
                scale=scale, name=name)


def deuteron_pw_basis():
    """Three plane-wave deuteron operators with upper-spin nucleons, one quark content, spin
    projection 0: p(up) n(down), p(down) n(up), and their sum."""
    types = (PROTON, NEUTRON)
    return [nucleus_from_terms("pn ud", types, [((0, 1), 1)]),
            nucleus_from_terms("pn du", types, [((1, 0), 1)]),
            nucleus_from_terms("pn ud+du", types, [((0, 1), 1), ((1, 0), 1)])]


def deuteron_np_planewave():
    """Eq. NP_op with a plane-wave sink: n^T (C gamma5 P+) p, plain nucleons of Eqs. 1000/1001 with all
    four spins, the paper's P+ (paper_projector)."""
    G = integer_matrix(cg5() @ paper_projector(+1))
    terms = [((a, b), int(G[a, b])) for a in range(4) for b in range(4) if G[a, b]]
    return nucleus_from_terms("2H NP", (NEUTRON, PROTON), terms, form="full")
