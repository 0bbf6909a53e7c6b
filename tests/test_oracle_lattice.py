"""Pins of the oracle's lattice algebra against what the paper fixes.

Sec. 3.3: D3Q19 weights and the isotropy conditions Eqs. (w0)-(w4) with
C4' = 0, C4 = C2^2, c_s^2 = C2 = 1/3.  Sec. 3.4: Table 1 basis, weighted
orthogonality Eq. (orthogonality) with q = a, the backward relation
Eq. (orthogonality_backward), and the hydrodynamic moments
Eqs. (hmodes_beg)-(hmodes_end).  Exact rational arithmetic where possible.
"""
import itertools
import os
from fractions import Fraction as Fr

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _frac_tables(ora):
    c, a, e, w, opp = ora.tables()
    af = []
    for i in range(19):
        s = int((c[i] ** 2).sum())
        af.append({0: Fr(1, 3), 1: Fr(1, 18), 2: Fr(1, 36)}[s])
    # the double weights are the nearest doubles to the paper's rationals
    assert np.allclose(a, [float(x) for x in af], rtol=0, atol=1e-17)
    ei = np.rint(e).astype(np.int64)
    assert np.array_equal(ei, e), "basis entries are integers for b = h = 1"
    return c, af, ei, w, opp


def test_velocity_set(ora):
    c, a, e, w, opp = ora.tables()
    assert len({tuple(v) for v in c}) == 19
    speeds = sorted(int((v ** 2).sum()) for v in c)
    assert speeds.count(0) == 1 and speeds.count(1) == 6 and speeds.count(2) == 12
    for i in range(19):
        assert np.array_equal(c[opp[i]], -c[i])
    # the project's ordering convention
    assert c[1].tolist() == [1, 0, 0] and c[2].tolist() == [-1, 0, 0]
    assert c[5].tolist() == [0, 0, 1] and c[6].tolist() == [0, 0, -1]
    assert c[7].tolist() == [1, 1, 0] and c[10].tolist() == [-1, -1, 0]
    assert c[11].tolist() == [0, 1, 1] and c[14].tolist() == [0, -1, -1]
    assert c[15].tolist() == [1, 0, 1] and c[16].tolist() == [1, 0, -1]
    assert c[17].tolist() == [-1, 0, 1] and c[18].tolist() == [-1, 0, -1]


def test_isotropy_exact(ora):
    """Eqs. (w0)-(w4): sum a = 1, odd moments 0, second moment C2 delta with
    C2 = c_s^2 = 1/3, fourth moment with C4' = 0 and C4 = C2^2 = 1/9."""
    c, a, e, w, opp = _frac_tables(ora)
    assert sum(a) == 1
    C2, C4 = Fr(1, 3), Fr(1, 9)
    for al in range(3):
        assert sum(a[i] * c[i][al] for i in range(19)) == 0
    for al, be in itertools.product(range(3), repeat=2):
        s = sum(a[i] * c[i][al] * c[i][be] for i in range(19))
        assert s == (C2 if al == be else 0)
    for al, be, ga in itertools.product(range(3), repeat=3):
        assert sum(a[i] * c[i][al] * c[i][be] * c[i][ga] for i in range(19)) == 0
    d = lambda x, y: 1 if x == y else 0
    for al, be, ga, de in itertools.product(range(3), repeat=4):
        s = sum(a[i] * c[i][al] * c[i][be] * c[i][ga] * c[i][de] for i in range(19))
        want = C4 * (d(al, be) * d(ga, de) + d(al, ga) * d(be, de) + d(al, de) * d(be, ga))
        assert s == want  # C4' = 0


def test_table1_orthogonality_exact(ora):
    """Eq. (orthogonality) with q = a: sum_i a_i e_ki e_li = w_k delta_kl, and
    w_k equal to the values printed in Table 1."""
    c, a, e, w, opp = _frac_tables(ora)
    printed = {}
    with open(os.path.join(GOLD, "table1_basis.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, poly, wk = line.split()
            printed[int(k)] = Fr(wk)
    for k in range(19):
        for l in range(19):
            s = sum(a[i] * int(e[k][i]) * int(e[l][i]) for i in range(19))
            if k == l:
                assert s == printed[k], (k, s, printed[k])
            else:
                assert s == 0, (k, l, s)
    assert np.allclose(w, [float(printed[k]) for k in range(19)], rtol=1e-15)


def test_backward_orthogonality_exact(ora):
    """Eq. (orthogonality_backward): sum_k e_ki e_kj / w_k = delta_ij / a_i."""
    c, a, e, w, opp = _frac_tables(ora)
    wf = [sum(a[i] * int(e[k][i]) ** 2 for i in range(19)) for k in range(19)]
    for i in range(19):
        for j in range(19):
            s = sum(Fr(int(e[k][i]) * int(e[k][j])) / wf[k] for k in range(19))
            assert s == (1 / a[i] if i == j else 0)


def test_hydrodynamic_moments_relations(ora):
    """Eqs. (hmodes_beg)-(hmodes_end): rho = m0, j = m1..3, pi from m0, m4..m9.
    moments() sums over populations directly; modes() uses Table 1."""
    p = ora.make_params((3, 4, 5))
    rng = np.random.default_rng(3)
    pops = rng.uniform(0.01, 0.3, size=(19, 5, 4, 3))
    rho, j, pi = ora.moments(p, pops)
    m = ora.modes(p, pops)
    assert np.allclose(rho, m[0], rtol=1e-14)
    for d in range(3):
        assert np.allclose(j[d], m[1 + d], rtol=1e-13, atol=1e-15)
    xx = (m[0] + m[4] + m[5]) / 3
    yy = (2 * m[0] + 2 * m[4] - m[5] + 3 * m[6]) / 6
    zz = (2 * m[0] + 2 * m[4] - m[5] - 3 * m[6]) / 6
    assert np.allclose(pi[0], xx, rtol=1e-13)
    assert np.allclose(pi[1], yy, rtol=1e-13)
    assert np.allclose(pi[2], zz, rtol=1e-13)
    assert np.allclose(pi[3], m[7], rtol=1e-12, atol=1e-15)
    assert np.allclose(pi[4], m[8], rtol=1e-12, atol=1e-15)
    assert np.allclose(pi[5], m[9], rtol=1e-12, atol=1e-15)
