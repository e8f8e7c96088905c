"""Pins for oracle/butcher.py: order conditions, textbook tables, Pade
stability function, LDU identities and the paper's printed condition numbers
(Table 2, Table 4)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import butcher as bt

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_kappa_tables.json")))


@pytest.mark.parametrize("s", range(1, 8))
def test_radau_order_conditions(s):
    # Table 1: Radau IIA has order 2s-1: B(2s-1) and C(s) simplifying assumptions
    A, b, c = bt.radau_iia(s)
    for q in range(1, 2 * s):
        assert abs(b @ c ** (q - 1) - 1.0 / q) < 1e-13
    for q in range(1, s + 1):
        assert np.max(np.abs(A @ c ** (q - 1) - c ** q / q)) < 1e-13
    # stiffly accurate: b is the last row, c_s = 1
    assert np.max(np.abs(A[-1] - b)) < 1e-14
    assert c[-1] == 1.0
    # order is exactly 2s-1, not 2s
    assert abs(b @ c ** (2 * s - 1) - 1.0 / (2 * s)) > 1e-11


def test_radau_s2_textbook():
    A, b, c = bt.radau_iia(2)
    assert np.allclose(c, [1 / 3, 1.0], atol=1e-15)
    assert np.allclose(A, [[5 / 12, -1 / 12], [3 / 4, 1 / 4]], atol=1e-15)
    assert np.allclose(b, [3 / 4, 1 / 4], atol=1e-15)


def test_radau_s3_nodes():
    # c = (4 - sqrt6)/10, (4 + sqrt6)/10, 1
    _, _, c = bt.radau_iia(3)
    r6 = math.sqrt(6.0)
    assert np.allclose(c, [(4 - r6) / 10, (4 + r6) / 10, 1.0], atol=1e-15)


def _pade(k, j, z):
    num = sum(math.factorial(k + j - i) * math.factorial(k)
              / (math.factorial(k + j) * math.factorial(i) * math.factorial(k - i)) * z ** i
              for i in range(k + 1))
    den = sum(math.factorial(k + j - i) * math.factorial(j)
              / (math.factorial(k + j) * math.factorial(i) * math.factorial(j - i)) * (-z) ** i
              for i in range(j + 1))
    return num / den


@pytest.mark.parametrize("s", range(1, 8))
def test_radau_stability_is_pade(s):
    # Radau IIA: R(z) is the (s-1, s) Pade approximant of e^z; L-stable
    A, b, _ = bt.radau_iia(s)
    for z in [-0.3, -2.0, -17.0, 0.4 + 1.3j, -5 + 8j]:
        R = bt.stability_function(A, b, z)
        assert abs(R - _pade(s - 1, s, z)) < 1e-12 * max(1.0, abs(R))
    assert abs(bt.stability_function(A, b, -1e9)) < 1e-8


@pytest.mark.parametrize("s", range(2, 6))
def test_lobatto_iiic(s):
    A, b, c = bt.lobatto_iiic(s)
    for q in range(1, 2 * s - 1):            # order 2s-2
        assert abs(b @ c ** (q - 1) - 1.0 / q) < 1e-13
    assert np.allclose(A[:, 0], b[0])
    for q in range(1, s):                    # C(s-1)
        assert np.max(np.abs(A @ c ** (q - 1) - c ** q / q)) < 1e-13
    # L-stable: (s-2, s) Pade
    for z in [-0.7, -9.0, 1j]:
        R = bt.stability_function(A, b, z)
        assert abs(R - _pade(s - 2, s, z)) < 1e-12


def test_lobatto_s2_textbook():
    A, _, _ = bt.lobatto_iiic(2)
    assert np.allclose(A, [[0.5, -0.5], [0.5, 0.5]], atol=1e-15)
    _, D, _ = bt.ldu(A)
    assert np.allclose(np.diag(D), [0.5, 1.0])


@pytest.mark.parametrize("s", range(2, 8))
def test_ldu_identities(s):
    A, _, _ = bt.radau_iia(s)
    Lm, D, Um = bt.ldu(A)
    assert np.max(np.abs(Lm @ D @ Um - A)) < 1e-14
    assert np.allclose(np.diag(Lm), 1) and np.allclose(np.diag(Um), 1)
    assert np.allclose(np.triu(Lm, 1), 0) and np.allclose(np.tril(Um, -1), 0)
    # product of the first k pivots = k-th leading principal minor
    d = np.diag(D)
    for k in range(1, s + 1):
        assert abs(np.prod(d[:k]) - np.linalg.det(A[:k, :k])) < 1e-13
    # all pivots positive for Radau IIA (diagonal blocks M + h d_jj F SPD)
    assert np.all(d > 0)
    # Section 4.1: (LD)^{-1} A = U and A (DU)^{-1} = L, eigenvalues all one
    assert np.allclose(np.linalg.solve(bt.atilde(A, "LD"), A), Um, atol=1e-13)
    assert np.allclose(A @ np.linalg.inv(bt.atilde(A, "DU")), Lm, atol=1e-13)


def test_ldu_s2_values():
    A, _, _ = bt.radau_iia(2)
    Lm, D, Um = bt.ldu(A)
    assert abs(Lm[1, 0] - 9 / 5) < 1e-14
    assert np.allclose(np.diag(D), [5 / 12, 2 / 5], atol=1e-15)
    assert abs(Um[0, 1] + 1 / 5) < 1e-14


def test_ldu_zero_pivot():
    with pytest.raises(ZeroDivisionError):
        bt.ldu(np.array([[0.0, 1.0], [1.0, 0.0]]))


def test_table4_kappa_LD_limit():
    """Table 4: kappa of the left-preconditioned system with P_LD.  Its
    s x s limit kappa((LD)^{-1} A) = kappa(U) (Section 4.1) lies within 5%
    below the printed values, for Radau IIA and Lobatto IIIC."""
    g = GOLD["table4_left_optimized_gsl"]
    for s, k1d, k2d in zip(g["radau_s"], g["radau_LD_1D"], g["radau_LD_2D"]):
        A, _, _ = bt.radau_iia(s)
        _, _, Um = bt.ldu(A)
        k = bt.kappa2(Um)
        assert 0.95 * k1d <= k <= k1d * 1.005, (s, k, k1d)
        assert k <= k2d
    for s, k1d in zip(g["lobatto_s"], g["lobatto_LD_1D"]):
        A, _, _ = bt.lobatto_iiic(s)
        _, _, Um = bt.ldu(A)
        k = bt.kappa2(Um)
        assert 0.95 * k1d <= k <= k1d * 1.005, (s, k, k1d)


def test_table2_right_limits_and_ordering():
    """Table 2 (right preconditioning, heat): the limits kappa(A A~^{-1}) lie
    0-15% below the printed full-system values, and every row keeps the
    printed ordering of the four preconditioners."""
    g = GOLD["table2_right_heat_radau"]
    for idx, s in enumerate(g["s"]):
        A, _, _ = bt.radau_iia(s)
        ours = {}
        for kind in ("J", "GSL", "DU", "LD"):
            ours[kind] = bt.kappa2(A @ np.linalg.inv(bt.atilde(A, kind)))
            ratio = ours[kind] / g[kind][idx]
            assert 0.85 <= ratio <= 1.0, (s, kind, ours[kind], g[kind][idx])
        paper_order = sorted(("J", "GSL", "DU", "LD"), key=lambda k: g[k][idx])
        our_order = sorted(ours, key=ours.get)
        assert paper_order == our_order, (s, paper_order, our_order)


def test_gsl_optimized():
    """Eq. GSLopt: the recomputed optimum keeps diag(A), is lower triangular,
    improves on tril(A), and is at least as good as the values quoted in
    Table 4 (the paper notes those may not be global minima)."""
    g = GOLD["table4_left_optimized_gsl"]
    for s, kq in zip(g["radau_s"], g["radau_GSLopt_1D"]):
        A, _, _ = bt.radau_iia(s)
        G = bt.gsl_optimized(A)
        assert np.allclose(np.diag(G), np.diag(A))
        assert np.allclose(np.triu(G, 1), 0)
        k = bt.kappa2(np.linalg.solve(G, A))
        assert k <= bt.kappa2(np.linalg.solve(np.tril(A), A)) + 1e-12
        assert k <= kq * 1.01, (s, k, kq)
