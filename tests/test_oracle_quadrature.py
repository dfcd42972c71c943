"""Pins of the oracle's quadrature and SDC matrices against closed forms,
library routines and algebraic identities (Sec. 3, Sec. 4.2, Sec. 4.3.3)."""
import numpy as np
import pytest

from oracle import quadrature as q


@pytest.mark.parametrize("J", [2, 5, 32, 64, 128, 256])
def test_gauss_legendre_matches_library(J):
    mu, w = q.gauss_legendre(J)
    xl, wl = np.polynomial.legendre.leggauss(J)
    order = np.argsort(mu)
    assert np.all(np.diff(mu) < 0), "north to south ordering"
    assert np.max(np.abs(mu[order] - xl)) < 2e-15
    assert np.max(np.abs(w[order] - wl)) < 1e-14
    assert abs(w.sum() - 2.0) < 1e-14


@pytest.mark.parametrize("J", [4, 17, 32])
def test_gauss_legendre_exact_monomials(J):
    mu, w = q.gauss_legendre(J)
    for k in range(2 * J):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * mu ** k) - exact) < 1e-14


def test_lobatto_closed_forms():
    assert np.allclose(q.lobatto_nodes(2), [0.0, 1.0], atol=0, rtol=0)
    assert np.max(np.abs(q.lobatto_nodes(3) - [0.0, 0.5, 1.0])) < 1e-16
    r = np.sqrt(3.0 / 7.0)
    ref = [0.0, (1 - r) / 2, 0.5, (1 + r) / 2, 1.0]
    assert np.max(np.abs(q.lobatto_nodes(5) - ref)) < 1e-15


def test_collocation_rows_are_lobatto_rules():
    Q3 = q.collocation_matrix(q.lobatto_nodes(3))
    assert np.max(np.abs(Q3[-1] - [1 / 6, 2 / 3, 1 / 6])) < 1e-15        # Simpson
    assert np.max(np.abs(Q3[1] - [5 / 24, 1 / 3, -1 / 24])) < 1e-15
    assert np.max(np.abs(Q3[0])) == 0.0
    Q5 = q.collocation_matrix(q.lobatto_nodes(5))
    assert np.max(np.abs(Q5[-1] - [1 / 20, 49 / 180, 16 / 45, 49 / 180, 1 / 20])) < 1e-15


@pytest.mark.parametrize("n", [2, 3, 5])
def test_collocation_integrates_polynomials(n):
    t = q.lobatto_nodes(n)
    Q = q.collocation_matrix(t)
    for k in range(n):
        assert np.max(np.abs(Q @ t ** k - t ** (k + 1) / (k + 1))) < 1e-15


@pytest.mark.parametrize("n", [2, 3, 5])
def test_explicit_euler_rows_sum_to_node_time(n):
    t = q.lobatto_nodes(n)
    QE = q.explicit_euler_matrix(t)
    assert np.max(np.abs(QE.sum(axis=1) - t)) < 1e-15
    assert np.all(np.triu(QE) == 0.0)


def test_lu_trick_three_nodes_by_hand():
    QI = q.lu_implicit_matrix(q.collocation_matrix(q.lobatto_nodes(3)))
    ref = np.array([[0, 0, 0], [0, 1 / 3, 0], [0, 2 / 3, 1 / 4]])
    assert np.max(np.abs(QI - ref)) < 1e-15


@pytest.mark.parametrize("n", [3, 5])
def test_lu_trick_nilpotent(n):
    Q = q.collocation_matrix(q.lobatto_nodes(n))
    QI = q.lu_implicit_matrix(Q)
    assert np.all(np.triu(QI, 1) == 0.0)
    E = np.eye(n - 1) - np.linalg.solve(QI[1:, 1:], Q[1:, 1:])
    assert np.max(np.abs(np.tril(E))) < 1e-14          # strictly upper triangular
    assert np.max(np.abs(np.linalg.matrix_power(E, n - 1))) < 1e-13


def test_time_transfer_is_injection_for_nested_lobatto():
    tf, tc = q.lobatto_nodes(5), q.lobatto_nodes(3)
    P = q.lagrange_matrix(tf, tc)
    sel = np.zeros((3, 5))
    sel[0, 0] = sel[1, 2] = sel[2, 4] = 1.0
    assert np.max(np.abs(P - sel)) < 1e-14
    P32 = q.lagrange_matrix(q.lobatto_nodes(3), q.lobatto_nodes(2))
    assert np.max(np.abs(P32 - [[1, 0, 0], [0, 0, 1]])) < 1e-15


def test_time_interpolation_reproduces_polynomials():
    tf, tc = q.lobatto_nodes(5), q.lobatto_nodes(3)
    P = q.lagrange_matrix(tc, tf)
    for k in range(3):
        assert np.max(np.abs(P @ tc ** k - tf ** k)) < 1e-15
