"""Pins of the oracle's scan machinery (eq. combination_rules, App. A)."""
import numpy as np
import pytest

from oracle import lq, scan
from paper_2604_07644_b300 import workloads as W


def _rand_elem(g, n, complete=False):
    M = g.standard_normal((n, n))
    P = M @ M.T / n + 0.1 * np.eye(n)
    M = g.standard_normal((n, n))
    C = M @ M.T / n
    A = g.standard_normal((n, n)) * 0.5
    if complete:
        A = np.zeros((n, n))
        C = np.zeros((n, n))
    b = np.zeros(n) if complete else g.standard_normal(n)
    return scan.Elem(P=P, p=g.standard_normal(n), A=A, C=C, b=b)


def _close(e1, e2, tol=1e-11):
    return all(np.allclose(getattr(e1, f), getattr(e2, f), atol=tol, rtol=tol) for f in "PpACb")


@pytest.mark.parametrize("seed", range(4))
def test_combine_is_associative(seed):
    g = np.random.default_rng(seed)
    a, b, c = (_rand_elem(g, 4) for _ in range(3))
    assert _close(scan.combine(scan.combine(a, b), c), scan.combine(a, scan.combine(b, c)), 1e-10)


def test_identity_element():
    g = np.random.default_rng(7)
    a = _rand_elem(g, 5)
    e = scan.identity(5)
    assert _close(scan.combine(e, a), a)
    assert _close(scan.combine(a, e), a)


@pytest.mark.parametrize("dims", [(2, 1, 3, 2, 1), (4, 2, 9, 3, 2), (6, 3, 17, 5, 0)])
def test_scan_reproduces_riccati(dims):
    """P_i = P~_{i,N+1}, p_i = p~_{i,N+1} (statement after eq. assoc_init),
    with S != 0 and b != 0."""
    qp = W.random_general(1, *dims)
    rho = 0.6
    Qh, Rh, Sh = lq.augmented(qp, rho)
    g = np.random.default_rng(2)
    qh, rh = lq.augmented_linear(qp, rho, g.standard_normal(qp.m), g.standard_normal(qp.m))
    P, p, K, kff, _ = lq.riccati(qp.A, qp.B, qp.c, Qh, Rh, Sh, qh, rh)
    els = scan.leaves(qp.A, qp.B, qp.c, Qh, Rh, Sh, qh, rh)
    Ps, ps = scan.riccati_from_scan(els)
    assert np.allclose(Ps, P, atol=1e-10, rtol=1e-10)
    assert np.allclose(ps, p, atol=1e-10, rtol=1e-10)
    K2, k2 = scan.gains(qp.A, qp.B, qp.c, Rh, Sh, rh, Ps, ps)
    assert np.allclose(K2, K, atol=1e-10) and np.allclose(k2, kff, atol=1e-10)
    x, u = lq.rollout(qp.A, qp.B, qp.c, K, kff, qp.x0)
    xf, uf = scan.forward_scan(qp.A, qp.B, qp.c, K2, k2, qp.x0)
    assert np.allclose(xf, x, atol=1e-10) and np.allclose(uf, u, atol=1e-10)


def test_minus_sign_reading_is_wrong(monkeypatch):
    """Planted mistake: the printed '-' in eq. comb_p breaks associativity and
    the Riccati match, so the pins above would catch it."""
    def bad(l, r):
        I = np.eye(l.P.shape[0])
        Ups = l.A.T @ np.linalg.inv(I + r.P @ l.C)
        Psi = r.A @ np.linalg.inv(I + l.C @ r.P)
        return scan.Elem(P=Ups @ r.P @ l.A + l.P, p=Ups @ (r.p - r.P @ l.b) + l.p, A=Psi @ l.A,
                         C=Psi @ l.C @ r.A.T + r.C, b=Psi @ (l.b - l.C @ r.p) + r.b)

    qp = W.random_general(1, 4, 2, 9, 3, 2)
    Qh, Rh, Sh = lq.augmented(qp, 0.6)
    qh, rh = lq.augmented_linear(qp, 0.6, np.ones(qp.m), np.zeros(qp.m))
    P, p, *_ = lq.riccati(qp.A, qp.B, qp.c, Qh, Rh, Sh, qh, rh)
    monkeypatch.setattr(scan, "combine", bad)
    els = scan.leaves(qp.A, qp.B, qp.c, Qh, Rh, Sh, qh, rh)
    _, ps = scan.riccati_from_scan(els)
    assert not np.allclose(ps, p, atol=1e-6)


@pytest.mark.parametrize("n", list(range(1, 34)))
def test_blelloch_schedule_integer_add(n):
    """App. A schedule with integer + (exact): inclusive prefixes equal the
    running sums for every length, including non powers of two."""
    a = list(range(3, 3 + n))
    res = scan.blelloch_inclusive(a, lambda x, y: x + y, 0)
    assert res == list(np.cumsum(a))


@pytest.mark.parametrize("n", [1, 2, 5, 8, 13])
def test_blelloch_schedule_matrix_product(n):
    """Non-commutative operator: ordered matrix products."""
    g = np.random.default_rng(n)
    mats = [g.standard_normal((3, 3)) for _ in range(n)]
    res = scan.blelloch_inclusive(mats, lambda x, y: x @ y, np.eye(3))
    acc = np.eye(3)
    for i in range(n):
        acc = acc @ mats[i]
        assert np.allclose(res[i], acc, atol=1e-12)


@pytest.mark.parametrize("N", [1, 2, 7, 16, 21])
def test_reverse_scan_blelloch_equals_fold(N):
    qp = W.random_general(4, 3, 2, N, 2, 1)
    Qh, Rh, Sh = lq.augmented(qp, 0.3)
    qh, rh = lq.augmented_linear(qp, 0.3, np.ones(qp.m), np.zeros(qp.m))
    els = scan.leaves(qp.A, qp.B, qp.c, Qh, Rh, Sh, qh, rh)
    s1 = scan.suffix_scan(els)
    s2 = scan.suffix_scan_blelloch(els)
    for a, b in zip(s1, s2):
        assert _close(a, b, 1e-10)
