"""The paper's parallel-associative-scan machinery for the LQ subproblem
(Sec. IV-A.1, App. A).

Test infrastructure only (see oracle/__init__.py).

An element is the conditional value function V_{i->j} of eq. CVF, stored as the
tuple (P~, p~, A~, C~, b~).  combine() is eq. combination_rules; leaves() is
eq. assoc_init.  Readings taken:
  * eq. comb_p is printed with "p~_kj - P~_kj b~_ik"; the sign that makes the
    operator associative and reproduces the Riccati recursion is "+":
    p~_ij = Ups (p~_kj + P~_kj b~_ik) + p~_ik.
  * the identity element is (0, 0, I, 0, 0).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Elem:
    P: np.ndarray
    p: np.ndarray
    A: np.ndarray
    C: np.ndarray
    b: np.ndarray


def identity(nx: int) -> Elem:
    """Identity of the combine: (P~, p~, A~, C~, b~) = (0, 0, I, 0, 0)."""
    return Elem(np.zeros((nx, nx)), np.zeros(nx), np.eye(nx), np.zeros((nx, nx)), np.zeros(nx))


def leaves(A, B, c, Qh, Rh, Sh, qh, rh) -> list[Elem]:
    """Initial scan elements, eq. assoc_init:

    P~_{i,i+1} = Q^_i - S^_i^T R^_i^{-1} S^_i,  p~_{i,i+1} = q^_i - S^_i^T Omega_i,
    A~_{i,i+1} = A_i - B_i R^_i^{-1} S^_i,     C~_{i,i+1} = B_i R^_i^{-1} B_i^T,
    b~_{i,i+1} = b_i - B_i Omega_i,            Omega_i = R^_i^{-1} r^_i,
    and the terminal element (Q^_N, q^_N, 0, 0, 0).
    """
    N, nx = A.shape[0], A.shape[1]
    out = []
    for i in range(N):
        Ri = np.linalg.inv(Rh[i])
        Om = Ri @ rh[i]
        out.append(Elem(P=Qh[i] - Sh[i].T @ Ri @ Sh[i],
                        p=qh[i] - Sh[i].T @ Om,
                        A=A[i] - B[i] @ Ri @ Sh[i],
                        C=B[i] @ Ri @ B[i].T,
                        b=c[i] - B[i] @ Om))
    out.append(Elem(P=Qh[N].copy(), p=qh[N].copy(), A=np.zeros((nx, nx)), C=np.zeros((nx, nx)),
                    b=np.zeros(nx)))
    return out


def combine(l: Elem, r: Elem) -> Elem:
    """V_{i->j} = V_{i->k} (x) V_{k->j}, eq. combination_rules, with
    Ups = A~_ik^T (I + P~_kj C~_ik)^{-1} and Psi = A~_kj (I + C~_ik P~_kj)^{-1}."""
    nx = l.P.shape[0]
    I = np.eye(nx)
    Ups = l.A.T @ np.linalg.inv(I + r.P @ l.C)
    Psi = r.A @ np.linalg.inv(I + l.C @ r.P)
    return Elem(P=Ups @ r.P @ l.A + l.P,
                p=Ups @ (r.p + r.P @ l.b) + l.p,
                A=Psi @ l.A,
                C=Psi @ l.C @ r.A.T + r.C,
                b=Psi @ (l.b - l.C @ r.p) + r.b)


def suffix_scan(elems: list[Elem]) -> list[Elem]:
    """Reverse scan eq. revere_assoc_scan written as its definition:
    s_i = a_i (x) a_{i+1} (x) ... (x) a_N, folded from the right."""
    n = len(elems)
    out = [None] * n
    out[n - 1] = elems[n - 1]
    for i in range(n - 2, -1, -1):
        out[i] = combine(elems[i], out[i + 1])
    return out


def blelloch_exclusive(a: list, op, e):
    """The App. A schedule (eq. prefix_sums, eq. downsweep_rules) on an
    arbitrary associative op with identity e: up-sweep builds the balanced
    tree of partial reductions bottom-up, down-sweep passes pref(L) = pref(P),
    pref(R) = pref(P) op val(L).  Returns the exclusive prefixes
    p_i = a_1 op ... op a_{i-1}.  Works for any length by padding with e."""
    n = len(a)
    size = 1
    while size < n:
        size *= 2
    levels = [list(a) + [e] * (size - n)]
    while len(levels[-1]) > 1:
        cur = levels[-1]
        levels.append([op(cur[2 * i], cur[2 * i + 1]) for i in range(len(cur) // 2)])
    pref = [e]
    for d in range(len(levels) - 2, -1, -1):
        vals = levels[d]
        nxt = []
        for i, pp in enumerate(pref):
            nxt.append(pp)                      # left child
            nxt.append(op(pp, vals[2 * i]))     # right child
        pref = nxt
    return pref[:n]


def blelloch_inclusive(a: list, op, e):
    """Inclusive prefixes s_i = p_i op a_i from the exclusive ones (App. A,
    last step)."""
    ex = blelloch_exclusive(a, op, e)
    return [op(ex[i], a[i]) for i in range(len(a))]


def suffix_scan_blelloch(elems: list[Elem]) -> list[Elem]:
    """Reverse scan computed with the App. A schedule: run the prefix schedule
    on the reversed sequence with the flipped operator (x * y = y (x) x)."""
    nx = elems[0].P.shape[0]
    rev = elems[::-1]
    res = blelloch_inclusive(rev, lambda x, y: combine(y, x), identity(nx))
    return res[::-1]


def riccati_from_scan(elems: list[Elem]):
    """P_i = P~_{i,N+1}, p_i = p~_{i,N+1} (the recovery stated after
    eq. assoc_init)."""
    s = suffix_scan(elems)
    return np.stack([e.P for e in s]), np.stack([e.p for e in s])


def gains(A, B, c, Rh, Sh, rh, P, p):
    """Feedback terms eq. controller_cache from the Riccati terms:
    Gamma_i = (R^_i + B_i^T P_{i+1} B_i)^{-1},
    K_i = -Gamma_i (S^_i + B_i^T P_{i+1} A_i),
    k_i = -Gamma_i (B_i^T (p_{i+1} + P_{i+1} b_i) + r^_i)."""
    N = A.shape[0]
    K = np.zeros((N, B.shape[2], A.shape[1]))
    k = np.zeros((N, B.shape[2]))
    for i in range(N):
        G = np.linalg.inv(Rh[i] + B[i].T @ P[i + 1] @ B[i])
        K[i] = -G @ (Sh[i] + B[i].T @ P[i + 1] @ A[i])
        k[i] = -G @ (B[i].T @ (p[i + 1] + P[i + 1] @ c[i]) + rh[i])
    return K, k


def forward_scan(A, B, c, K, k, x0):
    """Conditional optimal trajectory scan, eq. CVF_nominal / nom_recovery.

    Elements are affine maps h(x) = Abar x + bbar; composing h_{i->k} then
    h_{k->j} gives Abar_ij = Abar_kj Abar_ik, bbar_ij = Abar_kj bbar_ik + bbar_kj
    (reading: the printed order Abar_ik Abar_kj does not compose maps).  The
    first element is the constant map dx_1 = (A_0 + B_0 K_0) dx_0 + B_0 k_0 + b_0
    (reading: the printed bbar_01 omits the feedback), with Abar_01 = 0.
    """
    N, nx = A.shape[0], A.shape[1]
    els = []
    els.append((np.zeros((nx, nx)), (A[0] + B[0] @ K[0]) @ x0 + B[0] @ k[0] + c[0]))
    for i in range(1, N):
        els.append((A[i] + B[i] @ K[i], B[i] @ k[i] + c[i]))

    def op(l, r):
        return (r[0] @ l[0], r[0] @ l[1] + r[1])

    pref = blelloch_inclusive(els, op, (np.eye(nx), np.zeros(nx)))
    x = np.zeros((N + 1, nx))
    x[0] = x0
    for i in range(N):
        x[i + 1] = pref[i][1]
    u = np.stack([K[i] @ x[i] + k[i] for i in range(N)])
    return x, u
