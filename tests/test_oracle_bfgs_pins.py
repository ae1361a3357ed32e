"""Pins of the quasi-Newton / randomized-SVD oracle against textbook facts:
secant equation, Eq. 3 as the exact inverse of Eq. 2, quadratic termination
and hereditary secant property of BFGS with exact line search, the two-loop
recursions (Algorithms 1 and 2) against the dense recursion, and Algorithm 3
against exact eigenpairs; Philox against its published known-answer
vectors."""
import os

import numpy as np

import synth
from oracle import bfgs, philox

RNG = np.random.default_rng(2024)
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _pairs(n, k):
    S, Y, B0 = synth.synthetic_history(11, n, k, dtype=np.float64)
    return S, Y, B0


def test_secant_equation_last_pair():
    S, Y, B0 = _pairs(40, 7)
    B = np.diag(B0)
    for s, y in zip(S, Y):
        B = bfgs.dense_inverse_update(B, s, y)
        assert np.allclose(B @ y, s, rtol=1e-12, atol=1e-15)
        assert np.allclose(B, B.T, atol=1e-15 * np.abs(B).max())


def test_eq3_is_inverse_of_eq2():
    S, Y, B0 = _pairs(12, 6)
    B = np.diag(B0)
    H = np.diag(1.0 / B0)
    for s, y in zip(S, Y):
        B = bfgs.dense_inverse_update(B, s, y)
        H = bfgs.dense_hessian_update(H, s, y)
        assert np.allclose(B @ H, np.eye(len(s)), atol=1e-9)


def test_quadratic_termination_and_hereditary_secant():
    n = 8
    A, b = synth.quadratic_problem(3, n)
    x = np.zeros(n)
    B = np.eye(n)
    S, Y = [], []
    g = A @ x - b
    for k in range(n):
        p = -B @ g
        alpha = -(g @ p) / (p @ A @ p)                 # exact line search
        xn = x + alpha * p
        gn = A @ xn - b
        s, y = xn - x, gn - g
        B = bfgs.dense_inverse_update(B, s, y)
        S.append(s); Y.append(y)
        for si, yi in zip(S, Y):                       # B_k y_i = s_i for all i < k
            assert np.allclose(B @ yi, si, rtol=1e-8, atol=1e-10)
        x, g = xn, gn
    assert np.allclose(B, np.linalg.inv(A), rtol=1e-7, atol=1e-9)
    assert np.linalg.norm(A @ x - b) < 1e-8


def test_two_loop_equals_dense_bfgs():
    S, Y, B0 = _pairs(60, 9)
    g = RNG.standard_normal(60)
    Bd = bfgs.dense_inverse(B0, S, Y)
    # Algorithm 1, full memory, no gamma scaling == -B_k g
    z = bfgs.lbfgs_direction(g, S, Y, B0, m=None, use_gamma=False)
    assert np.allclose(z, -Bd @ g, rtol=1e-10)
    # with gamma: BFGS started from gamma_k B0
    gam = (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1])
    z = bfgs.lbfgs_direction(g, S, Y, B0, m=None, use_gamma=True)
    assert np.allclose(z, -bfgs.dense_inverse(gam * B0, S, Y) @ g, rtol=1e-10)
    # memory m >= k is full BFGS; m < k differs
    z9 = bfgs.lbfgs_direction(g, S, Y, B0, m=20, use_gamma=False)
    assert np.allclose(z9, -Bd @ g, rtol=1e-10)
    z3 = bfgs.lbfgs_direction(g, S, Y, B0, m=3, use_gamma=False)
    assert not np.allclose(z3, -Bd @ g, rtol=1e-6)
    # Algorithm 2: (B_{n+1} - B0) e_j is column j of the dense difference
    for j in (0, 17, 59):
        e = np.zeros(60); e[j] = 1
        assert np.allclose(bfgs.probe(e, S, Y, B0), (Bd - np.diag(B0))[:, j], atol=1e-12 * np.abs(Bd).max())


def test_rsvd_recovers_exact_low_rank():
    n, r, p = 300, 8, 12
    Q, _ = np.linalg.qr(RNG.standard_normal((n, r)))
    lam = np.array([5.0, -3.0, 2.5, 1.0, -0.7, 0.4, 0.2, 0.05])
    A = (Q * lam) @ Q.T
    X = RNG.standard_normal((p, n))
    E = (A @ X.T).T
    V, l = bfgs.rsvd_single_pass(E, X, r)
    order = np.argsort(-np.abs(lam))
    assert np.allclose(l, lam[order], rtol=1e-9, atol=1e-12)
    # eigenvectors up to sign
    for k in range(r):
        assert abs(abs(V[k] @ Q[:, order[k]]) - 1) < 1e-9


def test_rsvd_on_bfgs_history_matches_dense_eigh_and_std():
    n, k = 150, 5
    S, Y, B0 = _pairs(n, k)
    p = 2 * k + 4                                      # rank(B - B0) <= 2k
    X = RNG.standard_normal((p, n))
    E = bfgs.probe_block(X, S, Y, B0)
    V, l = bfgs.rsvd_single_pass(E, X, 2 * k)
    Ve, le = bfgs.exact_lowrank(S, Y, B0, 2 * k)
    assert np.allclose(l, le, rtol=1e-7, atol=1e-12 * np.abs(le).max())
    Bd = bfgs.dense_inverse(B0, S, Y)
    std = bfgs.posterior_std(V, l, B0, eps=2.0)
    assert np.allclose(std, np.sqrt(2.0 * np.diag(Bd)), rtol=1e-7)


def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox_kat.txt")) if l.strip() and not l.startswith("#")]
    for row in rows:
        vals = [int(v, 16) for v in row]
        ctr = np.array([vals[0:4]], dtype=np.uint64)
        key = np.array([vals[4:6]], dtype=np.uint64)
        out = philox.philox4x32_10(ctr, key)[0]
        assert [int(v) for v in out] == vals[6:10]


def test_philox_gaussian_block_moments():
    X = philox.gaussian_block(12345, 4, 50000)
    assert abs(X.mean()) < 0.01 and abs(X.var() - 1) < 0.01
    assert abs(np.mean(X[0] * X[1])) < 0.02
    assert not np.allclose(X, philox.gaussian_block(12346, 4, 50000))


def test_two_pass_rsvd_exact_on_low_rank_and_ritz_bounds():
    """Two-pass variant: with p >= rank(A) probes it recovers the exact
    eigenpairs; with fewer, its Ritz values lie inside the spectrum's range
    and the largest one is within the subspace-iteration bound of the true
    largest eigenvalue (a single pass has no such guarantee)."""
    n, r = 300, 8
    Q, _ = np.linalg.qr(RNG.standard_normal((n, r)))
    lam = np.array([5.0, -3.0, 2.5, 1.0, -0.7, 0.4, 0.2, 0.05])
    A = (Q * lam) @ Q.T
    apply = lambda M: (A @ np.asarray(M).T).T
    order = np.argsort(-np.abs(lam))
    V, l = bfgs.rsvd_two_pass(apply, RNG.standard_normal((12, n)), r)
    assert np.allclose(l, lam[order], rtol=1e-9, atol=1e-12)
    for k in range(r):
        assert abs(abs(V[k] @ Q[:, order[k]]) - 1) < 1e-9
    V4, l4 = bfgs.rsvd_two_pass(apply, RNG.standard_normal((4, n)), 4)
    assert np.all(l4 <= lam.max() + 1e-12) and np.all(l4 >= lam.min() - 1e-12)
    assert abs(l4[0]) <= 5.0 + 1e-12 and abs(l4[0]) > 0.5 * 5.0
    # the Ritz vectors are orthonormal
    assert np.allclose(V4 @ V4.T, np.eye(4), atol=1e-12)


def test_two_pass_rsvd_on_bfgs_history_equals_dense_eigh():
    n, k = 150, 5
    S, Y, B0 = _pairs(n, k)
    apply = lambda M: bfgs.probe_block(np.asarray(M), S, Y, B0)
    X = RNG.standard_normal((2 * k + 3, n))
    V, l = bfgs.rsvd_two_pass(apply, X, 2 * k)
    Ve, le = bfgs.exact_lowrank(S, Y, B0, 2 * k)
    assert np.allclose(l, le, rtol=1e-8, atol=1e-12 * np.abs(le).max())
    for j in range(2 * k):
        assert abs(abs(V[j] @ Ve[j]) - 1) < 1e-7


def test_probe_block_lies_in_span_of_pairs_with_compact_coordinates():
    """The compact representation of Byrd, Nocedal & Schnabel (1994):
    B_{n+1} - B0 = W M W^T with W = [S, B0 Y] (rows s_i, B0 y_i) and
    M = [[R^-T (D + Y^T B0 Y) R^-1, -R^-T], [-R^-1, 0]], R_ij = s_i^T y_j
    (i <= j), D = diag(s_i^T y_i).  So every row of E = (B_{n+1} - B0) X of
    Algorithm 2 lies in the span of the pairs, with coordinates
    C = (M W^T X)^T.  A two-loop recursion that kept the B0 e term, or put
    B0 on the wrong side of a loop, leaves E outside that span."""
    S, Y, B0 = _pairs(80, 7)
    k = len(S)
    X = RNG.standard_normal((9, 80))
    E = bfgs.probe_block(X, S, Y, B0)
    W = np.vstack([S, B0 * Y])
    Qw, _ = np.linalg.qr(W.T)
    outside = E - (E @ Qw) @ Qw.T
    assert np.abs(outside).max() < 1e-12 * np.abs(E).max()
    SY = S @ Y.T
    R = np.triu(SY)
    D = np.diag(np.diag(SY))
    YBY = Y @ (B0 * Y).T
    Ri = np.linalg.inv(R)
    M = np.block([[Ri.T @ (D + YBY) @ Ri, -Ri.T], [-Ri, np.zeros((k, k))]])
    C = (M @ (W @ X.T)).T
    assert np.abs(C @ W - E).max() < 1e-12 * np.abs(E).max()
