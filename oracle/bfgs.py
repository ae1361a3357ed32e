"""FP64 oracle for the quasi-Newton and uncertainty part of preconditioned-BFGS
FWI (Liu et al. 2020, Section 2.1 and 2.3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Functions follow the paper's notation: B is the inverse Hessian
approximation, B0 its diagonal initial guess (a vector here), s_i / y_i the
model and gradient differences (rows of S and Y).
"""
from __future__ import annotations

import numpy as np


def dense_inverse_update(B: np.ndarray, s: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Eq. 3: B_{k+1} = (I - s y^T / y^T s) B_k (I - y s^T / y^T s) + s s^T / y^T s."""
    rho = 1.0 / float(y @ s)
    n = len(s)
    I = np.eye(n)
    L = I - rho * np.outer(s, y)
    return L @ B @ L.T + rho * np.outer(s, s)


def dense_hessian_update(Hs: np.ndarray, s: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Eq. 2: H_{k+1} = H_k + y y^T / y^T s - H_k s s^T H_k^T / s^T H_k s."""
    Hs_s = Hs @ s
    return Hs + np.outer(y, y) / float(y @ s) - np.outer(Hs_s, Hs_s) / float(s @ Hs_s)


def dense_inverse(B0: np.ndarray, S: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """B_{n+1} from B0 = diag(B0) and pairs (s_i, y_i), i = 0..n, in order (Eq. 9)."""
    B = np.diag(np.asarray(B0, np.float64))
    for s, y in zip(S, Y):
        B = dense_inverse_update(B, s, y)
    return B


def lbfgs_direction(g: np.ndarray, S: np.ndarray, Y: np.ndarray, B0: np.ndarray,
                    m: int | None = None, use_gamma: bool = True) -> np.ndarray:
    """Algorithm 1: z = -gamma_k B_k g with memory m (None: all pairs) and
    B_k^0 = diag(B0); gamma_k = s_{k-1}^T y_{k-1} / y_{k-1}^T y_{k-1}."""
    k = len(S)
    lo = 0 if m is None else max(0, k - m)
    q = np.array(g, dtype=np.float64)
    a = np.zeros(k)
    r = np.zeros(k)
    for i in range(k - 1, lo - 1, -1):
        r[i] = 1.0 / float(Y[i] @ S[i])
        a[i] = r[i] * float(S[i] @ q)
        q = q - a[i] * Y[i]
    gamma = float(S[k - 1] @ Y[k - 1]) / float(Y[k - 1] @ Y[k - 1]) if (use_gamma and k > 0) else 1.0
    z = gamma * np.asarray(B0, np.float64) * q
    for i in range(lo, k):
        b = r[i] * float(Y[i] @ z)
        z = z + S[i] * (a[i] - b)
    return -z


def probe(e: np.ndarray, S: np.ndarray, Y: np.ndarray, B0: np.ndarray) -> np.ndarray:
    """Algorithm 2: z = (B_{n+1} - B0) e by the two-loop recursion with the
    fixed initial guess B0 and no gamma scaling."""
    n = len(S)
    q = np.array(e, dtype=np.float64)
    a = np.zeros(n)
    r = np.zeros(n)
    for i in range(n - 1, -1, -1):
        r[i] = 1.0 / float(Y[i] @ S[i])
        a[i] = r[i] * float(S[i] @ q)
        q = q - a[i] * Y[i]
    z = np.asarray(B0, np.float64) * q
    for i in range(n):
        b = r[i] * float(Y[i] @ z)
        z = z + S[i] * (a[i] - b)
    return z - np.asarray(B0, np.float64) * e


def probe_block(X: np.ndarray, S, Y, B0) -> np.ndarray:
    """Algorithm 2 applied to every row x_k of X (the E = (B_{n+1} - B0) X of
    Section 2.3).  X and the result are [p][n]."""
    return np.stack([probe(x, S, Y, B0) for x in X])


def rsvd_single_pass(E: np.ndarray, X: np.ndarray, rank: int):
    """Algorithm 3 on the sample E = B X (rows are vectors: E, X are [p][n]).

      QR = E;  Omega (Q^T X) = Q^T E;  U Lambda U^T = Omega;  V = Q U.

    Omega is symmetrised before the eigendecomposition (B is symmetric) and
    the eigenpairs are ordered by |lambda|, largest first; the first `rank`
    are returned as V [rank][n], lam [rank]."""
    Et = np.asarray(E, np.float64).T               # n x p
    Xt = np.asarray(X, np.float64).T
    Q, _ = np.linalg.qr(Et)                        # n x p, orthonormal columns
    QtX = Q.T @ Xt
    QtE = Q.T @ Et
    Omega = np.linalg.solve(QtX.T, QtE.T).T        # Omega QtX = QtE
    Omega = 0.5 * (Omega + Omega.T)
    lam, U = np.linalg.eigh(Omega)
    order = np.argsort(-np.abs(lam), kind="stable")
    lam, U = lam[order], U[:, order]
    V = (Q @ U).T
    return V[:rank], lam[:rank]


def rsvd_two_pass(apply, X: np.ndarray, rank: int):
    """Two-pass variant of Algorithm 3 (the Rayleigh-Ritz form of the
    randomized eigendecomposition, Halko, Martinsson & Tropp 2011, Alg. 5.3):
    the first pass E = A X gives the basis, QR = E; the second applies the
    operator to the basis, C = Q^T A Q, and C = U Lambda U^T, V = Q U.  No
    (Q^T X)^-1 appears, at the cost of a second application of A.
    `apply(M)` returns A M for a block M of rows ([m][n] -> [m][n]).  C is
    symmetrised; eigenpairs ordered by |lambda|, largest first; the first
    `rank` are returned as V [rank][n], lam [rank]."""
    E = np.asarray(apply(np.asarray(X, np.float64)), np.float64)
    Q, _ = np.linalg.qr(E.T)                       # n x p, orthonormal columns
    AQ = np.asarray(apply(Q.T), np.float64)        # rows: A q_j
    C = Q.T @ AQ.T
    C = 0.5 * (C + C.T)
    lam, U = np.linalg.eigh(C)
    order = np.argsort(-np.abs(lam), kind="stable")
    lam, U = lam[order], U[:, order]
    V = (Q @ U).T
    return V[:rank], lam[:rank]


def posterior_std(V: np.ndarray, lam: np.ndarray, B0: np.ndarray, eps: float = 1.0):
    """Eqs. 10 and 14 with C_m = eps I:  C_M = eps (V Lambda V^T + B0),
    std = sqrt(diag C_M); negative diagonals (from a truncated, indefinite
    low-rank part) are clipped at zero."""
    d = np.einsum("kn,k,kn->n", V, lam, V) + np.asarray(B0, np.float64)
    return np.sqrt(eps * np.maximum(d, 0.0))


def exact_lowrank(S, Y, B0, rank: int):
    """Eigenpairs of B_{n+1} - B0 from its dense form (small n only)."""
    B = dense_inverse(B0, S, Y) - np.diag(np.asarray(B0, np.float64))
    lam, U = np.linalg.eigh(0.5 * (B + B.T))
    order = np.argsort(-np.abs(lam), kind="stable")
    return U[:, order].T[:rank], lam[order][:rank]
