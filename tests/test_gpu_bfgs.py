"""GPU parity of the BFGS store, the compact inverse-Hessian apply and the
randomized-SVD uncertainty path against the FP64 oracle (Algorithms 1-3,
Eqs. 3, 9-14), through the C ABI.  Tolerance 1e-4 relative (FP32 vectors,
FP64 small matrices)."""
import numpy as np
import pytest

import synth
from oracle import bfgs as ob
from oracle import philox

torch = pytest.importorskip("torch")
import paper_2009_12663_gb300 as gb  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def t32(a):
    return torch.tensor(np.asarray(a, np.float32), device=DEV)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def store(n, k, seed=5, kmax=None):
    S, Y, B0 = synth.synthetic_history(seed, n, k)
    b = gb.Bfgs(n, kmax or k + 4, t32(B0))
    for i in range(k):
        b.update(t32(S[i]), t32(Y[i]))
    return b, S.astype(np.float64), Y.astype(np.float64), B0.astype(np.float64)


@pytest.mark.parametrize("n,k,p", [(1000, 1, 1), (7777, 9, 13), (50000, 30, 64), (20001, 12, 70)])
def test_apply_minus_b0_matches_algorithm_2(n, k, p):
    b, S, Y, B0 = store(n, k)
    assert b.count == k
    X = synth.gaussian_block(11, p, n)
    Z = torch.zeros(p, n, device=DEV)
    b.apply(t32(X), Z, 1.0, minus_B0=True)
    ref = ob.probe_block(X.astype(np.float64), S, Y, B0)
    assert rel(Z.cpu().numpy(), ref) < 1e-4


def test_apply_gamma_matches_algorithm_1():
    n, k = 6000, 8
    b, S, Y, B0 = store(n, k)
    g = np.random.default_rng(3).standard_normal(n)
    gam = float(S[-1] @ Y[-1] / (Y[-1] @ Y[-1]))
    z = torch.zeros(1, n, device=DEV)
    b.apply(t32(g[None]), z, gam, minus_B0=False)
    ref = -ob.lbfgs_direction(g, S, Y, B0, m=None, use_gamma=True)
    assert rel(z.cpu().numpy()[0], ref) < 1e-4


def test_apply_without_pairs_is_b0():
    n = 3000
    B0 = np.random.default_rng(1).uniform(0.5, 2.0, n).astype(np.float32)
    b = gb.Bfgs(n, 4, t32(B0))
    X = synth.gaussian_block(2, 3, n)
    Z = torch.zeros(3, n, device=DEV)
    b.apply(t32(X), Z, 2.0, minus_B0=False)
    assert np.allclose(Z.cpu().numpy(), 2.0 * B0 * X, rtol=1e-6)
    b.apply(t32(X), Z, 1.0, minus_B0=True)
    assert np.all(Z.cpu().numpy() == 0)


def test_curvature_rejection_and_full_store():
    n = 2000
    b, S, Y, B0 = store(n, 2, kmax=3)
    s = np.random.default_rng(0).standard_normal(n).astype(np.float32)
    with pytest.raises(gb.GbfwiError) as e:
        b.update(t32(s), t32(-s))                  # y^T s < 0
    assert e.value.name == "ECURV"
    assert b.count == 2
    b.update(t32(s), t32(2 * s))
    assert b.count == 3
    with pytest.raises(gb.GbfwiError) as e:
        b.update(t32(s), t32(2 * s))               # store full
    assert e.value.name == "EINVAL"


def test_host_arrays_accepted():
    n, k, p = 4000, 5, 4
    b, S, Y, B0 = store(n, k)
    X = synth.gaussian_block(4, p, n)
    Zh = np.zeros((p, n), np.float32)
    b.apply(X, Zh, 1.0, minus_B0=True)
    Zd = torch.zeros(p, n, device=DEV)
    b.apply(t32(X), Zd, 1.0, minus_B0=True)
    assert np.array_equal(Zh, Zd.cpu().numpy())


def _align(V, Vr):
    """Cosines between matching eigenvectors (sign-free), in FP64: with the
    norms of FP32 rows taken in FP32, sqrt(1 - cos^2) would carry ~3e-4 of
    rounding noise."""
    V = np.asarray(V, np.float64)
    Vr = np.asarray(Vr, np.float64)
    return np.abs(np.sum(V * Vr, axis=1)) / (np.linalg.norm(V, axis=1) * np.linalg.norm(Vr, axis=1))


def _check_vectors(V, Vr, lam_all, rank, tol=1e-4):
    """Eigenvector k may turn by ~ (perturbation of Omega) / (gap to the
    nearest other eigenvalue): require sin(angle) <= tol * max|lam| / gap_k + 1e-5."""
    cos = np.clip(_align(V, Vr), 0, 1)
    sin = np.sqrt(1 - cos ** 2)
    scale = np.abs(lam_all).max()
    for k in range(rank):
        gap = np.min(np.abs(np.delete(lam_all, k) - lam_all[k]))
        assert sin[k] <= tol * scale / gap + 1e-5, (k, sin[k], gap)


@pytest.mark.parametrize("n,k,p,rank", [(5000, 12, 16, 10), (30011, 20, 40, 24)])
def test_lowrank_matches_algorithm_3(n, k, p, rank):
    b, S, Y, B0 = store(n, k)
    X = synth.gaussian_block(7, p, n)
    V = torch.zeros(rank, n, device=DEV)
    lam = torch.zeros(rank, dtype=torch.float64, device=DEV)
    std = torch.zeros(n, device=DEV)
    b.lowrank_invhess(p, rank, eps_prior=2.0, X=t32(X), V=V, lam=lam, std=std)
    E = ob.probe_block(X.astype(np.float64), S, Y, B0)
    Vr, lr = ob.rsvd_single_pass(E, X.astype(np.float64), rank)
    _, lam_all = ob.rsvd_single_pass(E, X.astype(np.float64), p)
    lam = lam.cpu().numpy()
    assert np.allclose(lam, lr, rtol=1e-4, atol=1e-6 * np.abs(lr).max())
    _check_vectors(V.cpu().numpy(), Vr, lam_all, rank)
    sr = ob.posterior_std(Vr, lr, B0, eps=2.0)
    assert rel(std.cpu().numpy(), sr) < 1e-4


def test_lowrank_device_philox_matches_oracle_generator():
    n, k, p, rank, seed = 8000, 10, 16, 12, 0x1234_5678_9ABC
    b, S, Y, B0 = store(n, k)
    lam = torch.zeros(rank, dtype=torch.float64, device=DEV)
    std = torch.zeros(n, device=DEV)
    b.lowrank_invhess(p, rank, seed=seed, eps_prior=1.0, lam=lam, std=std)
    X = philox.gaussian_block(seed, p, n)
    E = ob.probe_block(X, S, Y, B0)
    Vr, lr = ob.rsvd_single_pass(E, X, rank)
    assert np.allclose(lam.cpu().numpy(), lr, rtol=1e-4, atol=1e-6 * np.abs(lr).max())
    assert rel(std.cpu().numpy(), ob.posterior_std(Vr, lr, B0, 1.0)) < 1e-4


def test_lowrank_full_rank_equals_dense_inverse_hessian():
    """With p >= 2k probes the low-rank part is exact: diag(V L V^T) + B0 is the
    diagonal of the dense B_{n+1} of Eq. 3 (12 x 6 element model size)."""
    n, k = 3675, 6
    b, S, Y, B0 = store(n, k)
    p = rank = 2 * k
    X = synth.gaussian_block(8, p, n)
    std = torch.zeros(n, device=DEV)
    lam = torch.zeros(rank, dtype=torch.float64, device=DEV)
    b.lowrank_invhess(p, rank, eps_prior=1.0, X=t32(X), std=std, lam=lam)
    Bd = ob.dense_inverse(B0, S, Y)
    assert rel(std.cpu().numpy(), np.sqrt(np.diag(Bd))) < 1e-4
    _, le = ob.exact_lowrank(S, Y, B0, rank)
    assert np.allclose(lam.cpu().numpy(), le, rtol=1e-4, atol=1e-6 * np.abs(le).max())


def test_lowrank_rank_deficient_probe_block():
    """p > 2k probes: E = (B_{n+1} - B0) X has rank 2k exactly, the other
    p - 2k directions of the FP32 block are rounding noise.  The basis keeps
    the 2k resolved directions: their eigenvalues equal the dense
    eigendecomposition of B_{n+1} - B0 and the rest are returned as zero."""
    n, k, p = 3675, 3, 11
    b, S, Y, B0 = store(n, k)
    X = synth.gaussian_block(9, p, n)
    lam = torch.zeros(p, dtype=torch.float64, device=DEV)
    V = torch.zeros(p, n, device=DEV)
    std = torch.zeros(n, device=DEV)
    b.lowrank_invhess(p, p, eps_prior=1.0, X=t32(X), V=V, lam=lam, std=std)
    _, le = ob.exact_lowrank(S, Y, B0, 2 * k)
    lg = lam.cpu().numpy()
    assert np.allclose(lg[:2 * k], le, rtol=1e-4, atol=1e-6 * np.abs(le).max())
    assert np.all(lg[2 * k:] == 0.0)
    assert np.all(V.cpu().numpy()[2 * k:] == 0.0)
    Bd = ob.dense_inverse(B0, S, Y)
    assert rel(std.cpu().numpy(), np.sqrt(np.diag(Bd))) < 1e-4


def test_exact_lowrank_equals_dense_inverse_hessian():
    """B_{n+1} - B0 has rank <= 2k (compact form): the exact decomposition
    from a QR of [S, B0 Y] gives the eigenpairs of the dense matrix and the
    diagonal of the dense B_{n+1} of Eq. 3 (12 x 6 element model size)."""
    n, k = 3675, 6
    b, S, Y, B0 = store(n, k)
    rank = 2 * k
    lam = torch.zeros(rank, dtype=torch.float64, device=DEV)
    V = torch.zeros(rank, n, device=DEV)
    std = torch.zeros(n, device=DEV)
    b.lowrank_exact(rank, eps_prior=1.0, V=V, lam=lam, std=std)
    Ue, le = ob.exact_lowrank(S, Y, B0, rank)
    assert np.allclose(lam.cpu().numpy(), le, rtol=1e-4, atol=1e-6 * np.abs(le).max())
    Bd = ob.dense_inverse(B0, S, Y)
    assert rel(std.cpu().numpy(), np.sqrt(np.diag(Bd))) < 1e-4
    # V diag(lam) V^T equals B_{n+1} - B0 on a probe vector
    x = np.random.default_rng(1).standard_normal(n)
    Vg, lg = V.cpu().numpy().astype(np.float64), lam.cpu().numpy()
    want = (Bd - np.diag(B0)) @ x
    assert rel(Vg.T @ (lg * (Vg @ x)), want) < 1e-4


@pytest.mark.parametrize("n,k,rank", [(30011, 20, 24), (200003, 50, 50)])
def test_exact_lowrank_matches_algorithm_3_with_full_probing(n, k, rank):
    """With p >= 2k probes the single-pass randomized SVD is exact (in
    FP64): the exact decomposition must give the same eigenvalues and
    posterior std without any probes."""
    b, S, Y, B0 = store(n, k)
    lam = torch.zeros(rank, dtype=torch.float64, device=DEV)
    std = torch.zeros(n, device=DEV)
    b.lowrank_exact(rank, eps_prior=2.0, lam=lam, std=std)
    p = 2 * k + 6
    X = synth.gaussian_block(11, p, n).astype(np.float64)
    Vr, lr = ob.rsvd_single_pass(ob.probe_block(X, S, Y, B0), X, rank)
    assert np.allclose(lam.cpu().numpy(), lr, rtol=1e-4, atol=1e-6 * np.abs(lr).max())
    assert rel(std.cpu().numpy(), ob.posterior_std(Vr, lr, B0, eps=2.0)) < 1e-4


def test_exact_and_randomized_agree_on_the_gpu():
    n, k = 50000, 15
    b, S, Y, B0 = store(n, k)
    rank = 2 * k
    le = torch.zeros(rank, dtype=torch.float64, device=DEV)
    lr = torch.zeros(rank, dtype=torch.float64, device=DEV)
    b.lowrank_exact(rank, lam=le)
    b.lowrank_invhess(2 * k + 8, rank, seed=9, lam=lr)
    a, c = le.cpu().numpy(), lr.cpu().numpy()
    assert np.allclose(a, c, rtol=1e-3, atol=1e-5 * np.abs(a).max())


def test_lowrank_ill_conditioned_history():
    """Nearly parallel model updates (as in a converging inversion) make the
    probe block E ill-conditioned; the rank-revealing basis must pivot
    correctly and the resolved eigenvalues match Algorithm 3 in FP64 with
    the same (device Philox) probes."""
    n, k, seed = 20000, 12, 2020
    rng = np.random.default_rng(31)
    A = rng.uniform(1.0, 10.0, n)
    base = rng.standard_normal(n) * 1e-2
    S = np.stack([base + 10.0 ** (-0.4 * i) * 1e-2 * rng.standard_normal(n) for i in range(k)])
    Y = S * A + 1e-6 * rng.standard_normal((k, n))
    B0 = (1.0 / A) * rng.uniform(0.5, 2.0, n)
    S, Y, B0 = S.astype(np.float32), Y.astype(np.float32), B0.astype(np.float32)
    b = gb.Bfgs(n, k, t32(B0))
    for i in range(k):
        b.update(t32(S[i]), t32(Y[i]))
    p = rank = k
    lam = torch.zeros(rank, dtype=torch.float64, device=DEV)
    b.lowrank_invhess(p, rank, seed=seed, eps_prior=1.0, lam=lam)
    X = philox.gaussian_block(seed, p, n)
    E = ob.probe_block(X, S.astype(np.float64), Y.astype(np.float64), B0.astype(np.float64))
    sv = np.linalg.svd(E, compute_uv=False)
    assert sv[-1] / sv[0] < 1e-3          # the case this test is about
    _, lr = ob.rsvd_single_pass(E, X, rank)
    lg = lam.cpu().numpy()
    big = np.abs(lr) >= 1e-3 * np.abs(lr).max()
    assert np.allclose(lg[big], lr[big], rtol=1e-2), (lg, lr)
    assert np.all(np.abs(lg[~big]) <= 2e-3 * np.abs(lr).max())


@pytest.mark.parametrize("n,k,p,rank", [(5000, 12, 16, 10), (30011, 20, 44, 40)])
def test_two_pass_matches_oracle_two_pass(n, k, p, rank):
    """The Rayleigh-Ritz (two-pass) variant of Algorithm 3 against the
    oracle's, on the same probes: eigenvalues 1e-4, eigenvectors by the
    gap-scaled angle bound; with p >= 2k probes (second case) both are the
    exact eigendecomposition of B_{n+1} - B0."""
    b, S, Y, B0 = store(n, k)
    X = synth.gaussian_block(8, p, n)
    V = torch.zeros(rank, n, device=DEV)
    lam = torch.zeros(rank, dtype=torch.float64, device=DEV)
    std = torch.zeros(n, device=DEV)
    b.lowrank_twopass(p, rank, eps_prior=1.5, X=t32(X), V=V, lam=lam, std=std)
    apply = lambda M: ob.probe_block(np.asarray(M, np.float64), S, Y, B0)
    Vr, lr = ob.rsvd_two_pass(apply, X.astype(np.float64), rank)
    _, lam_all = ob.rsvd_two_pass(apply, X.astype(np.float64), p)
    lg = lam.cpu().numpy()
    assert np.allclose(lg, lr, rtol=1e-4, atol=1e-6 * np.abs(lr).max())
    _check_vectors(V.cpu().numpy(), Vr, lam_all, rank)
    assert rel(std.cpu().numpy(), ob.posterior_std(Vr, lr, B0, eps=1.5)) < 1e-4
    if p >= 2 * k:
        Ve = torch.zeros(rank, n, device=DEV)
        le = torch.zeros(rank, dtype=torch.float64, device=DEV)
        b.lowrank_exact(rank, eps_prior=1.5, V=Ve, lam=le)
        assert np.allclose(lg, le.cpu().numpy(), rtol=1e-4, atol=1e-6 * np.abs(lr).max())
