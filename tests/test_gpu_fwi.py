"""The FWI driver around the C ABI (Algorithm 1 directions through the
compact apply, Armijo steps) and the post-convergence uncertainty step."""
import numpy as np
import pytest

from oracle import bfgs as ob

torch = pytest.importorskip("torch")
from paper_2009_12663_gb300 import experiments  # noqa: E402
from paper_2009_12663_gb300.fwi import Problem, fwi, pack, preconditioner  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    return experiments.build(nex=40, nez=10, nshot=3, nt=900, f0=12.0)


def test_bfgs_reduces_misfit_and_lbfgs_with_full_memory_is_bfgs(small):
    mesh, ids, d_obs, true, start = small
    prob = Problem(mesh, ids, d_obs)
    _, h_full, store = fwi(prob, start, 4)
    _, h_lbfgs, _ = fwi(prob, start, 4, memory=10)
    rel = [h["rel_misfit"] for h in h_full]
    assert rel[-1] < 0.9 * rel[0]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(rel, rel[1:]))
    assert [h["misfit"] for h in h_full] == [h["misfit"] for h in h_lbfgs]
    assert store.count >= 2


def test_p4_preconditioned_run_and_uncertainty_maps(small):
    mesh, ids, d_obs, true, start = small
    prob = Problem(mesh, ids, d_obs)
    B0 = preconditioner(mesh, ids, start, 4, sigma=100.0)
    assert torch.isfinite(B0).all() and (B0 > 0).all()
    stored = []
    m, hist, store = fwi(prob, start, 4, B0=B0, pairs_out=stored)
    rel = [h["rel_misfit"] for h in hist]
    assert rel[-1] < rel[0] and all(b <= a * (1 + 1e-12) for a, b in zip(rel, rel[1:]))
    k = store.count
    p = r = k
    V = torch.zeros(r, store.n, device=start.device)
    lam = torch.zeros(r, dtype=torch.float64, device=start.device)
    std = torch.zeros(store.n, device=start.device)
    store.lowrank_invhess(p, r, seed=1, eps_prior=1.0, V=V, lam=lam, std=std)
    s = std.cpu().numpy()
    assert np.isfinite(s).all() and (s >= 0).all()
    # with no data information the posterior std would be sqrt(eps B0)
    # (Eqs. 12-14); the BFGS history must change it
    b0 = B0[1:].reshape(-1).cpu().numpy()
    assert np.abs(s - np.sqrt(b0)).max() > 1e-3 * np.sqrt(b0).max()
    assert np.isfinite(lam.cpu().numpy()).all()
    # the eigenvalues against Algorithm 3 in FP64 on exactly the stored FP32
    # pairs and probes; this history is ill-conditioned (singular values of
    # E spread over several decades), so only directions an FP32 block
    # resolves are compared
    assert len(stored) == store.count
    S = np.stack([a.double().cpu().numpy() for a, _ in stored])
    Y = np.stack([b.double().cpu().numpy() for _, b in stored])
    X = np.random.default_rng(3).standard_normal((p, store.n)).astype(np.float32)
    b0v = pack(B0, prob.mask).double().cpu().numpy()
    store.lowrank_invhess(p, r, eps_prior=1.0, X=torch.tensor(X, device=start.device), lam=lam)
    X64 = X.astype(np.float64)
    _, lr = ob.rsvd_single_pass(ob.probe_block(X64, S, Y, b0v), X64, r)
    lg = lam.cpu().numpy()
    big = np.abs(lr) >= 1e-3 * np.abs(lr).max()
    assert np.allclose(lg[big], lr[big], rtol=1e-2), (lg, lr)
    assert np.all(np.abs(lg[~big]) <= 2e-3 * np.abs(lr).max())


def test_uncertainty_structure_on_a_real_history(small):
    """Section 3.2 in kind, on the pairs of a P4-preconditioned inversion:
    the retrieved inverse Hessian's low-rank part B_{n+1} - B0 = W M W^T
    (W = [S, B0 Y]) has rank at most 2k (not k, as Section 2.3 states);
    with p > 2k probes the randomized eigendecomposition (single and two
    pass) returns no resolved eigenvalue beyond 2k, its resolved spectrum
    matches the exact decomposition, and the eigenvectors are orthonormal."""
    mesh, ids, d_obs, true, start = small
    prob = Problem(mesh, ids, d_obs)
    B0 = preconditioner(mesh, ids, start, 4, sigma=100.0)
    m, hist, store = fwi(prob, start, 5, B0=B0)
    k = store.count
    assert k >= 3
    dev = start.device
    m2 = 2 * k
    Ve = torch.zeros(m2, store.n, device=dev)
    le = torch.zeros(m2, dtype=torch.float64, device=dev)
    store.lowrank_exact(m2, eps_prior=1.0, V=Ve, lam=le)
    le = le.cpu().numpy()
    top = np.abs(le).max()
    resolved = np.abs(le) >= 1e-3 * top
    assert resolved.sum() <= m2
    Vh = Ve.double().cpu().numpy()[resolved]
    assert np.abs(Vh @ Vh.T - np.eye(len(Vh))).max() < 1e-4
    p = m2 + 6
    for method in ("lowrank_invhess", "lowrank_twopass"):
        V = torch.zeros(p, store.n, device=dev)
        lam = torch.zeros(p, dtype=torch.float64, device=dev)
        getattr(store, method)(p, p, seed=11, eps_prior=1.0, V=V, lam=lam)
        lg = lam.cpu().numpy()
        # nothing resolved beyond 2k directions
        assert np.all(np.abs(lg[m2:]) <= 2e-3 * top), (method, lg)
        # the resolved eigenvalues are the exact ones
        assert np.allclose(lg[:m2][resolved], le[resolved], rtol=1e-2), (method, lg[:m2], le)
        Vg = V.double().cpu().numpy()[:m2][resolved]
        assert np.abs(Vg @ Vg.T - np.eye(len(Vg))).max() < 1e-3, method
