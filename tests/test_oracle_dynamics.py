"""Dynamic pins of the FP64 oracle:

* a closed box conserves the discrete energy of the central-difference
  scheme exactly (to rounding);
* the adjoint recurrence is the exact transpose of the forward map
  (dot-product test, with Stacey edges and a free surface);
* the gradient equals central finite differences of the misfit along random
  model perturbations: the difference shrinks as eps^2 and is below 1e-6 at
  a relative step of 1e-5;
* the 2-D full-space point-force response matches the closed-form
  frequency-domain Green's tensor (Hankel functions) convolved with the
  Ricker wavelet.
"""
import numpy as np
import pytest

from oracle import sem

RNG = np.random.default_rng(99)


def _homog(m, vp=3000.0, vs=1732.0, rho=2500.0):
    return (np.full((m.nz, m.nx), rho), np.full((m.nz, m.nx), vp), np.full((m.nz, m.nx), vs))


def test_energy_conserved_in_closed_box():
    m = sem.Mesh(8, 6, 25.0)
    st = sem.Setup(m, 5e-4, 500, np.array([[40.0, 30.0]]), free_top=1, absorb=0)
    x, z = m.coords()
    rho = 2400 + 200 * np.sin(x / 70.0)
    vp = 3000 + 300 * np.cos(z / 50.0)
    vs = vp / 1.8
    model = (rho, vp, vs)
    f = m.source_vector(97.0, 61.0, 0, 1e6)
    stf = sem.ricker(st.nt, st.dt, 25.0, 0.05)
    stf[120:] = 0.0                                   # source off after step 119
    _, uh, _ = st.forward(model, f, stf, keep=True)
    lam, mu = sem.lame(*model)
    M = m.mass(rho)[..., None]
    E = []
    for n in range(125, st.nt):
        du = (uh[n + 1] - uh[n]) / st.dt
        E.append(0.5 * np.sum(du * M * du) + 0.5 * np.sum(uh[n + 1] * m.stiffness(lam, mu, uh[n])))
    E = np.array(E)
    assert E[0] > 0
    assert np.max(np.abs(E - E[0])) / E[0] < 1e-12


def test_adjoint_dot_product():
    """sum_k d_k . P u_k == dt^2 sum_n stf[n] f . lam_n  (forward source f stf,
    adjoint source P^T d), Stacey edges + free surface, heterogeneous model."""
    m = sem.Mesh(7, 5, 20.0)
    rec = np.stack([RNG.uniform(0, 140, 6), RNG.uniform(0, 100, 6)], 1)
    st = sem.Setup(m, 4e-4, 300, rec, free_top=1, absorb=1)
    x, z = m.coords()
    model = (2300 + 100 * np.cos(x / 40), 2800 + 200 * np.sin(z / 30 + x / 90), 1600 + 100 * np.cos(z / 25))
    f = RNG.standard_normal((m.nz, m.nx, 2))
    stf = RNG.standard_normal(st.nt + 1)
    d = RNG.standard_normal((st.nrec, 2, st.nt))
    seis = st.forward(model, f, stf)
    lam = st.adjoint(model, d)
    lhs = np.sum(d * seis)
    rhs = st.dt ** 2 * sum(stf[n] * np.sum(f * lam[n]) for n in range(1, st.nt))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-300) * 10
    assert abs(lhs) > 0


def _fd_setup():
    m = sem.Mesh(8, 6, 25.0)
    rec = np.stack([np.linspace(0, 200, 9), np.full(9, 5.0)], 1)
    st = sem.Setup(m, 5e-4, 420, rec, free_top=1, absorb=1)
    x, z = m.coords()
    true = (2500 + 150 * np.exp(-((x - 110) ** 2 + (z - 80) ** 2) / 900),
            3000 + 250 * np.exp(-((x - 90) ** 2 + (z - 70) ** 2) / 1200),
            1732 + 150 * np.exp(-((x - 120) ** 2 + (z - 90) ** 2) / 800))
    start = _homog(m)
    srcs = [dict(x=60.0, z=15.0, type=0, f0=25.0, t0=0.048, amp=1e7),
            dict(x=150.0, z=15.0, type=0, f0=25.0, t0=0.048, amp=1e7)]
    obs = []
    for s in srcs:
        fv, stf = st.source(s)
        obs.append(st.forward(true, fv, stf))
    return st, start, srcs, obs


def _misfit(st, model, srcs, obs):
    f = 0.0
    for s, d in zip(srcs, obs):
        fv, stf = st.source(s)
        f += sem.misfit(st.dt, st.forward(model, fv, stf), d)
    return f


@pytest.mark.slow
def test_gradient_matches_central_differences():
    st, m0, srcs, obs = _fd_setup()
    f0, g, _ = sem.misfit_gradient(st, m0, srcs, obs)
    assert f0 > 0
    m = st.mesh
    x, z = m.coords()
    worst = 0.0
    for trial in range(6):
        # smooth random perturbation (Gaussian bumps incl. the boundary) on one
        # or all parameters, relative size 1e-3
        bump = np.zeros((3, m.nz, m.nx))
        for c in range(3):
            cx, cz = RNG.uniform(0, m.nex * m.h), RNG.uniform(0, m.nez * m.h)
            bump[c] = np.exp(-((x - cx) ** 2 + (z - cz) ** 2) / (2 * 40.0 ** 2))
        if trial < 3:
            keep = np.zeros(3); keep[trial] = 1
            bump *= keep[:, None, None]
        dm = bump * np.stack(m0)
        an = float(np.sum(g * dm))

        def fd(eps):
            fp = _misfit(st, tuple(np.stack(m0) + eps * dm), srcs, obs)
            fm = _misfit(st, tuple(np.stack(m0) - eps * dm), srcs, obs)
            return (fp - fm) / (2 * eps)
        # a central difference converges as eps^2 to the exact derivative: the
        # error quarters when eps halves, and at eps = 1e-5 it is below 1e-6
        e1 = (fd(1e-3) - an) / an
        e2 = (fd(5e-4) - an) / an
        assert 3.6 < e1 / e2 < 4.4, (e1, e2)
        worst = max(worst, abs((fd(1e-5) - an) / an))
    assert worst < 1e-6


def _green_2d(omega, dx, dz, vp, vs, rho):
    """Frequency-domain 2-D Green's tensor for a line force (e^{-i w t}):
    G_ij = [k_s^2 g_s delta_ij + d_i d_j (g_s - g_p)] / (rho w^2),
    g_c = (i/4) H0^(1)(k_c r) (Helmholtz decomposition of the elastic
    wave operator)."""
    from scipy.special import hankel1
    r = np.hypot(dx, dz)
    xh = np.array([dx, dz]) / r
    G = np.zeros((len(omega), 2, 2), dtype=complex)
    for c, sign in ((vs, 1.0), (vp, -1.0)):
        k = omega / c
        kr = k * r
        g = 0.25j * hankel1(0, kr)
        gp = -0.25j * k * hankel1(1, kr)
        gpp = -0.25j * k * k * (hankel1(0, kr) - hankel1(1, kr) / kr)
        for i in range(2):
            for j in range(2):
                dd = gpp * xh[i] * xh[j] + gp * ((1.0 if i == j else 0.0) / r - xh[i] * xh[j] / r)
                G[:, i, j] += sign * dd
                if i == j and sign > 0:
                    G[:, i, j] += k * k * g
    return G / (rho * omega[:, None, None] ** 2)


def _green_error(h, dt, L=1200.0, f0=15.0, T=0.31):
    """Largest relative L2 difference between the oracle's point-force
    records and the closed-form Green's tensor convolved with the Ricker
    wavelet, over two force directions, three receivers 250 m from the
    source and both components (window ends before boundary reflections)."""
    ne = int(round(L / h))
    m = sem.Mesh(ne, ne, h)
    xs = zs = L / 2
    vp, vs, rho = 3000.0, 1732.0, 2500.0
    t0, nt = 1.2 / f0, int(round(T / dt))
    offs = np.array([[250.0, 0.0], [0.0, 250.0], [177.0, 177.0]])
    st = sem.Setup(m, dt, nt, offs + [xs, zs], free_top=0, absorb=1)
    model = _homog(m, vp, vs, rho)
    nfft = 1 << int(np.ceil(np.log2(6.0 / dt)))
    omega = 2 * np.pi * np.fft.rfftfreq(nfft, dt)
    tt = np.arange(nfft) * dt
    arg = (np.pi * f0 * (tt - t0)) ** 2
    F = np.fft.rfft((1 - 2 * arg) * np.exp(-arg))
    worst = 0.0
    for ftype, j in ((1, 0), (2, 1)):
        seis = st.forward(model, m.source_vector(xs, zs, ftype, 1e9), sem.ricker(nt, dt, f0, t0))
        for r, (dx, dz) in enumerate(offs):
            G = np.zeros((len(omega), 2, 2), dtype=complex)
            G[1:] = _green_2d(omega[1:], dx, dz, vp, vs, rho)
            ana = [np.fft.irfft(np.conj(G[:, i, j]) * F * 1e9, nfft)[1:nt + 1] for i in range(2)]
            scale = max(np.linalg.norm(u) for u in ana)
            worst = max(worst, max(np.linalg.norm(seis[r, i] - ana[i]) / scale for i in range(2)))
    return worst


@pytest.mark.slow
def test_green_function_error_converges_under_refinement():
    """The point-force comparison converges as the scheme's orders say:
    halving dt on a fine mesh quarters the error (central differences,
    second order in time), and on a short time step going from 60 m to 40 m
    elements cuts it by more than (3/2)^3 (degree-4 GLL elements converge
    at least that fast; measured order ~5)."""
    e_dt1, e_dt2 = _green_error(20.0, 4e-4), _green_error(20.0, 2e-4)
    assert 3.5 < e_dt1 / e_dt2 < 4.6, (e_dt1, e_dt2)
    e_h1, e_h2 = _green_error(60.0, 1e-4), _green_error(40.0, 1e-4)
    assert e_h1 / e_h2 > 1.5 ** 3, (e_h1, e_h2)
    assert e_dt2 < 5e-4 and e_h2 < 1e-2


@pytest.mark.slow
def test_point_force_matches_closed_form_green_function():
    h, ne = 20.0, 60
    m = sem.Mesh(ne, ne, h)
    L = ne * h
    xs = zs = L / 2
    vp, vs, rho = 3000.0, 1732.0, 2500.0
    dt, f0 = 4e-4, 15.0
    t0 = 1.2 / f0
    nt = 775                                   # ends before boundary returns
    offs = np.array([[250.0, 0.0], [0.0, 250.0], [177.0, 177.0], [-120.0, 220.0]])
    st = sem.Setup(m, dt, nt, offs + [xs, zs], free_top=0, absorb=1)
    model = _homog(m, vp, vs, rho)
    nfft = 16384
    omega = 2 * np.pi * np.fft.rfftfreq(nfft, dt)
    tt = np.arange(nfft) * dt
    a = (np.pi * f0 * (tt - t0)) ** 2
    wav = (1 - 2 * a) * np.exp(-a)
    Fnp = np.fft.rfft(wav)
    for ftype, j in ((1, 0), (2, 1)):
        fvec = m.source_vector(xs, zs, ftype, 1e9)
        stf = sem.ricker(nt, dt, f0, t0)
        seis = st.forward(model, fvec, stf)
        for r, (dx, dz) in enumerate(offs):
            G = np.zeros((len(omega), 2, 2), dtype=complex)
            G[1:] = _green_2d(omega[1:], dx, dz, vp, vs, rho)
            # samples at t_1..t_nt of the two displacement components
            ana = [np.fft.irfft(np.conj(G[:, i, j]) * Fnp * 1e9, nfft)[1:nt + 1] for i in range(2)]
            scale = max(np.linalg.norm(u) for u in ana)
            for i in range(2):
                err = np.linalg.norm(seis[r, i] - ana[i]) / scale
                assert err < 5e-3, (ftype, r, i, err)
