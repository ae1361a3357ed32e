"""Pins of the oracle's diagonal-Hessian (preconditioner) maps.

* Eqs. A21/A22 closed forms: the factors 8 rho^2 alpha^2, 16 rho^2 beta^2
  and 4 rho^2 beta^2 are checked against a numerical derivative of the
  stiffness matrix C(alpha, beta, rho) of Eq. A7 applied to strain vectors.
* The time integrals (ref_precond_sums) on histories with a known constant
  velocity gradient, where every integral has a closed form.
* The second difference used for the receiver-field acceleration equals
  the Newmark acceleration of a forward run.
* Gaussian smoothing keeps constants, stays within the data range and turns
  an interior spike into the expected Gaussian.
"""
import numpy as np

from oracle import sem

RNG = np.random.default_rng(7)


def _C(alpha, beta, rho):
    """Isotropic stiffness of Eq. A7 in the (alpha, beta, rho) parametrisation,
    ordering (xx, zz, xz): lambda + 2 mu = rho alpha^2, mu = rho beta^2."""
    mu = rho * beta ** 2
    lam = rho * alpha ** 2 - 2 * mu
    return np.array([[lam + 2 * mu, lam, 0.0], [lam, lam + 2 * mu, 0.0], [0.0, 0.0, mu]])


def _dC(which, alpha, beta, rho, eps=1e-6):
    p = dict(alpha=alpha, beta=beta, rho=rho)
    hp, hm = dict(p), dict(p)
    hp[which] += eps * p[which]
    hm[which] -= eps * p[which]
    return (_C(**hp) - _C(**hm)) / (2 * eps * p[which])


def test_a21_a22_factors_from_numerical_dC():
    alpha, beta, rho = 3100.0, 1800.0, 2400.0
    one = np.ones((1, 1))
    model = (rho * one, alpha * one, beta * one)
    W = one
    for _ in range(5):
        # strain-rate vectors D v = (dx vx, dz vz, dz vx + dx vz) of the two fields
        dv = RNG.standard_normal(3)
        db = RNG.standard_normal(3)
        Ka = _dC("alpha", alpha, beta, rho) @ dv
        Kab = _dC("alpha", alpha, beta, rho) @ db
        Kb = _dC("beta", alpha, beta, rho) @ dv
        Kbb = _dC("beta", alpha, beta, rho) @ db
        S = np.zeros((4, 1, 1))
        S[1] = (dv[0] + dv[1]) * (db[0] + db[1])
        S[2] = dv[0] * db[0] + dv[1] * db[1]
        S[3] = dv[2] * db[2]
        H = sem.precond_maps(model, W, S, kind=3)
        # signs of the two beta terms agree only if the product has one sign per term;
        # compare the unsigned pieces term by term as Eq. A22 does
        assert np.isclose(H[1, 0, 0], abs(Ka @ Kab), rtol=1e-7)
        dCb = _dC("beta", alpha, beta, rho)
        t1 = (dCb[:2, :2] @ dv[:2]) @ (dCb[:2, :2] @ db[:2])   # normal-stress part
        t2 = (dCb[2, 2] * dv[2]) * (dCb[2, 2] * db[2])          # shear part
        assert np.isclose(t1 + t2, Kb @ Kbb, rtol=1e-7)
        assert np.isclose(H[2, 0, 0], abs(t1) + abs(t2), rtol=1e-7)
        # P3 (same field twice): the absolute values change nothing
        S[1] = (dv[0] + dv[1]) ** 2
        S[2] = dv[0] ** 2 + dv[1] ** 2
        S[3] = dv[2] ** 2
        H = sem.precond_maps(model, W, S, kind=3)
        assert np.isclose(H[1, 0, 0], Ka @ Ka, rtol=1e-7)
        assert np.isclose(H[2, 0, 0], Kb @ Kb, rtol=1e-7)


def test_precond_sums_constant_velocity_gradient():
    """u_n = n dt (a x + b z, c x + d z): v is constant in space-time, so
    S1 = T W (a+d)^2, S2 = T W (a^2 + d^2), S3 = T W (b+c)^2 with T = nt dt;
    a constant acceleration q gives S0 = nt dt |q|^2."""
    m = sem.Mesh(5, 3, 20.0)
    nt, dt = 17, 1e-3
    st = sem.Setup(m, dt, nt, np.array([[10.0, 10.0]]))
    x, z = m.coords()
    a, b, c, d = 0.3, -0.7, 1.1, 0.4
    v = np.stack([a * x + b * z, c * x + d * z], -1)
    u = np.stack([n * dt * v for n in range(nt + 1)])
    q = np.array([2.0, -3.0])
    acc = np.broadcast_to(q, u.shape).copy()
    S = st.precond_sums(u, acc, u, acc)
    W = m.measure()
    T = nt * dt
    assert np.allclose(S[0], T * (q @ q), rtol=1e-12)
    assert np.allclose(S[1], T * W * (a + d) ** 2, rtol=1e-10)
    assert np.allclose(S[2], T * W * (a * a + d * d), rtol=1e-10)
    assert np.allclose(S[3], T * W * (b + c) ** 2, rtol=1e-10)
    # cross terms with a second field with other gradients
    a2, b2, c2, d2 = -0.2, 0.5, 0.9, 1.3
    v2 = np.stack([a2 * x + b2 * z, c2 * x + d2 * z], -1)
    u2 = np.stack([n * dt * v2 for n in range(nt + 1)])
    S = st.precond_sums(u, acc, u2, -acc)
    assert np.allclose(S[0], -T * (q @ q), rtol=1e-12)
    assert np.allclose(S[1], T * W * (a + d) * (a2 + d2), rtol=1e-10)
    assert np.allclose(S[2], T * W * (a * a2 + d * d2), rtol=1e-10)
    assert np.allclose(S[3], T * W * (b + c) * (b2 + c2), rtol=1e-10)


def test_second_difference_matches_newmark_acceleration():
    m = sem.Mesh(6, 4, 25.0)
    st = sem.Setup(m, 5e-4, 200, np.array([[50.0, 5.0]]))
    x, z = m.coords()
    model = (2500 + 0 * x, 3000 + 100 * np.sin(x / 50), 1700 + 0 * x)
    fv, stf = st.source(dict(x=75.0, z=30.0, type=0, f0=30.0, t0=0.04, amp=1e6))
    _, uh, ah = st.forward(model, fv, stf, keep=True)
    a2 = sem.accel_from_hist(uh, st.dt)
    scale = np.max(np.abs(ah))
    # interior (away from the Stacey edges the damping term is zero and the
    # second difference is exactly the acceleration)
    assert np.max(np.abs(a2[1:-1, 1:-1, 1:-1] - ah[1:-1, 1:-1, 1:-1])) < 1e-7 * scale


def test_smoothing_constant_range_and_spike():
    m = sem.Mesh(16, 16, 20.0)
    c = np.full((m.nz, m.nx), 3.5)
    assert np.allclose(m.smooth(c, 40.0), 3.5, rtol=1e-13)
    f = RNG.uniform(-1, 2, (m.nz, m.nx))
    s = m.smooth(f, 30.0)
    assert s.min() >= f.min() - 1e-12 and s.max() <= f.max() + 1e-12
    # spike far (> 6 sigma) from every edge: the normalising sum is the full
    # Gaussian integral 2 pi sigma^2 up to quadrature error
    m = sem.Mesh(24, 24, 20.0)
    spike = np.zeros((m.nz, m.nx))
    iz, ix = m.nz // 2, m.nx // 2
    spike[iz, ix] = 1.0
    sig = 30.0
    out = m.smooth(spike, sig)
    x, z = m.coords()
    W = m.measure()
    expect = W[iz, ix] * np.exp(-((x - x[iz, ix]) ** 2 + (z - z[iz, ix]) ** 2) / (2 * sig ** 2)) \
        / (2 * np.pi * sig ** 2)
    centre = np.hypot(x - x[iz, ix], z - z[iz, ix]) < 40
    assert np.allclose(out[centre], expect[centre], rtol=1e-3)


def test_smooth_damp_invert_median_rule():
    m = sem.Mesh(4, 3, 20.0)
    st = sem.Setup(m, 1e-3, 10, np.array([[10.0, 10.0]]))
    H = np.stack([np.full((m.nz, m.nx), v) for v in (1.0, 2.0, 4.0)])
    Hs, B0 = sem.smooth_damp_invert(st, H, 30.0, damp_factor=0.5)
    for c, v in enumerate((1.0, 2.0, 4.0)):
        assert np.allclose(Hs[c], v)
        assert np.allclose(B0[c], 1.0 / (v + 0.5 * v))


def _receiver_case():
    m = sem.Mesh(7, 5, 20.0)
    rng = np.random.default_rng(21)
    rec = np.stack([rng.uniform(5, 135, 5), rng.uniform(0, 95, 5)], 1)
    st = sem.Setup(m, 4e-4, 260, rec, free_top=1, absorb=1)
    x, z = m.coords()
    model = (2300 + 100 * np.cos(x / 40), 2900 + 200 * np.sin(z / 30 + x / 90), 1650 + 100 * np.cos(z / 25))
    f = m.source_vector(63.0, 41.0, 0, 1e6)
    stf = rng.standard_normal(st.nt + 1)          # no symmetry a time shift could hide behind
    seis = st.forward(model, f, stf)
    return st, model, f, stf, seis


def test_receiver_field_level_and_time_alignment_by_duality():
    """The receiver wavefield of Eqs. 6 and 8 is the backward simulation
    driven by the synthetics s(m0) (after Eq. A22).  The scheme's duality
    (its adjoint is the same recurrence run backwards) fixes both its level
    and which step each returned level belongs to: with s = P u the records
    of the source f stf[n] and lam_n the returned receiver field,
        dt^2 sum_{n=1}^{nt-1} stf[n] f . lam_n = dt sum_k |s_k|^2.
    A missing dt factor, or lam shifted by one step, breaks the identity."""
    st, model, f, stf, seis = _receiver_case()
    lam, _ = sem.receiver_field(st, model, seis)
    assert lam.shape[0] == st.nt + 1
    rhs = st.dt * np.sum(seis * seis)
    lhs = st.dt ** 2 * sum(stf[n] * np.sum(f * lam[n]) for n in range(1, st.nt))
    assert rhs > 0 and abs(lhs - rhs) <= 1e-12 * rhs
    for shift in (-1, 1):
        moved = st.dt ** 2 * sum(stf[n] * np.sum(f * lam[n + shift]) for n in range(1, st.nt))
        assert abs(moved - rhs) > 1e-2 * rhs


def test_receiver_field_acceleration_is_the_recurrence_acceleration():
    """P2/P4 pair the forward acceleration a_n with the receiver field's
    acceleration at the same step n.  Where the Stacey damping is zero the
    backward recurrence reads M (lam_{n+1} - 2 lam_n + lam_{n-1}) =
    -dt^2 K lam_n + P^T g_n (g_n = dt s_n, its driving term), so the stored
    acceleration at index n must equal M^-1 (-K lam_n + P^T s_n / dt),
    built here from the oracle's stiffness, mass and receiver weights."""
    st, model, f, stf, seis = _receiver_case()
    lam, acc = sem.receiver_field(st, model, seis)
    m = st.mesh
    rho = model[0]
    M = m.mass(rho)[..., None]
    C = m.stacey(*model, free_top=st.free_top, absorb=st.absorb)
    lam_, mu_ = sem.lame(*model)
    free = C == 0.0
    scale = np.max(np.abs(acc))
    for n in (1, 37, 130, st.nt - 1, st.nt):
        force = -m.stiffness(lam_, mu_, lam[n])
        flat = force.reshape(-1, 2)
        for r in range(st.nrec):
            for c in range(2):
                np.add.at(flat[:, c], st.ridx[r], st.rw[r] * seis[r, c, n - 1] / st.dt)
        expect = force / M
        assert np.max(np.abs(acc[n][free] - expect[free])) <= 1e-9 * scale, n


def test_p1_homogeneous_full_space_closed_form():
    """P1 (Eq. 5, the forward field's int a.a dt, times the node's quadrature
    measure) for a point force in a homogeneous full space against the same
    integral of the closed-form field: the acceleration is -omega^2 times the
    2-D Green's tensor convolved with the Ricker wavelet (the tensor the
    point-force pin of test_oracle_dynamics uses), summed over the same
    samples t_1..t_nt.  Nodes 150 m from the source; the window ends before
    the first boundary reflection reaches them.  Loose: 1%."""
    from test_oracle_dynamics import _green_2d, _homog
    h, ne, dt, f0, T = 20.0, 40, 4e-4, 25.0, 0.2
    L = ne * h
    xs = zs = L / 2
    vp, vs, rho = 3000.0, 1732.0, 2500.0
    t0, nt = 1.2 / f0, int(round(T / dt))
    m = sem.Mesh(ne, ne, h)
    st = sem.Setup(m, dt, nt, np.array([[xs, zs]]), free_top=0, absorb=1)
    model = _homog(m, vp, vs, rho)
    x, z = m.coords()
    W = m.measure()
    nfft = 1 << int(np.ceil(np.log2(6.0 / dt)))
    omega = 2 * np.pi * np.fft.rfftfreq(nfft, dt)
    tt = np.arange(nfft) * dt
    arg = (np.pi * f0 * (tt - t0)) ** 2
    F = np.fft.rfft((1 - 2 * arg) * np.exp(-arg))
    for ftype, j in ((1, 0), (2, 1)):
        P1 = sem.precond_raw(st, model, [dict(x=xs, z=zs, type=ftype, f0=f0, t0=t0, amp=1e9)], 1)
        assert np.array_equal(P1[0], P1[1]) and np.array_equal(P1[0], P1[2])
        for dx, dz in ((150.0, 0.0), (0.0, 150.0), (-110.0, 110.0), (130.0, -70.0)):
            ix = int(np.argmin(np.abs(x[0] - (xs + dx))))
            iz = int(np.argmin(np.abs(z[:, 0] - (zs + dz))))
            G = np.zeros((len(omega), 2, 2), dtype=complex)
            G[1:] = _green_2d(omega[1:], x[iz, ix] - xs, z[iz, ix] - zs, vp, vs, rho)
            acc = [np.fft.irfft(-omega ** 2 * np.conj(G[:, i, j]) * F * 1e9, nfft)[1:nt + 1] for i in range(2)]
            expect = dt * sum(np.sum(a * a) for a in acc)
            got = P1[0, iz, ix] / W[iz, ix]
            assert abs(got / expect - 1) < 1e-2, (ftype, dx, dz, got, expect)
