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
