"""Pins of the FP64 spectral-element oracle against facts the mathematics
fixes independently of the oracle's own code: polynomial exactness of GLL
quadrature and differentiation, rigid-body modes and symmetry of K, the
exact strain energy and boundary traction of a linear displacement field,
moment-tensor moments of the explosive source, polynomial reproduction by
the receiver interpolation, and Ricker wavelet zeros."""
import numpy as np
import pytest

from oracle import sem

RNG = np.random.default_rng(1234)


def test_gll_quadrature_exact_to_degree_7():
    xi, w, _ = sem.gll()
    assert abs(w.sum() - 2.0) < 1e-15
    for k in range(8):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * xi ** k) - exact) < 1e-14
    # degree 8 is not integrated exactly by 5-point Lobatto (2N-3 = 7)
    assert abs(np.sum(w * xi ** 8) - 2.0 / 9) > 1e-4


def test_gll_derivative_matrix_exact_to_degree_4():
    xi, _, D = sem.gll()
    for k in range(5):
        f = xi ** k
        df = k * xi ** (k - 1) if k > 0 else np.zeros(5)
        assert np.allclose(D @ f, df, atol=1e-13)


def test_lagrange_partition_of_unity_and_cardinality():
    xi, _, _ = sem.gll()
    for s in np.linspace(-1, 1, 13):
        l, dl = sem.lagrange(s)
        assert abs(l.sum() - 1) < 1e-14 and abs(dl.sum()) < 1e-12
    for i in range(5):
        l, _ = sem.lagrange(xi[i])
        assert np.allclose(l, np.eye(5)[i], atol=1e-14)


def _rand_material(m):
    lam = RNG.uniform(1e9, 3e9, (m.nz, m.nx))
    mu = RNG.uniform(0.5e9, 2e9, (m.nz, m.nx))
    return lam, mu


def test_stiffness_rigid_body_modes_vanish():
    m = sem.Mesh(5, 4, 30.0)
    lam, mu = _rand_material(m)
    x, z = m.coords()
    scale = 1e9 * 1e-3
    for u in (np.stack([np.ones_like(x), 0 * x], -1),
              np.stack([0 * x, np.ones_like(x)], -1),
              np.stack([-z, x], -1) * 1e-3):           # infinitesimal rotation
        Ku = m.stiffness(lam, mu, u)
        assert np.max(np.abs(Ku)) < 1e-9 * scale * m.h


def test_stiffness_symmetric():
    m = sem.Mesh(4, 3, 25.0)
    lam, mu = _rand_material(m)
    u = RNG.standard_normal((m.nz, m.nx, 2))
    v = RNG.standard_normal((m.nz, m.nx, 2))
    a = np.sum(v * m.stiffness(lam, mu, u))
    b = np.sum(u * m.stiffness(lam, mu, v))
    assert abs(a - b) <= 1e-12 * abs(a)


def test_stiffness_linear_field_energy_and_traction():
    """u = (a x + b z, c x + d z) in a homogeneous medium has constant strain:
    u^T K u = area * [(lam+2mu)(a^2+d^2) + 2 lam a d + mu (b+c)^2], the
    interior force vanishes and the boundary force is the traction sigma.n
    integrated against the edge basis (Eqs. A6-A7, weak form)."""
    m = sem.Mesh(6, 4, 20.0)
    lamv, muv = 2.1e9, 1.3e9
    lam = np.full((m.nz, m.nx), lamv)
    mu = np.full((m.nz, m.nx), muv)
    x, z = m.coords()
    a, b, c, d = 1.0e-3, -0.4e-3, 0.7e-3, 2.0e-3
    u = np.stack([a * x + b * z, c * x + d * z], -1)
    Ku = m.stiffness(lam, mu, u)
    area = (m.nex * m.h) * (m.nez * m.h)
    energy = area * ((lamv + 2 * muv) * (a * a + d * d) + 2 * lamv * a * d + muv * (b + c) ** 2)
    assert abs(np.sum(u * Ku) - energy) < 1e-12 * energy
    interior = Ku[1:-1, 1:-1]
    assert np.max(np.abs(interior)) < 1e-9 * np.max(np.abs(Ku))
    sxx = (lamv + 2 * muv) * a + lamv * d
    szz = lamv * a + (lamv + 2 * muv) * d
    sxz = muv * (b + c)
    H = m.nez * m.h
    L = m.nex * m.h
    # left edge, outward normal -x: nodal forces sum to -(sxx, sxz) * H
    # (corners are shared with the top/bottom edges; compare edge interiors
    # plus half-weights through the full-edge sums of the 1D quadrature)
    left = Ku[:, 0].sum(axis=0)
    right = Ku[:, -1].sum(axis=0)
    top = Ku[0, :].sum(axis=0)
    bottom = Ku[-1, :].sum(axis=0)
    # each edge sum = its own traction integral + the corner shares of the
    # two neighbouring edges; the corner share of an edge is w_0 h/2 * traction
    wc = 0.1 * m.h / 2
    t_left = -np.array([sxx, sxz]); t_right = -t_left
    t_top = -np.array([sxz, szz]); t_bot = -t_top
    exp_left = t_left * H + wc * (t_top + t_bot)
    exp_right = t_right * H + wc * (t_top + t_bot)
    exp_top = t_top * L + wc * (t_left + t_right)
    exp_bot = t_bot * L + wc * (t_left + t_right)
    for got, exp in ((left, exp_left), (right, exp_right), (top, exp_top), (bottom, exp_bot)):
        assert np.allclose(got, exp, rtol=1e-11, atol=1e-9 * abs(sxx) * H)


def test_mass_and_measure_integrate_area():
    m = sem.Mesh(7, 3, 15.0)
    W = m.measure()
    area = m.nex * m.h * m.nez * m.h
    assert abs(W.sum() - area) < 1e-10 * area
    rho = np.full((m.nz, m.nx), 2200.0)
    assert abs(m.mass(rho).sum() - 2200.0 * area) < 1e-10 * 2200 * area


def test_stacey_edge_integrals():
    m = sem.Mesh(6, 5, 10.0)
    rho = np.full((m.nz, m.nx), 2000.0)
    vp = np.full((m.nz, m.nx), 3000.0)
    vs = np.full((m.nz, m.nx), 1700.0)
    C = m.stacey(rho, vp, vs, free_top=1, absorb=1)
    H = m.nez * m.h
    L = m.nex * m.h
    # x-damping: rho vp on left+right edges, rho vs on the bottom edge
    assert abs(C[..., 0].sum() - (2 * 2000 * 3000 * H + 2000 * 1700 * L)) < 1e-6
    assert abs(C[..., 1].sum() - (2 * 2000 * 1700 * H + 2000 * 3000 * L)) < 1e-6
    assert np.all(C[1:-1, 1:-1] == 0)
    assert np.all(C[0, 1:-1] == 0)          # traction-free top
    assert np.all(m.stacey(rho, vp, vs, absorb=0) == 0)


def test_explosive_source_moments():
    """f_a(g) = M0 d psi_g / d x_a (x_s): zero net force, first moments M0 I."""
    m = sem.Mesh(6, 4, 25.0)
    x, z = m.coords()
    for xs, zs in ((63.0, 41.0), (75.0, 10.0), (100.0, 50.0)):
        f = m.source_vector(xs, zs, 0, 2.5)
        assert abs(f[..., 0].sum()) < 1e-12 and abs(f[..., 1].sum()) < 1e-12
        assert abs((x * f[..., 0]).sum() - 2.5) < 1e-12
        assert abs((z * f[..., 1]).sum() - 2.5) < 1e-12
        assert abs((x * f[..., 1]).sum()) < 1e-12
        assert abs((z * f[..., 0]).sum()) < 1e-12


def test_point_force_and_interpolation_reproduce_polynomials():
    m = sem.Mesh(5, 5, 20.0)
    x, z = m.coords()
    field = 1 + 0.3 * x - 0.2 * z + 1e-3 * x * z + 2e-4 * x ** 2 - 1e-8 * z ** 4
    for xs, zs in ((13.0, 77.0), (40.0, 40.0), (99.0, 3.0)):
        idx, w = m.interp(xs, zs)
        val = np.sum(w * field.ravel()[idx])
        exact = 1 + 0.3 * xs - 0.2 * zs + 1e-3 * xs * zs + 2e-4 * xs ** 2 - 1e-8 * zs ** 4
        assert abs(val - exact) < 1e-10 * abs(exact)
        f = m.source_vector(xs, zs, 2, 1.0)
        assert abs(f[..., 1].sum() - 1.0) < 1e-13 and np.all(f[..., 0] == 0)


def test_locate_tie_break_smaller_element():
    m = sem.Mesh(4, 4, 25.0)
    idx, _ = m.interp(50.0, 30.0)          # x on the edge between elements 1 and 2
    f = m.source_vector(50.0, 30.0, 0, 1.0)
    nz_cols = np.unique(np.nonzero(np.abs(f).sum(-1))[1])
    assert nz_cols.min() >= 4 and nz_cols.max() <= 8   # element 1 spans nodes 4..8


def test_ricker_peak_and_zeros():
    f0, dt = 10.0, 1e-4
    t0 = 0.12
    stf = sem.ricker(3000, dt, f0, t0, 2.0)
    n0 = int(round(t0 / dt))
    assert abs(stf[n0] - 2.0) < 1e-12
    tz = t0 + 1.0 / (np.pi * f0 * np.sqrt(2.0))
    t = np.arange(3001) * dt
    i = np.searchsorted(t, tz)
    assert stf[i - 1] * stf[i] <= 0
