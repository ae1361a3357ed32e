/*
 * FP64 CPU oracle for the 2-D isotropic elastic spectral-element path of
 * preconditioned-BFGS elastic FWI (Liu, Beller, Lei, Peter & Tromp 2020).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  It shares no
 * source with the CUDA library and is written to be read against the paper:
 * plain loops, double precision, no blocking or fusion.
 *
 * What it computes (passages of the paper it follows):
 *   - elastic wave equation, stiffness C(lambda, mu) and strain operator D:
 *     Appendix A, Eqs. A6-A7 (written here in displacement weak form, the
 *     form a spectral-element solver discretises, Section 3.1);
 *   - misfit f = 1/2 |R u - d|^2: Eq. A1 (with the rectangle-rule dt);
 *   - adjoint state and gradient: Eqs. A8-A18, taken as the exact adjoint of
 *     the discrete time stepping;
 *   - preconditioner maps P1-P4: Eqs. 5-8 with the closed forms of
 *     Eqs. A21-A22.
 *
 * Discretisation (readings where the paper is silent):
 *   - structured mesh of nex x nez square elements of side h, NGLL = 5
 *     Gauss-Lobatto-Legendre points per direction; global node grid
 *     nx = 4 nex + 1 by nz = 4 nez + 1, row 0 at the surface, z = depth;
 *   - model (rho, vp, vs) given per global node; lambda = rho (vp^2 - 2 vs^2),
 *     mu = rho vs^2 (Eq. A7 with lambda + 2 mu = rho vp^2);
 *   - first-order Stacey absorbing edges (diagonal damping C), traction-free
 *     top when free_top = 1;
 *   - Newmark beta = 0, gamma = 1/2 with the damping term taken implicitly,
 *     (M + dt/2 C) a_{n+1} = F_{n+1} - K u_{n+1} - C (v_n + dt/2 a_n), which
 *     is the damped central-difference scheme; the medium starts at rest,
 *     u_0 = v_0 = a_0 = 0, and the records are s_n = P u_n, n = 1..nt.
 *
 * Array conventions: scalar node fields are [nz][nx]; vector node fields
 * are [nz][nx][2] (x component, then z component).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NG 5

/* ------------------------------------------------------------------ */
/* GLL points, weights and Lagrange polynomials                        */
/* ------------------------------------------------------------------ */

static void gll_points(double xi[NG], double w[NG])
{
    double a = sqrt(3.0 / 7.0);
    xi[0] = -1.0; xi[1] = -a; xi[2] = 0.0; xi[3] = a; xi[4] = 1.0;
    w[0] = 1.0 / 10.0; w[1] = 49.0 / 90.0; w[2] = 32.0 / 45.0;
    w[3] = 49.0 / 90.0; w[4] = 1.0 / 10.0;
}

/* l[k] = Lagrange polynomial k through the GLL points, at s; dl[k] its
 * derivative (product rule over the factors). */
void ref_lagrange(double s, double l[NG], double dl[NG])
{
    double xi[NG], w[NG];
    gll_points(xi, w);
    for (int k = 0; k < NG; ++k) {
        double val = 1.0;
        for (int m = 0; m < NG; ++m)
            if (m != k) val *= (s - xi[m]) / (xi[k] - xi[m]);
        l[k] = val;
        double der = 0.0;
        for (int p = 0; p < NG; ++p) {
            if (p == k) continue;
            double term = 1.0 / (xi[k] - xi[p]);
            for (int m = 0; m < NG; ++m)
                if (m != k && m != p) term *= (s - xi[m]) / (xi[k] - xi[m]);
            der += term;
        }
        dl[k] = der;
    }
}

/* xi, w and D[i*5+k] = l_k'(xi_i). */
void ref_gll(double *xi, double *w, double *D)
{
    gll_points(xi, w);
    for (int i = 0; i < NG; ++i) {
        double l[NG], dl[NG];
        ref_lagrange(xi[i], l, dl);
        for (int k = 0; k < NG; ++k) D[i * NG + k] = dl[k];
    }
}

/* ------------------------------------------------------------------ */
/* Mesh helpers                                                        */
/* ------------------------------------------------------------------ */

typedef struct {
    int nex, nez, nx, nz;
    double h;
    double xi[NG], w[NG], D[NG][NG];
} mesh_t;

static void mesh_init(mesh_t *m, int nex, int nez, double h)
{
    double Dflat[NG * NG];
    m->nex = nex; m->nez = nez; m->h = h;
    m->nx = 4 * nex + 1; m->nz = 4 * nez + 1;
    ref_gll(m->xi, m->w, Dflat);
    for (int i = 0; i < NG; ++i)
        for (int k = 0; k < NG; ++k) m->D[i][k] = Dflat[i * NG + k];
}

/* global node of local point (i along x, j along z) in element (ex, ez) */
static int node_of(const mesh_t *m, int ex, int ez, int i, int j)
{
    return (4 * ez + j) * m->nx + (4 * ex + i);
}

void ref_node_coords(int nex, int nez, double h, double *x, double *z)
{
    mesh_t m;
    mesh_init(&m, nex, nez, h);
    for (int ez = 0; ez < nez; ++ez)
        for (int ex = 0; ex < nex; ++ex)
            for (int j = 0; j < NG; ++j)
                for (int i = 0; i < NG; ++i) {
                    int g = node_of(&m, ex, ez, i, j);
                    x[g] = ex * h + (1.0 + m.xi[i]) * h / 2.0;
                    z[g] = ez * h + (1.0 + m.xi[j]) * h / 2.0;
                }
}

/* Diagonal (GLL-lumped) mass: M_g = sum over local points of rho w_i w_j (h/2)^2. */
void ref_mass(int nex, int nez, double h, const double *rho, double *M)
{
    mesh_t m;
    mesh_init(&m, nex, nez, h);
    memset(M, 0, sizeof(double) * (size_t)m.nx * m.nz);
    double jac = (h / 2.0) * (h / 2.0);
    for (int ez = 0; ez < nez; ++ez)
        for (int ex = 0; ex < nex; ++ex)
            for (int j = 0; j < NG; ++j)
                for (int i = 0; i < NG; ++i) {
                    int g = node_of(&m, ex, ez, i, j);
                    M[g] += rho[g] * m.w[i] * m.w[j] * jac;
                }
}

/* Quadrature measure per node, sum of w_i w_j (h/2)^2 over local points. */
void ref_node_measure(int nex, int nez, double h, double *W)
{
    mesh_t m;
    mesh_init(&m, nex, nez, h);
    int N = m.nx * m.nz;
    double *one = (double *)malloc(sizeof(double) * N);
    for (int g = 0; g < N; ++g) one[g] = 1.0;
    ref_mass(nex, nez, h, one, W);
    free(one);
}

/*
 * First-order Stacey damping, diagonal on this axis-aligned mesh.
 * Traction on an absorbing edge with outward normal n:
 *   t = -rho vp (v.n) n - rho vs (v - (v.n) n),
 * integrated with the edge GLL weights times h/2.  C[g*2+0] damps the x
 * component, C[g*2+1] the z component.  absorb = 0 gives a closed box with
 * no damping at all; free_top = 1 keeps the top edge traction-free.
 * ref_stacey_weights returns the edge weights split by role: Wn[g*2+c]
 * multiplies rho vp on component c, Wt[g*2+c] multiplies rho vs, so that
 * C = rho vp Wn + rho vs Wt (ref_stacey).
 */
void ref_stacey_weights(int nex, int nez, double h, int free_top, int absorb,
                        double *Wn, double *Wt)
{
    mesh_t m;
    mesh_init(&m, nex, nez, h);
    int N = m.nx * m.nz;
    memset(Wn, 0, sizeof(double) * 2 * N);
    memset(Wt, 0, sizeof(double) * 2 * N);
    if (!absorb) return;
    double jac = h / 2.0;
    /* left (x = 0) and right (x = L) edges: normal along x */
    for (int ez = 0; ez < nez; ++ez)
        for (int j = 0; j < NG; ++j) {
            int gl = node_of(&m, 0, ez, 0, j);
            int gr = node_of(&m, nex - 1, ez, NG - 1, j);
            double wq = m.w[j] * jac;
            Wn[gl * 2 + 0] += wq; Wt[gl * 2 + 1] += wq;
            Wn[gr * 2 + 0] += wq; Wt[gr * 2 + 1] += wq;
        }
    /* bottom edge (z = H), and the top edge unless it is free: normal along z */
    for (int ex = 0; ex < nex; ++ex)
        for (int i = 0; i < NG; ++i) {
            double wq = m.w[i] * jac;
            int gb = node_of(&m, ex, nez - 1, i, NG - 1);
            Wn[gb * 2 + 1] += wq; Wt[gb * 2 + 0] += wq;
            if (!free_top) {
                int gt = node_of(&m, ex, 0, i, 0);
                Wn[gt * 2 + 1] += wq; Wt[gt * 2 + 0] += wq;
            }
        }
}

void ref_stacey(int nex, int nez, double h, int free_top, int absorb,
                const double *rho, const double *vp, const double *vs, double *C)
{
    int N = (4 * nex + 1) * (4 * nez + 1);
    double *Wn = (double *)malloc(sizeof(double) * 2 * N);
    double *Wt = (double *)malloc(sizeof(double) * 2 * N);
    ref_stacey_weights(nex, nez, h, free_top, absorb, Wn, Wt);
    for (int g = 0; g < N; ++g)
        for (int c = 0; c < 2; ++c)
            C[g * 2 + c] = rho[g] * vp[g] * Wn[g * 2 + c] + rho[g] * vs[g] * Wt[g * 2 + c];
    free(Wn); free(Wt);
}

/* Strain of a displacement field at every local point of element (ex, ez):
 * exx = d ux/dx, ezz = d uz/dz, gam = d ux/dz + d uz/dx   (rows of D, Eq. A7). */
static void element_strain(const mesh_t *m, int ex, int ez, const double *u,
                           double exx[NG][NG], double ezz[NG][NG], double gam[NG][NG])
{
    double ux[NG][NG], uz[NG][NG];   /* [j][i] */
    for (int j = 0; j < NG; ++j)
        for (int i = 0; i < NG; ++i) {
            int g = node_of(m, ex, ez, i, j);
            ux[j][i] = u[g * 2 + 0];
            uz[j][i] = u[g * 2 + 1];
        }
    double s = 2.0 / m->h;   /* d xi / dx = d eta / dz */
    for (int j = 0; j < NG; ++j)
        for (int i = 0; i < NG; ++i) {
            double ux_xi = 0, ux_eta = 0, uz_xi = 0, uz_eta = 0;
            for (int k = 0; k < NG; ++k) {
                ux_xi += m->D[i][k] * ux[j][k];
                uz_xi += m->D[i][k] * uz[j][k];
                ux_eta += m->D[j][k] * ux[k][i];
                uz_eta += m->D[j][k] * uz[k][i];
            }
            exx[j][i] = s * ux_xi;
            ezz[j][i] = s * uz_eta;
            gam[j][i] = s * ux_eta + s * uz_xi;
        }
}

/*
 * Internal force K u (weak form of D^T C D u, Eq. A7):
 *   (K u)_a(node mn) = sum_{local points ij} W_ij sigma_ab(ij) d psi_mn/d x_b (ij),
 * with psi_mn(ij) = delta_im delta_jn, d psi_mn/dx (ij) = (2/h) D[i][m] delta_jn
 * and d psi_mn/dz (ij) = (2/h) delta_im D[j][n]; the Kronecker deltas are
 * evaluated, which leaves one sum over i and one over j.
 */
void ref_stiffness(int nex, int nez, double h, const double *lam, const double *mu,
                   const double *u, double *Ku)
{
    mesh_t m;
    mesh_init(&m, nex, nez, h);
    int N = m.nx * m.nz;
    memset(Ku, 0, sizeof(double) * 2 * N);
    double jac = (h / 2.0) * (h / 2.0);
    double s = 2.0 / h;
    for (int ez = 0; ez < nez; ++ez)
        for (int ex = 0; ex < nex; ++ex) {
            double exx[NG][NG], ezz[NG][NG], gam[NG][NG];
            double sxx[NG][NG], szz[NG][NG], sxz[NG][NG];
            element_strain(&m, ex, ez, u, exx, ezz, gam);
            for (int j = 0; j < NG; ++j)
                for (int i = 0; i < NG; ++i) {
                    int g = node_of(&m, ex, ez, i, j);
                    double L = lam[g], U = mu[g];
                    sxx[j][i] = (L + 2 * U) * exx[j][i] + L * ezz[j][i];
                    szz[j][i] = L * exx[j][i] + (L + 2 * U) * ezz[j][i];
                    sxz[j][i] = U * gam[j][i];
                }
            for (int n = 0; n < NG; ++n)
                for (int mm = 0; mm < NG; ++mm) {
                    double fx = 0, fz = 0;
                    for (int i = 0; i < NG; ++i) {   /* d/dx part: points (i, n) */
                        double Wq = m.w[i] * m.w[n] * jac;
                        fx += Wq * sxx[n][i] * s * m.D[i][mm];
                        fz += Wq * sxz[n][i] * s * m.D[i][mm];
                    }
                    for (int j = 0; j < NG; ++j) {   /* d/dz part: points (mm, j) */
                        double Wq = m.w[mm] * m.w[j] * jac;
                        fx += Wq * sxz[j][mm] * s * m.D[j][n];
                        fz += Wq * szz[j][mm] * s * m.D[j][n];
                    }
                    int g = node_of(&m, ex, ez, mm, n);
                    Ku[g * 2 + 0] += fx;
                    Ku[g * 2 + 1] += fz;
                }
        }
}

/* ------------------------------------------------------------------ */
/* Sources and receivers                                               */
/* ------------------------------------------------------------------ */

/* Element containing (x, z) and its local coordinates.  A point on a shared
 * element edge is given to the element with the smaller index (ex, then ez). */
int ref_locate(int nex, int nez, double h, double x, double z,
               int *ex, int *ez, double *xi, double *eta)
{
    if (x < 0 || z < 0 || x > nex * h || z > nez * h) return -1;
    int e = (int)ceil(x / h) - 1; if (e < 0) e = 0; if (e > nex - 1) e = nex - 1;
    int f = (int)ceil(z / h) - 1; if (f < 0) f = 0; if (f > nez - 1) f = nez - 1;
    *ex = e; *ez = f;
    *xi = 2.0 * (x - e * h) / h - 1.0;
    *eta = 2.0 * (z - f * h) / h - 1.0;
    return 0;
}

/* Receiver interpolation: s = sum_{ij} psi_ij(x_r) u(node ij). */
int ref_interp(int nex, int nez, double h, double x, double z, int *idx, double *wts)
{
    mesh_t m;
    int ex, ez; double xi, eta;
    mesh_init(&m, nex, nez, h);
    if (ref_locate(nex, nez, h, x, z, &ex, &ez, &xi, &eta)) return -1;
    double lx[NG], dlx[NG], lz[NG], dlz[NG];
    ref_lagrange(xi, lx, dlx);
    ref_lagrange(eta, lz, dlz);
    for (int j = 0; j < NG; ++j)
        for (int i = 0; i < NG; ++i) {
            idx[j * NG + i] = node_of(&m, ex, ez, i, j);
            wts[j * NG + i] = lx[i] * lz[j];
        }
    return 0;
}

/*
 * Nodal source vector f [nz][nx][2].
 *   type 0: explosive moment tensor M0 I; weak form f_a(ij) = M0 d psi_ij/d x_a (x_s)
 *   type 1: point force along x, f_x(ij) = amp psi_ij(x_s)
 *   type 2: point force along z.
 */
int ref_source_vector(int nex, int nez, double h, double x, double z, int type,
                      double amp, double *f)
{
    mesh_t m;
    int ex, ez; double xi, eta;
    mesh_init(&m, nex, nez, h);
    memset(f, 0, sizeof(double) * 2 * (size_t)m.nx * m.nz);
    if (ref_locate(nex, nez, h, x, z, &ex, &ez, &xi, &eta)) return -1;
    double lx[NG], dlx[NG], lz[NG], dlz[NG];
    ref_lagrange(xi, lx, dlx);
    ref_lagrange(eta, lz, dlz);
    double s = 2.0 / h;
    for (int j = 0; j < NG; ++j)
        for (int i = 0; i < NG; ++i) {
            int g = node_of(&m, ex, ez, i, j);
            if (type == 0) {
                f[g * 2 + 0] += amp * s * dlx[i] * lz[j];
                f[g * 2 + 1] += amp * lx[i] * s * dlz[j];
            } else if (type == 1) {
                f[g * 2 + 0] += amp * lx[i] * lz[j];
            } else if (type == 2) {
                f[g * 2 + 1] += amp * lx[i] * lz[j];
            } else {
                return -2;
            }
        }
    return 0;
}

/* Ricker wavelet r(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2),
 * sampled at t_n = n dt, n = 0..nt. */
void ref_ricker(int nt, double dt, double f0, double t0, double amp, double *stf)
{
    double pi = 3.14159265358979323846;
    for (int n = 0; n <= nt; ++n) {
        double t = n * dt - t0;
        double a = pi * pi * f0 * f0 * t * t;
        stf[n] = amp * (1.0 - 2.0 * a) * exp(-a);
    }
}

/* ------------------------------------------------------------------ */
/* Forward, adjoint, gradient                                          */
/* ------------------------------------------------------------------ */

static void lame(int N, const double *rho, const double *vp, const double *vs,
                 double *lam, double *mu)
{
    for (int g = 0; g < N; ++g) {
        lam[g] = rho[g] * (vp[g] * vp[g] - 2.0 * vs[g] * vs[g]);
        mu[g] = rho[g] * vs[g] * vs[g];
    }
}

/*
 * Newmark (beta = 0, gamma = 1/2) forward simulation from rest.
 *   u_{n+1} = u_n + dt v_n + dt^2/2 a_n
 *   (M + dt/2 C) a_{n+1} = f stf[n+1] - K u_{n+1} - C (v_n + dt/2 a_n)
 *   v_{n+1} = v_n + dt/2 (a_n + a_{n+1})
 * seis[r][c][n-1] = sum_k wts[r][k] u_n(idx[r][k])_c for n = 1..nt.
 * u_hist / a_hist (optional) receive u_n, a_n for n = 0..nt.
 * Returns 0, or -3 if the field stops being finite.
 */
int ref_forward(int nex, int nez, double h, int free_top, int absorb,
                const double *rho, const double *vp, const double *vs,
                const double *fvec, const double *stf,
                int nrec, const int *ridx, const double *rw,
                double dt, int nt, double *seis, double *u_hist, double *a_hist)
{
    int N = (4 * nex + 1) * (4 * nez + 1);
    size_t V = (size_t)2 * N;
    double *lam = malloc(sizeof(double) * N), *mu = malloc(sizeof(double) * N);
    double *M = malloc(sizeof(double) * N), *C = malloc(sizeof(double) * V);
    double *u = calloc(V, sizeof(double)), *v = calloc(V, sizeof(double));
    double *a = calloc(V, sizeof(double)), *un = malloc(sizeof(double) * V);
    double *an = malloc(sizeof(double) * V), *Ku = malloc(sizeof(double) * V);
    int status = 0;
    lame(N, rho, vp, vs, lam, mu);
    ref_mass(nex, nez, h, rho, M);
    ref_stacey(nex, nez, h, free_top, absorb, rho, vp, vs, C);
    if (u_hist) memset(u_hist, 0, sizeof(double) * V);
    if (a_hist) memset(a_hist, 0, sizeof(double) * V);
    for (int n = 0; n < nt; ++n) {
        for (size_t q = 0; q < V; ++q) un[q] = u[q] + dt * v[q] + 0.5 * dt * dt * a[q];
        ref_stiffness(nex, nez, h, lam, mu, un, Ku);
        for (int g = 0; g < N; ++g)
            for (int c = 0; c < 2; ++c) {
                size_t q = (size_t)g * 2 + c;
                double rhs = fvec[q] * stf[n + 1] - Ku[q] - C[q] * (v[q] + 0.5 * dt * a[q]);
                an[q] = rhs / (M[g] + 0.5 * dt * C[q]);
            }
        for (size_t q = 0; q < V; ++q) {
            v[q] = v[q] + 0.5 * dt * (a[q] + an[q]);
            a[q] = an[q];
            u[q] = un[q];
        }
        for (int r = 0; r < nrec; ++r)
            for (int c = 0; c < 2; ++c) {
                double sacc = 0;
                for (int k = 0; k < NG * NG; ++k)
                    sacc += rw[r * NG * NG + k] * u[(size_t)ridx[r * NG * NG + k] * 2 + c];
                seis[((size_t)r * 2 + c) * nt + n] = sacc;
            }
        if (u_hist) memcpy(u_hist + (size_t)(n + 1) * V, u, sizeof(double) * V);
        if (a_hist) memcpy(a_hist + (size_t)(n + 1) * V, a, sizeof(double) * V);
        if (!isfinite(u[0]) || !isfinite(u[V / 2])) { status = -3; break; }
    }
    free(lam); free(mu); free(M); free(C); free(u); free(v); free(a);
    free(un); free(an); free(Ku);
    return status;
}

/*
 * Discrete adjoint of the forward map above.  Eliminating v and a, the
 * forward scheme is
 *   A u_{n+1} = B u_n - A' u_{n-1} + dt^2 f stf[n],  n = 1..nt-1,  u_0 = u_1 = 0,
 * with A = M + dt/2 C, B = 2M - dt^2 K, A' = M - dt/2 C (all symmetric).  For
 * a functional with d/du_k = P^T g_k the Lagrange multipliers solve the same
 * recurrence backwards from rest:
 *   A lam_{k-1} = B lam_k - A' lam_{k+1} + P^T g_k,  k = nt..1,
 *   lam_nt = lam_{nt+1} = 0.
 * gsrc[r][c][k-1] = g_k at receiver r, component c.  lam_hist receives
 * lam_0..lam_{nt+1}, (nt+2) vector fields.
 */
int ref_adjoint(int nex, int nez, double h, int free_top, int absorb,
                const double *rho, const double *vp, const double *vs,
                int nrec, const int *ridx, const double *rw,
                const double *gsrc, double dt, int nt, double *lam_hist)
{
    int N = (4 * nex + 1) * (4 * nez + 1);
    size_t V = (size_t)2 * N;
    double *lam = malloc(sizeof(double) * N), *mu = malloc(sizeof(double) * N);
    double *M = malloc(sizeof(double) * N), *C = malloc(sizeof(double) * V);
    double *Kl = malloc(sizeof(double) * V), *rhs = malloc(sizeof(double) * V);
    int status = 0;
    lame(N, rho, vp, vs, lam, mu);
    ref_mass(nex, nez, h, rho, M);
    ref_stacey(nex, nez, h, free_top, absorb, rho, vp, vs, C);
    memset(lam_hist + (size_t)nt * V, 0, sizeof(double) * 2 * V);
    for (int k = nt; k >= 1; --k) {
        const double *lk = lam_hist + (size_t)k * V;
        const double *lk1 = lam_hist + (size_t)(k + 1) * V;
        double *lkm = lam_hist + (size_t)(k - 1) * V;
        ref_stiffness(nex, nez, h, lam, mu, lk, Kl);
        for (int g = 0; g < N; ++g)
            for (int c = 0; c < 2; ++c) {
                size_t q = (size_t)g * 2 + c;
                rhs[q] = 2.0 * M[g] * lk[q] - dt * dt * Kl[q] - (M[g] - 0.5 * dt * C[q]) * lk1[q];
            }
        for (int r = 0; r < nrec; ++r)
            for (int c = 0; c < 2; ++c) {
                double gk = gsrc[((size_t)r * 2 + c) * nt + (k - 1)];
                for (int q = 0; q < NG * NG; ++q)
                    rhs[(size_t)ridx[r * NG * NG + q] * 2 + c] += rw[r * NG * NG + q] * gk;
            }
        for (int g = 0; g < N; ++g)
            for (int c = 0; c < 2; ++c) {
                size_t q = (size_t)g * 2 + c;
                lkm[q] = rhs[q] / (M[g] + 0.5 * dt * C[q]);
            }
        if (!isfinite(lkm[0]) || !isfinite(lkm[V / 2])) { status = -3; break; }
    }
    free(lam); free(mu); free(M); free(C); free(Kl); free(rhs);
    return status;
}

/*
 * Gradient of the discrete misfit with respect to the nodal model
 * (rho, vp, vs), from the Lagrangian of the scheme above (the discrete form
 * of Eqs. A16-A18):
 *   g_m = - sum_{n=1}^{nt-1} lam_n^T [ dM/dm (u_{n+1} - 2 u_n + u_{n-1})
 *                                     + dt/2 dC/dm (u_{n+1} - u_{n-1})
 *                                     + dt^2 dK/dm u_n ].
 * lam_n^T dK/dm_g u_n = sum over local points l at node g of
 *   W_l [ dlambda/dm (div lam)(div u) + dmu/dm (2 exx exx' + 2 ezz ezz' + gam gam') ],
 * the derivative of the strain energy with the stiffness C of Eq. A7.
 * u_hist holds u_0..u_nt, lam_hist lam_0..lam_{nt+1}.  grad is [3][nz][nx]
 * in the order rho, vp, vs.
 */
int ref_gradient(int nex, int nez, double h, int free_top, int absorb,
                 const double *rho, const double *vp, const double *vs,
                 const double *u_hist, const double *lam_hist, double dt, int nt,
                 double *grad)
{
    mesh_t m;
    mesh_init(&m, nex, nez, h);
    int N = m.nx * m.nz;
    size_t V = (size_t)2 * N;
    double *W = malloc(sizeof(double) * N);
    double *Wn = malloc(sizeof(double) * V), *Wt = malloc(sizeof(double) * V);
    double *gr = grad, *gp = grad + N, *gs = grad + 2 * N;
    ref_node_measure(nex, nez, h, W);
    ref_stacey_weights(nex, nez, h, free_top, absorb, Wn, Wt);
    memset(grad, 0, sizeof(double) * 3 * N);
    double jac = (h / 2.0) * (h / 2.0);
    for (int n = 1; n <= nt - 1; ++n) {
        const double *ln = lam_hist + (size_t)n * V;
        const double *up = u_hist + (size_t)(n + 1) * V;
        const double *u0 = u_hist + (size_t)n * V;
        const double *um = u_hist + (size_t)(n - 1) * V;
        /* mass and damping terms, node by node */
        for (int g = 0; g < N; ++g)
            for (int c = 0; c < 2; ++c) {
                size_t q = (size_t)g * 2 + c;
                double acc2 = up[q] - 2.0 * u0[q] + um[q];
                double dif = up[q] - um[q];
                /* M_g = rho_g W_g */
                gr[g] -= ln[q] * W[g] * acc2;
                /* C_q = rho vp Wn_q + rho vs Wt_q */
                gr[g] -= ln[q] * 0.5 * dt * (vp[g] * Wn[q] + vs[g] * Wt[q]) * dif;
                gp[g] -= ln[q] * 0.5 * dt * (rho[g] * Wn[q]) * dif;
                gs[g] -= ln[q] * 0.5 * dt * (rho[g] * Wt[q]) * dif;
            }
        /* stiffness term, local point by local point */
        for (int ez = 0; ez < nez; ++ez)
            for (int ex = 0; ex < nex; ++ex) {
                double axx[NG][NG], azz[NG][NG], ag[NG][NG];
                double bxx[NG][NG], bzz[NG][NG], bg[NG][NG];
                element_strain(&m, ex, ez, ln, axx, azz, ag);
                element_strain(&m, ex, ez, u0, bxx, bzz, bg);
                for (int j = 0; j < NG; ++j)
                    for (int i = 0; i < NG; ++i) {
                        int g = node_of(&m, ex, ez, i, j);
                        double Wl = m.w[i] * m.w[j] * jac;
                        double dd = (axx[j][i] + azz[j][i]) * (bxx[j][i] + bzz[j][i]);
                        double ee = 2.0 * axx[j][i] * bxx[j][i] + 2.0 * azz[j][i] * bzz[j][i]
                                    + ag[j][i] * bg[j][i];
                        double r = rho[g], p = vp[g], s = vs[g];
                        /* lambda = r (p^2 - 2 s^2), mu = r s^2 */
                        double dlam_dr = p * p - 2.0 * s * s, dmu_dr = s * s;
                        double dlam_dp = 2.0 * r * p;
                        double dlam_ds = -4.0 * r * s, dmu_ds = 2.0 * r * s;
                        double f = dt * dt * Wl;
                        gr[g] -= f * (dlam_dr * dd + dmu_dr * ee);
                        gp[g] -= f * (dlam_dp * dd);
                        gs[g] -= f * (dlam_ds * dd + dmu_ds * ee);
                    }
            }
    }
    free(W); free(Wn); free(Wt);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Diagonal preconditioner maps, Eqs. 5-8 and A21-A22                  */
/* ------------------------------------------------------------------ */

/*
 * Time-integrated products of a source-side field A and a second field B
 * (B = A for P1 and P3; B = receiver wavefield for P2 and P4).
 *   particle velocity v_{n+1/2} = (u_{n+1} - u_n) / dt, n = 0..nt-1
 *   its time derivative a_n (acceleration), n = 1..nt
 * Per global node g, with W_l the quadrature weight of local point l, the
 * four signed time integrals entering Eqs. 5-8 / A21-A22:
 *   S[0] = sum_n dt aA_n . aB_n                                    (Eq. 5/6, A21c)
 *   S[1] = sum_n dt sum_l W_l div vA div vB                        (Eq. A21a/A22a)
 *   S[2] = sum_n dt sum_l W_l (dx vAx dx vBx + dz vAz dz vBz)      (Eq. A21b/A22b, 1st term)
 *   S[3] = sum_n dt sum_l W_l gam(vA) gam(vB)                      (Eq. A21b/A22b, 2nd term)
 * uA, uB: displacement histories n = 0..nt; aA, aB: acceleration
 * histories, index n = 0..nt (entry 0 unused).  S is [4][nz][nx].
 */
int ref_precond_sums(int nex, int nez, double h, const double *uA, const double *aA,
                     const double *uB, const double *aB, double dt, int nt, double *S)
{
    mesh_t m;
    mesh_init(&m, nex, nez, h);
    int N = m.nx * m.nz;
    size_t V = (size_t)2 * N;
    double *sr = S, *sa = S + N, *sb1 = S + 2 * N, *sb2 = S + 3 * N;
    double *vA = malloc(sizeof(double) * V), *vB = malloc(sizeof(double) * V);
    memset(S, 0, sizeof(double) * 4 * N);
    double jac = (h / 2.0) * (h / 2.0);
    for (int n = 1; n <= nt; ++n)
        for (int g = 0; g < N; ++g)
            sr[g] += dt * (aA[(size_t)n * V + g * 2] * aB[(size_t)n * V + g * 2]
                           + aA[(size_t)n * V + g * 2 + 1] * aB[(size_t)n * V + g * 2 + 1]);
    for (int n = 0; n <= nt - 1; ++n) {
        for (size_t q = 0; q < V; ++q) {
            vA[q] = (uA[(size_t)(n + 1) * V + q] - uA[(size_t)n * V + q]) / dt;
            vB[q] = (uB[(size_t)(n + 1) * V + q] - uB[(size_t)n * V + q]) / dt;
        }
        for (int ez = 0; ez < nez; ++ez)
            for (int ex = 0; ex < nex; ++ex) {
                double axx[NG][NG], azz[NG][NG], ag[NG][NG];
                double bxx[NG][NG], bzz[NG][NG], bg[NG][NG];
                element_strain(&m, ex, ez, vA, axx, azz, ag);
                element_strain(&m, ex, ez, vB, bxx, bzz, bg);
                for (int j = 0; j < NG; ++j)
                    for (int i = 0; i < NG; ++i) {
                        int g = node_of(&m, ex, ez, i, j);
                        double Wl = m.w[i] * m.w[j] * jac;
                        sa[g] += dt * Wl * (axx[j][i] + azz[j][i]) * (bxx[j][i] + bzz[j][i]);
                        sb1[g] += dt * Wl * (axx[j][i] * bxx[j][i] + azz[j][i] * bzz[j][i]);
                        sb2[g] += dt * Wl * ag[j][i] * bg[j][i];
                    }
            }
    }
    free(vA); free(vB);
    return 0;
}

/*
 * Gaussian smoothing of a node field in physical space: the quadrature-
 * weighted average
 *   S(H)(x) = sum_y H(y) G(x - y) W(y) / sum_y G(x - y) W(y),
 *   G(d) = exp(-|d|^2 / (2 sigma^2)),
 * summed over every node y (no truncation).
 */
void ref_smooth(int nex, int nez, double h, const double *in, double sigma, double *out)
{
    int nx = 4 * nex + 1, nz = 4 * nez + 1, N = nx * nz;
    double *x = malloc(sizeof(double) * N), *z = malloc(sizeof(double) * N);
    double *W = malloc(sizeof(double) * N);
    ref_node_coords(nex, nez, h, x, z);
    ref_node_measure(nex, nez, h, W);
    for (int g = 0; g < N; ++g) {
        double num = 0, den = 0;
        for (int q = 0; q < N; ++q) {
            double dx = x[g] - x[q], dz = z[g] - z[q];
            double G = exp(-(dx * dx + dz * dz) / (2.0 * sigma * sigma));
            num += in[q] * G * W[q];
            den += G * W[q];
        }
        out[g] = num / den;
    }
    free(x); free(z); free(W);
}
