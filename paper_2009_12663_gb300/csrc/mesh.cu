// Mesh, model and ABI plumbing of the gbfwi library.
//
// Structured mesh of nex x nez square elements with NGLL = 5
// Gauss-Lobatto-Legendre points per direction (the spectral-element
// discretisation the paper runs with SPECFEM2D, Section 3.1); global node
// grid nx = 4 nex + 1 by nz = 4 nez + 1, row 0 at the surface.

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>

#include "gbfwi_internal.h"

int gb_upload_gll(const double *D, const double *w);

// ---------------------------------------------------------------------------
// errors, buffers
// ---------------------------------------------------------------------------

static thread_local char g_err[512];
static thread_local char g_nonfinite[256];
static std::atomic<long long> g_launches{0};

void gb_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void gb_note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long gb_launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

extern "C" long long gbfwi_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

gbfwi_mesh::~gbfwi_mesh()
{
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (Lane *l : lanes) delete l;
}

extern "C" int gbfwi_enable_timing(gbfwi_mesh *m, int on)
{
    if (!m || (on != 0 && on != 1)) return GBFWI_EINVAL;
    m->timing = on != 0;
    return GBFWI_OK;
}

extern "C" int gbfwi_last_phase_times(const gbfwi_mesh *m, double *fwd_ms, double *adj_ms,
                                      long long *fwd_launches, long long *adj_launches)
{
    if (!m || !m->timed_valid) return GBFWI_EINVAL;
    if (fwd_ms) *fwd_ms = m->fwd_ms;
    if (adj_ms) *adj_ms = m->adj_ms;
    if (fwd_launches) *fwd_launches = m->fwd_launches;
    if (adj_launches) *adj_launches = m->adj_launches;
    return GBFWI_OK;
}

void gb_set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    snprintf(g_err, sizeof(g_err), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}

int gb_nonfinite(const char *what)
{
    snprintf(g_nonfinite, sizeof(g_nonfinite), "non-finite value: %s", what);
    return GBFWI_ENONFINITE;
}

int DevBuf::ensure(size_t nbytes)
{
    if (nbytes <= bytes && p) return GBFWI_OK;
    release();
    if (nbytes == 0) nbytes = 16;
    if (cudaMalloc(&p, nbytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        bytes = 0;
        return GBFWI_ENOMEM;
    }
    bytes = nbytes;
    return GBFWI_OK;
}

void DevBuf::release()
{
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

static_assert(cudaMemoryTypeUnregistered == GB_MEMTYPE_UNREGISTERED && cudaMemoryTypeHost == GB_MEMTYPE_HOST &&
                  cudaMemoryTypeDevice == GB_MEMTYPE_DEVICE && cudaMemoryTypeManaged == GB_MEMTYPE_MANAGED,
              "memory type values of ptrclass.h");

int gb_ptr_class(const void *ptr)
{
    if (!ptr) return GB_PTR_HOST;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return GB_PTR_HOST;
    }
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        cur = -1;
    }
    return gb_classify_pointer((int)at.type, at.device, cur);
}

bool gb_is_device_ptr(const void *ptr) { return gb_ptr_class(ptr) == GB_PTR_LOCAL; }

extern "C" const char *gbfwi_strerror(int code)
{
    switch (code) {
    case GBFWI_OK: return "ok";
    case GBFWI_EINVAL: return "invalid argument";
    case GBFWI_ENOMEM: return "out of memory";
    case GBFWI_ECUDA: return g_err[0] ? g_err : "CUDA error";
    case GBFWI_ECFL: return "time step violates the stability bound dt*vp_max/dx_min <= 0.5";
    case GBFWI_ECURV: return "BFGS pair rejected (curvature y^T s <= 0)";
    case GBFWI_ENONFINITE: return g_nonfinite[0] ? g_nonfinite : "non-finite value";
    case GBFWI_ENOMODEL: return "no model set";
    case GBFWI_ETIMEOUT: return "a time-step kernel's bounded wait for its staged inputs gave up";
    case GBFWI_ESCRATCH: return "request exceeds the fixed scratch of a no-allocation entry point (at most 256 shots)";
    }
    return "unknown error";
}

// ---------------------------------------------------------------------------
// GLL points and Lagrange polynomials (monomial expansion + Horner)
// ---------------------------------------------------------------------------

static void gll5(double xi[5], double w[5])
{
    const double a = std::sqrt(3.0 / 7.0);
    const double x[5] = {-1.0, -a, 0.0, a, 1.0};
    const double q[5] = {0.1, 49.0 / 90.0, 32.0 / 45.0, 49.0 / 90.0, 0.1};
    for (int i = 0; i < 5; ++i) { xi[i] = x[i]; w[i] = q[i]; }
}

// monomial coefficients c[k][0..4] of the Lagrange polynomial l_k
static void lagrange_coeffs(const double xi[5], double c[5][5])
{
    for (int k = 0; k < 5; ++k) {
        double poly[5] = {1, 0, 0, 0, 0};   // running product, ascending powers
        int deg = 0;
        double den = 1.0;
        for (int m = 0; m < 5; ++m) {
            if (m == k) continue;
            // poly *= (s - xi_m)
            for (int p = deg + 1; p >= 1; --p) poly[p] = poly[p - 1] - xi[m] * poly[p];
            poly[0] = -xi[m] * poly[0];
            ++deg;
            den *= (xi[k] - xi[m]);
        }
        for (int p = 0; p < 5; ++p) c[k][p] = poly[p] / den;
    }
}

static void lagrange_eval(const double c[5][5], double s, double l[5], double dl[5])
{
    for (int k = 0; k < 5; ++k) {
        double v = 0, d = 0;
        for (int p = 4; p >= 0; --p) v = v * s + c[k][p];
        for (int p = 4; p >= 1; --p) d = d * s + p * c[k][p];
        l[k] = v;
        dl[k] = d;
    }
}

// ---------------------------------------------------------------------------
// point location: a point on a shared edge goes to the smaller element index
// ---------------------------------------------------------------------------

static int locate(const gbfwi_mesh *m, double x, double z, int &ex, int &ez, double &xi, double &eta)
{
    const double L = m->d.nex * m->d.h, H = m->d.nez * m->d.h;
    if (!(x >= 0 && x <= L && z >= 0 && z <= H)) return GBFWI_EINVAL;
    ex = (int)std::ceil(x / m->d.h) - 1;
    ez = (int)std::ceil(z / m->d.h) - 1;
    ex = std::min(std::max(ex, 0), m->d.nex - 1);
    ez = std::min(std::max(ez, 0), m->d.nez - 1);
    xi = 2.0 * (x - ex * m->d.h) / m->d.h - 1.0;
    eta = 2.0 * (z - ez * m->d.h) / m->d.h - 1.0;
    return GBFWI_OK;
}

// ---------------------------------------------------------------------------
// mesh create / destroy
// ---------------------------------------------------------------------------

static std::mutex g_gll_mutex;
static bool g_gll_done[64];

extern "C" int gbfwi_mesh_create(const gbfwi_mesh_desc *desc, const gbfwi_source *src, int nsrc,
                                 const double *rec_xz, int nrec, gbfwi_mesh **out)
{
    if (!desc || !out || nsrc < 0 || nrec < 0 || (nsrc > 0 && !src) || (nrec > 0 && !rec_xz))
        return GBFWI_EINVAL;
    const gbfwi_mesh_desc &d = *desc;
    if (d.nex < 1 || d.nez < 1 || !(d.h > 0) || d.ngll != 5 || !(d.dt > 0) || d.nt < 2 ||
        d.precision != 0 || (d.free_surface_top != 0 && d.free_surface_top != 1))
        return GBFWI_EINVAL;
    if ((long long)(4 * d.nex + 2) * (4 * d.nez + 1) > (1LL << 30)) return GBFWI_EINVAL;

    gbfwi_mesh *m = new (std::nothrow) gbfwi_mesh();
    if (!m) return GBFWI_ENOMEM;
    m->d = d;
    m->nx = 4 * d.nex + 1;
    m->nz = 4 * d.nez + 1;
    // row pitch: a multiple of 4 nodes, so every row of every node field
    // (float, float2, float4) starts on a 16-byte boundary, as the 16-byte
    // asynchronous copies of the step kernel require
    m->pitch = (m->nx + 3) & ~3;
    double c[5][5];
    gll5(m->xi, m->w);
    lagrange_coeffs(m->xi, c);
    for (int i = 0; i < 5; ++i) {
        double l[5], dl[5];
        lagrange_eval(c, m->xi[i], l, dl);
        for (int k = 0; k < 5; ++k) m->D[i][k] = dl[k];
    }
    m->dx_min = d.h * (m->xi[1] - m->xi[0]) / 2.0;

    // assembled 1-D weights
    m->wx1.assign(m->nx, 0.0);
    m->wz1.assign(m->nz, 0.0);
    for (int e = 0; e < d.nex; ++e)
        for (int i = 0; i < 5; ++i) m->wx1[4 * e + i] += m->w[i] * d.h / 2.0;
    for (int e = 0; e < d.nez; ++e)
        for (int j = 0; j < 5; ++j) m->wz1[4 * e + j] += m->w[j] * d.h / 2.0;

    // receivers
    m->nrec = nrec;
    m->rec_xz.assign(rec_xz, rec_xz + 2 * (size_t)nrec);
    m->rec_ex.resize(nrec);
    m->rec_ez.resize(nrec);
    m->rec_w.resize((size_t)nrec * 25);
    for (int r = 0; r < nrec; ++r) {
        int ex, ez;
        double xi, eta, lx[5], dlx[5], lz[5], dlz[5];
        if (locate(m, rec_xz[2 * r], rec_xz[2 * r + 1], ex, ez, xi, eta)) { delete m; return GBFWI_EINVAL; }
        lagrange_eval(c, xi, lx, dlx);
        lagrange_eval(c, eta, lz, dlz);
        m->rec_ex[r] = ex;
        m->rec_ez[r] = ez;
        for (int j = 0; j < 5; ++j)
            for (int i = 0; i < 5; ++i) m->rec_w[(size_t)r * 25 + j * 5 + i] = (float)(lx[i] * lz[j]);
    }
    // sources
    m->src.assign(src, src + nsrc);
    m->src_nodes.resize(nsrc);
    std::vector<float> stf((size_t)nsrc * (d.nt + 1));
    const double pi = 3.14159265358979323846;
    for (int s = 0; s < nsrc; ++s) {
        const gbfwi_source &S = src[s];
        int ex, ez;
        double xi, eta, lx[5], dlx[5], lz[5], dlz[5];
        if (S.type < 0 || S.type > 2 || !(S.f0 > 0) || locate(m, S.x, S.z, ex, ez, xi, eta)) {
            delete m;
            return GBFWI_EINVAL;
        }
        lagrange_eval(c, xi, lx, dlx);
        lagrange_eval(c, eta, lz, dlz);
        const double sc = 2.0 / d.h;
        for (int j = 0; j < 5; ++j)
            for (int i = 0; i < 5; ++i) {
                double fx = 0, fz = 0;
                if (S.type == 0) { fx = sc * dlx[i] * lz[j]; fz = lx[i] * sc * dlz[j]; }
                else if (S.type == 1) fx = lx[i] * lz[j];
                else fz = lx[i] * lz[j];
                if (fx == 0.0 && fz == 0.0) continue;
                m->src_nodes[s].push_back({4 * ex + i, 4 * ez + j, (float)fx, (float)fz});
            }
        for (int n = 0; n <= d.nt; ++n) {
            double t = n * d.dt - S.t0;
            double q = pi * pi * S.f0 * S.f0 * t * t;
            stf[(size_t)s * (d.nt + 1) + n] = (float)(S.amp * (1.0 - 2.0 * q) * std::exp(-q));
        }
    }

    // device tables
    int rc = GBFWI_OK;
    {
        std::lock_guard<std::mutex> lk(g_gll_mutex);
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 64 || !g_gll_done[dev]) {
            double Df[25];
            for (int i = 0; i < 5; ++i)
                for (int k = 0; k < 5; ++k) Df[i * 5 + k] = m->D[i][k];
            rc = gb_upload_gll(Df, m->w);
            if (rc == GBFWI_OK && dev >= 0 && dev < 64) g_gll_done[dev] = true;
        }
    }
    const size_t NP = (size_t)m->nz * m->pitch;
    if (!rc) rc = m->d_lm.ensure(NP * sizeof(float2));
    if (!rc) rc = m->d_minv.ensure(NP * sizeof(float));
    if (!rc) rc = m->d_bnd.ensure(NP * sizeof(float4));
    if (!rc) rc = m->d_bw.ensure(NP * sizeof(float4));
    if (!rc) rc = m->d_model.ensure(3 * NP * sizeof(float));
    if (!rc) rc = m->d_wx.ensure(m->nx * sizeof(float));
    if (!rc) rc = m->d_wz.ensure(m->nz * sizeof(float));
    if (!rc) rc = m->d_recw.ensure(std::max<size_t>(1, m->rec_w.size()) * sizeof(float));
    if (!rc) rc = m->w_status.ensure(16);
    if (!rc && cudaMemset(m->w_status.p, 0, 16) != cudaSuccess) rc = GBFWI_ECUDA;
    if (!rc) rc = m->d_rec_e.ensure(std::max(1, nrec) * sizeof(int2));
    if (!rc) rc = m->d_stf.ensure(std::max<size_t>(1, stf.size()) * sizeof(float));
    if (rc) { delete m; return rc; }

    // Stacey edge weights (first-order Stacey: t = -rho vp (v.n) n - rho vs (v - (v.n) n))
    std::vector<float4> bw(NP, make_float4(0, 0, 0, 0));
    for (int iz = 0; iz < m->nz; ++iz) {
        for (int side = 0; side < 2; ++side) {
            int ix = side == 0 ? 0 : m->nx - 1;
            float4 &q = bw[(size_t)iz * m->pitch + ix];
            q.x += (float)m->wz1[iz];   // normal (x) component <- rho vp
            q.w += (float)m->wz1[iz];   // tangential (z) component <- rho vs
        }
    }
    for (int ix = 0; ix < m->nx; ++ix) {
        for (int side = 0; side < 2; ++side) {
            if (side == 0 && d.free_surface_top) continue;
            int iz = side == 0 ? 0 : m->nz - 1;
            float4 &q = bw[(size_t)iz * m->pitch + ix];
            q.y += (float)m->wx1[ix];   // normal (z) component <- rho vp
            q.z += (float)m->wx1[ix];   // tangential (x) component <- rho vs
        }
    }
    std::vector<float> wxf(m->wx1.begin(), m->wx1.end()), wzf(m->wz1.begin(), m->wz1.end());
    std::vector<int2> re(std::max(1, nrec));
    for (int r = 0; r < nrec; ++r) re[r] = make_int2(m->rec_ex[r], m->rec_ez[r]);
    auto up = [&](DevBuf &b, const void *h, size_t n) -> int {
        if (n == 0) return GBFWI_OK;
        GB_CUDA(cudaMemcpy(b.p, h, n, cudaMemcpyHostToDevice));
        return GBFWI_OK;
    };
    rc = up(m->d_bw, bw.data(), NP * sizeof(float4));
    if (!rc) rc = up(m->d_wx, wxf.data(), wxf.size() * sizeof(float));
    if (!rc) rc = up(m->d_wz, wzf.data(), wzf.size() * sizeof(float));
    if (!rc) rc = up(m->d_recw, m->rec_w.data(), m->rec_w.size() * sizeof(float));
    if (!rc) rc = up(m->d_rec_e, re.data(), nrec * sizeof(int2));
    if (!rc) rc = up(m->d_stf, stf.data(), stf.size() * sizeof(float));
    if (rc) { delete m; return rc; }
    *out = m;
    return GBFWI_OK;
}

extern "C" int gbfwi_mesh_destroy(gbfwi_mesh *m)
{
    delete m;
    return GBFWI_OK;
}

extern "C" int gbfwi_mesh_dims(const gbfwi_mesh *m, int *nx, int *nz)
{
    if (!m || !nx || !nz) return GBFWI_EINVAL;
    *nx = m->nx;
    *nz = m->nz;
    return GBFWI_OK;
}

extern "C" int gbfwi_node_coords(const gbfwi_mesh *m, double *x, double *z)
{
    if (!m || !x || !z) return GBFWI_EINVAL;
    for (int iz = 0; iz < m->nz; ++iz)
        for (int ix = 0; ix < m->nx; ++ix) {
            int ex = std::min(ix / 4, m->d.nex - 1), i = ix - 4 * ex;
            int ez = std::min(iz / 4, m->d.nez - 1), j = iz - 4 * ez;
            x[(size_t)iz * m->nx + ix] = ex * m->d.h + (1.0 + m->xi[i]) * m->d.h / 2.0;
            z[(size_t)iz * m->nx + ix] = ez * m->d.h + (1.0 + m->xi[j]) * m->d.h / 2.0;
        }
    return GBFWI_OK;
}

extern "C" int gbfwi_num_tiles(void) { return kNumTiles; }

extern "C" int gbfwi_tile_shape(int tile, int *tx, int *tz)
{
    if (tile < 0 || tile >= kNumTiles || !tx || !tz) return GBFWI_EINVAL;
    *tx = kTiles[tile].tx;
    *tz = kTiles[tile].tz;
    return GBFWI_OK;
}

extern "C" int gbfwi_get_schedule(const gbfwi_mesh *m, gbfwi_schedule *s)
{
    if (!m || !s) return GBFWI_EINVAL;
    *s = m->sch;
    return GBFWI_OK;
}

extern "C" int gbfwi_set_schedule(gbfwi_mesh *m, const gbfwi_schedule *s)
{
    if (!m || !s) return GBFWI_EINVAL;
    if (s->shots_per_launch < 1 || s->tile < 0 || s->tile >= kNumTiles || s->ckpt_every < 0 ||
        (s->use_graph != 0 && s->use_graph != 1) || s->streams < 1 || s->streams > 8)
        return GBFWI_EINVAL;
    m->sch = *s;
    return GBFWI_OK;
}

// ---------------------------------------------------------------------------
// per-tile injection and recording lists
// ---------------------------------------------------------------------------

namespace {
struct RawEntry { int tile, node, key; InjEntry e; };

void build_groups(std::vector<RawEntry> &raw, int ntiles, std::vector<int> &gptr,
                  std::vector<InjGroup> &groups, std::vector<InjEntry> &entries)
{
    std::stable_sort(raw.begin(), raw.end(), [](const RawEntry &a, const RawEntry &b) {
        if (a.tile != b.tile) return a.tile < b.tile;
        if (a.node != b.node) return a.node < b.node;
        return a.key < b.key;
    });
    size_t g0 = groups.size();
    std::vector<int> counts(ntiles + 1, 0);
    for (size_t q = 0; q < raw.size();) {
        size_t r = q;
        while (r < raw.size() && raw[r].tile == raw[q].tile && raw[r].node == raw[q].node) ++r;
        InjGroup G;
        G.node = raw[q].node;
        G.begin = (int)entries.size();
        for (size_t t = q; t < r; ++t) entries.push_back(raw[t].e);
        G.end = (int)entries.size();
        G.pad = 0;
        groups.push_back(G);
        counts[raw[q].tile + 1]++;
        q = r;
    }
    for (int t = 0; t < ntiles; ++t) counts[t + 1] += counts[t];
    for (int t = 0; t <= ntiles; ++t) gptr.push_back((int)g0 + counts[t]);
}
}  // namespace

int gb_build_tile_lists(gbfwi_mesh *m, int tile)
{
    TileLists &L = m->lists[tile];
    if (L.built) return GBFWI_OK;
    const int TX = kTiles[tile].tx, TZ = kTiles[tile].tz;
    L.ntx = (m->d.nex + TX - 1) / TX;
    L.ntz = (m->d.nez + TZ - 1) / TZ;
    const int ntiles = L.ntx * L.ntz;
    auto owner = [&](int ix, int iz, int &t, int &node) {
        int tx = std::min(ix / (4 * TX), L.ntx - 1), tz = std::min(iz / (4 * TZ), L.ntz - 1);
        int ox = ix - 4 * TX * tx, oz = iz - 4 * TZ * tz;
        t = tz * L.ntx + tx;
        node = oz * (4 * TX + 1) + ox;
    };
    // sources
    std::vector<int> sgptr;
    std::vector<InjGroup> sgroups;
    std::vector<InjEntry> sentries;
    for (size_t s = 0; s < m->src.size(); ++s) {
        std::vector<RawEntry> raw;
        for (auto &sn : m->src_nodes[s]) {
            RawEntry r;
            owner(sn.ix, sn.iz, r.tile, r.node);
            r.key = 0;
            r.e = InjEntry{0, 0, sn.wx, sn.wz};
            raw.push_back(r);
        }
        build_groups(raw, ntiles, sgptr, sgroups, sentries);
    }
    // adjoint sources at the receivers (P^T): channel 2r (x), 2r+1 (z)
    std::vector<int> rgptr;
    std::vector<InjGroup> rgroups;
    std::vector<InjEntry> rentries;
    {
        std::vector<RawEntry> raw;
        for (int r = 0; r < m->nrec; ++r)
            for (int j = 0; j < 5; ++j)
                for (int i = 0; i < 5; ++i) {
                    float w = m->rec_w[(size_t)r * 25 + j * 5 + i];
                    if (w == 0.0f) continue;
                    RawEntry e;
                    owner(4 * m->rec_ex[r] + i, 4 * m->rec_ez[r] + j, e.tile, e.node);
                    e.key = r;
                    e.e = InjEntry{2 * r, 2 * r + 1, w, w};
                    raw.push_back(e);
                }
        build_groups(raw, ntiles, rgptr, rgroups, rentries);
    }
    // recording: receivers by the tile of their element
    std::vector<int> tcount(ntiles + 1, 0), rlist(m->nrec);
    std::vector<int> rtile(m->nrec);
    for (int r = 0; r < m->nrec; ++r) {
        rtile[r] = (m->rec_ez[r] / TZ) * L.ntx + m->rec_ex[r] / TX;
        tcount[rtile[r] + 1]++;
    }
    for (int t = 0; t < ntiles; ++t) tcount[t + 1] += tcount[t];
    {
        std::vector<int> fill(tcount.begin(), tcount.end() - 1);
        for (int r = 0; r < m->nrec; ++r) rlist[fill[rtile[r]]++] = r;
    }
    auto up = [&](DevBuf &b, const void *h, size_t n) -> int {
        GB_TRY(b.ensure(std::max<size_t>(n, 16)));
        if (n) GB_CUDA(cudaMemcpy(b.p, h, n, cudaMemcpyHostToDevice));
        return GBFWI_OK;
    };
    if (sgptr.empty()) sgptr.assign(ntiles + 1, 0);
    GB_TRY(up(L.src_gptr, sgptr.data(), sgptr.size() * sizeof(int)));
    GB_TRY(up(L.src_groups, sgroups.data(), sgroups.size() * sizeof(InjGroup)));
    GB_TRY(up(L.src_entries, sentries.data(), sentries.size() * sizeof(InjEntry)));
    GB_TRY(up(L.rec_gptr, rgptr.data(), rgptr.size() * sizeof(int)));
    GB_TRY(up(L.rec_groups, rgroups.data(), rgroups.size() * sizeof(InjGroup)));
    GB_TRY(up(L.rec_entries, rentries.data(), rentries.size() * sizeof(InjEntry)));
    GB_TRY(up(L.rec_tptr, tcount.data(), tcount.size() * sizeof(int)));
    GB_TRY(up(L.rec_list, rlist.data(), rlist.size() * sizeof(int)));
    L.built = true;
    return GBFWI_OK;
}

// ---------------------------------------------------------------------------
// model
// ---------------------------------------------------------------------------

__global__ void material_kernel(const float *__restrict__ model, const float *__restrict__ wx,
                                const float *__restrict__ wz, const float4 *__restrict__ bw, int nx,
                                int nz, int pitch, float dt, float2 *__restrict__ lm,
                                float *__restrict__ minv, float4 *__restrict__ bnd)
{
    long long NP = (long long)nz * pitch;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < NP;
         g += (long long)gridDim.x * blockDim.x) {
        int iz = (int)(g / pitch), ix = (int)(g - (long long)iz * pitch);
        if (ix >= nx) {
            lm[g] = make_float2(0.f, 0.f);
            minv[g] = 0.f;
            bnd[g] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        float rho = model[g], vp = model[NP + g], vs = model[2 * NP + g];
        float mu = rho * vs * vs;
        float lam = rho * vp * vp - 2.f * mu;
        float M = rho * wx[ix] * wz[iz];
        float4 w = bw[g];
        float cx = rho * vp * w.x + rho * vs * w.z;
        float cz = rho * vp * w.y + rho * vs * w.w;
        lm[g] = make_float2(lam, mu);
        minv[g] = 1.f / M;
        bnd[g] = make_float4(cx, cz, 1.f / (M + 0.5f * dt * cx), 1.f / (M + 0.5f * dt * cz));
    }
}

extern "C" int gbfwi_set_model(gbfwi_mesh *m, const float *rho, const float *vp, const float *vs,
                               void *stream)
{
    if (!m || !rho || !vp || !vs) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(rho, vp, vs));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)m->nx * m->nz;
    std::vector<float> h(3 * N);
    const float *src[3] = {rho, vp, vs};
    for (int c = 0; c < 3; ++c) {
        if (gb_is_device_ptr(src[c]))
            GB_CUDA(cudaMemcpyAsync(h.data() + c * N, src[c], N * sizeof(float), cudaMemcpyDeviceToHost, s));
        else
            std::memcpy(h.data() + c * N, src[c], N * sizeof(float));
    }
    GB_CUDA(cudaStreamSynchronize(s));
    double vmax = 0;
    for (size_t g = 0; g < N; ++g) {
        float r = h[g], p = h[N + g], q = h[2 * N + g];
        if (!std::isfinite(r) || !std::isfinite(p) || !std::isfinite(q)) return gb_nonfinite("model parameter");
        if (!(r > 0) || !(q > 0) || !(p > q)) return GBFWI_EINVAL;
        vmax = std::max(vmax, (double)p);
    }
    if (m->d.dt * vmax / m->dx_min > 0.5) return GBFWI_ECFL;
    // pitched upload
    const size_t NP = (size_t)m->nz * m->pitch;
    std::vector<float> hp(3 * NP, 0.f);
    for (int c = 0; c < 3; ++c)
        for (int iz = 0; iz < m->nz; ++iz)
            std::memcpy(&hp[c * NP + (size_t)iz * m->pitch], &h[c * N + (size_t)iz * m->nx],
                        m->nx * sizeof(float));
    GB_CUDA(cudaMemcpyAsync(m->d_model.p, hp.data(), 3 * NP * sizeof(float), cudaMemcpyHostToDevice, s));
    material_kernel<<<304, 256, 0, s>>>(m->d_model.as<float>(), m->d_wx.as<float>(), m->d_wz.as<float>(),
                                        m->d_bw.as<float4>(), m->nx, m->nz, m->pitch, (float)m->d.dt,
                                        m->d_lm.as<float2>(), m->d_minv.as<float>(), m->d_bnd.as<float4>());
    GB_LAUNCHED();
    GB_CUDA(cudaStreamSynchronize(s));
    m->have_model = true;
    return GBFWI_OK;
}
