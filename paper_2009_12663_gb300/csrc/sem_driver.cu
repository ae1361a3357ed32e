// Simulation driver of the gbfwi library: forward runs, misfit + adjoint
// gradient, and the diagonal preconditioners, as sequences of step launches
// (sem_step.cu) plus a few small kernels.
//
// Time indexing (records s_n = P u_n, n = 1..nt; sources F_n = f stf(t_n)):
//   forward launch n (n = 0..nt-1) reads u_{n+1}, vh_n, uses F_{n+1}, records
//   s_{n+1} and writes u_{n+2}, vh_{n+1};
//   adjoint launch j (j = 0..nt-1) is the same recurrence for w (w_0 = w_1 =
//   0) driven by F_{j+1} = P^T r_{nt-j} / dt; w_{j+1} is the Lagrange
//   multiplier lam_k with k = nt - j, which is correlated with u_k:
//     g = -dt^2 sum_k u_k^T [dM/dm a^w + dC/dm v^w + dK/dm w]
//   (the discrete gradient of Eqs. A16-A18 after summation by parts in time).
//
// Storage: fields are [slot][shot][nz][pitch] float2.  The forward history is
// either kept whole (nt + 2 slots) or as snapshots every C steps with the
// segment recomputed into C + 2 slots during the backward pass.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "gbfwi_internal.h"

namespace {

struct Ctx {
    gbfwi_mesh *m;
    TileLists *L;
    int tile;
    int B;                 // shots in this batch
    cudaStream_t s;
    const int *d_shots;    // [B] source ids
    long long NP;          // nz * pitch
};

void base_args(StepArgs &a, const Ctx &c)
{
    std::memset(&a, 0, sizeof(a));
    gbfwi_mesh *m = c.m;
    a.nex = m->d.nex; a.nez = m->d.nez; a.nx = m->nx; a.nz = m->nz; a.pitch = m->pitch;
    a.dt = (float)m->d.dt;
    a.fstride = c.NP;
    a.hstride = c.NP;
    a.lm = m->d_lm.as<float2>();
    a.minv = m->d_minv.as<float>();
    a.bnd = m->d_bnd.as<float4>();
    a.bw = m->d_bw.as<float4>();
    a.wxs = m->d_wx.as<float>();
    a.wzs = m->d_wz.as<float>();
    a.ntiles = c.L->ntx * c.L->ntz;
    a.rec_tptr = c.L->rec_tptr.as<int>();
    a.rec_list = c.L->rec_list.as<int>();
    a.recw = m->d_recw.as<float>();
    a.rec_e = m->d_rec_e.as<int2>();
    a.nt = m->d.nt;
    a.seis_shot_stride = (long long)m->nrec * 2 * m->d.nt;
    a.status = m->w_status.as<int>();
}

using SlotFn = std::function<float2 *(int)>;

// forward launches n in [n0, n1)
int fwd_range(const Ctx &c, int mode, int n0, int n1, const SlotFn &slot, float2 *vh, float *seis,
              float *acc, long long acc_shot_stride, long long acc_comp_stride)
{
    StepArgs a;
    base_args(a, c);
    a.vh = vh;
    a.gptr = c.L->src_gptr.as<int>();
    a.groups = c.L->src_groups.as<InjGroup>();
    a.entries = c.L->src_entries.as<InjEntry>();
    a.per_shot_groups = 1;
    a.sig = c.m->d_stf.as<float>();
    a.sig_shot_stride = c.m->d.nt + 1;
    a.sig_chan_stride = 0;
    a.sig_scale = 1.0f;
    a.shot_map = c.d_shots;
    a.seis = seis;
    a.acc = acc;
    a.acc_shot_stride = acc_shot_stride;
    a.acc_comp_stride = acc_comp_stride;
    for (int n = n0; n < n1; ++n) {
        a.ucur = slot(n + 1);
        a.unext = slot(n + 2);
        a.uold = slot(n);
        a.tsig = n + 1;
        a.trec = n;
        GB_TRY(gb_launch_step(mode, c.tile, a, c.B, c.s));
    }
    return GBFWI_OK;
}

// adjoint launches j in [j0, j1); the adjoint field cycles through wring[3]
int adj_range(const Ctx &c, int mode, int j0, int j1, float2 *wring, float2 *wh, const SlotFn &hist,
              const float *sig, float *acc, long long acc_shot_stride, long long acc_comp_stride)
{
    const int nt = c.m->d.nt;
    StepArgs a;
    base_args(a, c);
    a.vh = wh;
    a.gptr = c.L->rec_gptr.as<int>();
    a.groups = c.L->rec_groups.as<InjGroup>();
    a.entries = c.L->rec_entries.as<InjEntry>();
    a.per_shot_groups = 0;
    a.sig = sig;
    a.sig_shot_stride = (long long)2 * c.m->nrec * nt;
    a.sig_chan_stride = nt;
    a.sig_scale = (float)(1.0 / c.m->d.dt);
    a.shot_map = nullptr;
    a.acc = acc;
    a.acc_shot_stride = acc_shot_stride;
    a.acc_comp_stride = acc_comp_stride;
    const long long lev = (long long)c.B * c.NP;
    for (int j = j0; j < j1; ++j) {
        int k = nt - j;
        a.ucur = wring + ((j + 1) % 3) * lev;
        a.unext = wring + ((j + 2) % 3) * lev;
        a.uold = wring + (j % 3) * lev;
        if (mode == MODE_ADJ_G) {
            a.h0 = hist(k);
        } else {
            a.h0 = hist(k + 1);
            a.h1 = hist(k);
            a.h2 = hist(k - 1);
        }
        a.tsig = nt - 1 - j;
        GB_TRY(gb_launch_step(mode, c.tile, a, c.B, c.s));
    }
    return GBFWI_OK;
}

}  // namespace

int gb_take_status(gbfwi_mesh *m)
{
    int st = 0;
    GB_CUDA(cudaMemcpy(&st, m->w_status.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) {
        GB_CUDA(cudaMemset(m->w_status.p, 0, sizeof(int)));
        return GBFWI_ETIMEOUT;
    }
    return GBFWI_OK;
}

namespace {

// ------------------------------------------------------------------ kernels

// r = s - d in place, per-shot partial sums of r^2: grid (kMisfitBlocks, B)
constexpr int kMisfitBlocks = 64;

__global__ void residual_kernel(float *__restrict__ syn, const float *__restrict__ obs, long long per_shot,
                                double *__restrict__ partial, int *__restrict__ flag)
{
    const int shot = blockIdx.y;
    float *s = syn + (long long)shot * per_shot;
    const float *d = obs + (long long)shot * per_shot;
    double acc = 0.0;
    int bad = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < per_shot;
         q += (long long)gridDim.x * blockDim.x) {
        float r = s[q] - d[q];
        if (!isfinite(r)) bad = 1;
        s[q] = r;
        acc += (double)r * (double)r;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[shot * kMisfitBlocks + blockIdx.x] = red[0];
    if (bad) atomicOr(flag, 1);
}

// total += 1/2 dt sum_b partial[s][b], shot by shot in order, so the result
// does not depend on how the shots were batched
__global__ void misfit_finish(const double *__restrict__ partial, int nshot, double half_dt,
                              double *__restrict__ total)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = *total;
        for (int sh = 0; sh < nshot; ++sh) {
            double s = 0.0;
            for (int b = 0; b < kMisfitBlocks; ++b) s += partial[sh * kMisfitBlocks + b];
            t += half_dt * s;
        }
        *total = t;
    }
}

__global__ void finite_check(const float *__restrict__ x, long long n, int *__restrict__ flag)
{
    int bad = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x)
        if (!isfinite(x[q])) bad = 1;
    if (bad) atomicOr(flag, 1);
}

// total[c][g] += sum_b acc[b][c][g]  (fixed order over b)
__global__ void acc_reduce(const float *__restrict__ acc, int B, int ncomp, long long NP,
                           float *__restrict__ total)
{
    long long n = (long long)ncomp * NP;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        float s = total[q];
        for (int b = 0; b < B; ++b) s += acc[(long long)b * n + q];
        total[q] = s;
    }
}

// gradient chain rule: (g_lambda, g_mu, sum u.a^w, g_Zp, g_Zs) -> (rho, vp, vs), times -dt^2;
// dM_g/drho_g = W_g = wx[ix] wz[iz]
__global__ void chain_kernel(const float *__restrict__ tot, const float *__restrict__ model,
                             const float *__restrict__ wx, const float *__restrict__ wz, int nx, int nz,
                             int pitch, float mdt2, float *__restrict__ grad)
{
    long long NP = (long long)nz * pitch, N = (long long)nz * nx;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
         q += (long long)gridDim.x * blockDim.x) {
        int iz = (int)(q / nx), ix = (int)(q - (long long)iz * nx);
        long long g = (long long)iz * pitch + ix;
        float gl = tot[g], gm = tot[NP + g], gp = tot[3 * NP + g], gs = tot[4 * NP + g];
        float gM = wx[ix] * wz[iz] * tot[2 * NP + g];
        float r = model[g], p = model[NP + g], s = model[2 * NP + g];
        float grho = gl * (p * p - 2.f * s * s) + gm * s * s + gM + gp * p + gs * s;
        float gvp = gl * (2.f * r * p) + gp * r;
        float gvs = gl * (-4.f * r * s) + gm * (2.f * r * s) + gs * r;
        grad[q] = mdt2 * grho;
        grad[N + q] = mdt2 * gvp;
        grad[2 * N + q] = mdt2 * gvs;
    }
}

// Preconditioner maps from the time integrals (Eqs. 5-8, A21-A22):
//   H_rho = W |f0 S0|, H_a = 8 rho^2 vp^2 |f1 S1|,
//   H_b = 16 rho^2 vs^2 |f1 S2| + 4 rho^2 vs^2 |f1 S3|
// kind 1/2 replicate H_rho.  Output [3][nz][nx].
__global__ void precond_finish(const float *__restrict__ tot, const float *__restrict__ model,
                               const float *__restrict__ wx, const float *__restrict__ wz, int nx, int nz,
                               int pitch, int kind, float f0, float f1, float *__restrict__ H)
{
    long long NP = (long long)nz * pitch, N = (long long)nz * nx;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
         q += (long long)gridDim.x * blockDim.x) {
        int iz = (int)(q / nx), ix = (int)(q - (long long)iz * nx);
        long long g = (long long)iz * pitch + ix;
        float hr = wx[ix] * wz[iz] * fabsf(f0 * tot[g]);
        float ha = hr, hb = hr;
        if (kind >= 3) {
            float r = model[g], p = model[NP + g], s = model[2 * NP + g];
            float r2 = r * r;
            ha = 8.f * r2 * p * p * fabsf(f1 * tot[NP + g]);
            hb = 16.f * r2 * s * s * fabsf(f1 * tot[2 * NP + g]) + 4.f * r2 * s * s * fabsf(f1 * tot[3 * NP + g]);
        }
        H[q] = hr;
        H[N + q] = ha;
        H[2 * N + q] = hb;
    }
}

// Separable Gaussian smoothing along one axis of [3][nz][nx]:
// out(i) = sum_j G(c_i - c_j) w_j f(j) / sum_j G(c_i - c_j) w_j over |c_i - c_j| <= 5 sigma
__global__ void smooth_axis(const float *__restrict__ in, float *__restrict__ out, int nx, int nz, int axis,
                            const float *__restrict__ coord, const float *__restrict__ wts,
                            const int2 *__restrict__ range, float inv2s2)
{
    long long N = (long long)nx * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 3 * N;
         q += (long long)gridDim.x * blockDim.x) {
        long long c = q / N, r = q - c * N;
        int iz = (int)(r / nx), ix = (int)(r - (long long)iz * nx);
        int i = axis == 0 ? ix : iz;
        int2 rg = range[i];
        float ci = coord[i];
        float num = 0.f, den = 0.f;
        const float *base = in + c * N;
        for (int jj = rg.x; jj <= rg.y; ++jj) {
            float d = ci - coord[jj];
            float gw = __expf(-d * d * inv2s2) * wts[jj];
            float f = axis == 0 ? base[(long long)iz * nx + jj] : base[(long long)jj * nx + ix];
            num = fmaf(gw, f, num);
            den += gw;
        }
        out[q] = num / den;
    }
}

// radix select of rank k over n floats (one parameter map), 8 bits per pass
__device__ __forceinline__ unsigned fkey(float f)
{
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void radix_hist(const float *__restrict__ x, long long n, const unsigned *__restrict__ state,
                           int shift, unsigned *__restrict__ hist)
{
    __shared__ unsigned h[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
    __syncthreads();
    unsigned prefix = state[0], mask = state[1];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        unsigned k = fkey(x[q]);
        if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        if (h[t]) atomicAdd(&hist[t], h[t]);
}

// state = {prefix, mask, rank}
__global__ void radix_pick(unsigned *__restrict__ state, unsigned *__restrict__ hist, int shift,
                           float *__restrict__ result)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned rank = state[2], cum = 0;
    int bin = 0;
    for (; bin < 256; ++bin) {
        if (cum + hist[bin] > rank) break;
        cum += hist[bin];
    }
    if (bin > 255) bin = 255;
    state[0] |= ((unsigned)bin) << shift;
    state[1] |= 0xFFu << shift;
    state[2] = rank - cum;
    for (int t = 0; t < 256; ++t) hist[t] = 0;
    if (shift == 0) {
        unsigned k = state[0];
        unsigned u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
        *result = __uint_as_float(u);
    }
}

__global__ void radix_init(unsigned *__restrict__ state, unsigned rank)
{
    if (threadIdx.x == 0) { state[0] = 0; state[1] = 0; state[2] = rank; }
}

__global__ void b0_kernel(const float *__restrict__ S, const float *__restrict__ med, long long N, float damp,
                          float *__restrict__ B0)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 3 * N;
         q += (long long)gridDim.x * blockDim.x) {
        int c = (int)(q / N);
        B0[q] = 1.f / (S[q] + damp * med[c]);
    }
}

// ------------------------------------------------------------------ helpers

int grid_for(long long n) { return (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 152 * 8); }

struct Staged {
    const void *dptr = nullptr;
};

int stage_in(DevBuf &buf, const void *user, size_t bytes, cudaStream_t s, const void **dptr)
{
    if (gb_is_device_ptr(user)) { *dptr = user; return GBFWI_OK; }
    GB_TRY(buf.ensure(bytes));
    GB_CUDA(cudaMemcpyAsync(buf.p, user, bytes, cudaMemcpyHostToDevice, s));
    *dptr = buf.p;
    return GBFWI_OK;
}

int check_shots(const gbfwi_mesh *m, const int *shot_ids, int nshot)
{
    if (nshot < 1 || !shot_ids) return GBFWI_EINVAL;
    for (int i = 0; i < nshot; ++i)
        if (shot_ids[i] < 0 || shot_ids[i] >= (int)m->src.size()) return GBFWI_EINVAL;
    return GBFWI_OK;
}

// history layout for one batch
struct History {
    float2 *base = nullptr;    // [slots][B][NP]
    int slots = 0;
    int kbase = 0;             // time level held by slot 0
    long long lev = 0;         // B * NP
    float2 *at(int k) const { return base + (long long)(k - kbase) * lev; }
};

}  // namespace

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------

extern "C" int gbfwi_forward(gbfwi_mesh *m, const int *shot_ids, int nshot, float *seis, void *stream)
{
    if (!m || !seis) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(seis));
    GB_TRY(check_shots(m, shot_ids, nshot));
    if (!m->have_model) return GBFWI_ENOMODEL;
    cudaStream_t s = (cudaStream_t)stream;
    const int tile = m->sch.tile;
    GB_TRY(gb_build_tile_lists(m, tile));
    const int nt = m->d.nt;
    const long long NP = (long long)m->nz * m->pitch;
    const int Bmax = std::min(m->sch.shots_per_launch, nshot);
    const size_t seis_shot = (size_t)m->nrec * 2 * nt;
    const bool dev_out = gb_is_device_ptr(seis);
    GB_TRY(m->w_hist.ensure((size_t)3 * Bmax * NP * sizeof(float2)));
    GB_TRY(m->w_vh.ensure((size_t)Bmax * NP * sizeof(float2)));
    GB_TRY(m->w_shots.ensure((size_t)nshot * sizeof(int)));
    if (!dev_out) GB_TRY(m->w_seis.ensure(seis_shot * Bmax * sizeof(float)));
    GB_CUDA(cudaMemcpyAsync(m->w_shots.p, shot_ids, nshot * sizeof(int), cudaMemcpyHostToDevice, s));
    for (int i0 = 0; i0 < nshot; i0 += Bmax) {
        int B = std::min(Bmax, nshot - i0);
        Ctx c{m, &m->lists[tile], tile, B, s, m->w_shots.as<int>() + i0, NP};
        float2 *ring = m->w_hist.as<float2>();
        long long lev = (long long)B * NP;
        GB_CUDA(cudaMemsetAsync(ring, 0, 3 * lev * sizeof(float2), s));
        GB_CUDA(cudaMemsetAsync(m->w_vh.p, 0, lev * sizeof(float2), s));
        float *out = dev_out ? seis + seis_shot * i0 : m->w_seis.as<float>();
        SlotFn slot = [&](int k) { return ring + (long long)(k % 3) * lev; };
        GB_TRY(fwd_range(c, MODE_FWD, 0, nt, slot, m->w_vh.as<float2>(), out, nullptr, 0, 0));
        if (!dev_out)
            GB_CUDA(cudaMemcpyAsync(seis + seis_shot * i0, out, seis_shot * B * sizeof(float),
                                    cudaMemcpyDeviceToHost, s));
    }
    if (!dev_out) {
        GB_CUDA(cudaStreamSynchronize(s));
        GB_TRY(gb_take_status(m));
    }
    return GBFWI_OK;
}

// ---------------------------------------------------------------------------
// misfit only
// ---------------------------------------------------------------------------

extern "C" int gbfwi_misfit(gbfwi_mesh *m, const int *shot_ids, int nshot, const float *d_obs, double *misfit,
                            void *stream)
{
    if (!m || !d_obs || !misfit) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(d_obs, misfit));
    GB_TRY(check_shots(m, shot_ids, nshot));
    if (!m->have_model) return GBFWI_ENOMODEL;
    cudaStream_t s = (cudaStream_t)stream;
    const int tile = m->sch.tile;
    GB_TRY(gb_build_tile_lists(m, tile));
    const int nt = m->d.nt;
    const long long NP = (long long)m->nz * m->pitch;
    const int Bmax = std::min(m->sch.shots_per_launch, nshot);
    const size_t seis_shot = (size_t)m->nrec * 2 * nt;
    GB_TRY(m->w_hist.ensure((size_t)3 * Bmax * NP * sizeof(float2)));
    GB_TRY(m->w_vh.ensure((size_t)Bmax * NP * sizeof(float2)));
    GB_TRY(m->w_shots.ensure((size_t)nshot * sizeof(int)));
    GB_TRY(m->w_seis.ensure(seis_shot * Bmax * sizeof(float)));
    const int npart = kMisfitBlocks * Bmax;
    GB_TRY(m->w_red.ensure((size_t)(npart + 8) * sizeof(double) + 4096));
    GB_TRY(m->w_flag.ensure(16));
    const void *obs_d = nullptr;
    GB_TRY(stage_in(m->w_obs, d_obs, seis_shot * nshot * sizeof(float), s, &obs_d));
    double *partial = m->w_red.as<double>();
    double *mis_d = partial + npart;
    int *flag = m->w_flag.as<int>();
    GB_CUDA(cudaMemcpyAsync(m->w_shots.p, shot_ids, nshot * sizeof(int), cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaMemsetAsync(mis_d, 0, sizeof(double), s));
    GB_CUDA(cudaMemsetAsync(flag, 0, 16, s));
    for (int i0 = 0; i0 < nshot; i0 += Bmax) {
        int B = std::min(Bmax, nshot - i0);
        Ctx c{m, &m->lists[tile], tile, B, s, m->w_shots.as<int>() + i0, NP};
        float2 *ring = m->w_hist.as<float2>();
        long long lev = (long long)B * NP;
        GB_CUDA(cudaMemsetAsync(ring, 0, 3 * lev * sizeof(float2), s));
        GB_CUDA(cudaMemsetAsync(m->w_vh.p, 0, lev * sizeof(float2), s));
        SlotFn slot = [&](int k) { return ring + (long long)(k % 3) * lev; };
        float *seis_d = m->w_seis.as<float>();
        GB_TRY(fwd_range(c, MODE_FWD, 0, nt, slot, m->w_vh.as<float2>(), seis_d, nullptr, 0, 0));
        residual_kernel<<<dim3(kMisfitBlocks, B), 256, 0, s>>>(seis_d, (const float *)obs_d + seis_shot * i0,
                                                              (long long)seis_shot, partial, flag);
        GB_LAUNCHED();
        misfit_finish<<<1, 32, 0, s>>>(partial, B, 0.5 * m->d.dt, mis_d);
        GB_LAUNCHED();
    }
    double mis_h = 0;
    int flag_h = 0;
    GB_CUDA(cudaMemcpyAsync(&mis_h, mis_d, sizeof(double), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(&flag_h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    GB_TRY(gb_take_status(m));
    if (flag_h || !std::isfinite(mis_h)) return gb_nonfinite("misfit");
    *misfit = mis_h;
    return GBFWI_OK;
}

// ---------------------------------------------------------------------------
// forward pass with history (full) or snapshots (checkpointed) for one batch
// ---------------------------------------------------------------------------

namespace {

struct BatchHist {
    History full;              // ckpt == 0
    float2 *ring = nullptr;    // ckpt > 0: 3-slot ring for the forward pass
    float2 *seg = nullptr;     // ckpt > 0: C + 2 slots
    float2 *snap = nullptr;    // ckpt > 0: [nseg][3][B][NP]: u_{sC}, u_{sC+1}, vh_{sC}
    float2 *vh_rec = nullptr;  // recompute velocity
    float2 *vh = nullptr;      // forward half-step velocity
    float2 *wring = nullptr;   // adjoint field, 3 levels
    float2 *wh = nullptr;      // adjoint half-step velocity
    int C = 0, nseg = 0;
};

// the work buffers of one concurrent lane
struct LaneRef {
    DevBuf *hist, *snap, *vh, *adj, *wh, *seis, *batch, *acc;
    cudaStream_t st;
};

LaneRef lane0(gbfwi_mesh *m, cudaStream_t s)
{
    return LaneRef{&m->w_hist, &m->w_snap, &m->w_vh, &m->w_adj, &m->w_wh, &m->w_seis, &m->w_batch, &m->w_lacc, s};
}

int alloc_hist(gbfwi_mesh *m, const LaneRef &L, int B, int ckpt, long long NP, BatchHist &h, bool adjoint)
{
    const int nt = m->d.nt;
    long long lev = (long long)B * NP;
    if (ckpt <= 0 || ckpt >= nt) {
        GB_TRY(L.hist->ensure((size_t)(nt + 2) * lev * sizeof(float2)));
        h.full.base = L.hist->as<float2>();
        h.full.slots = nt + 2;
        h.full.kbase = 0;
        h.full.lev = lev;
        h.C = 0;
    } else {
        h.C = ckpt;
        h.nseg = (nt + ckpt - 1) / ckpt;
        size_t ring = 3, seg = (size_t)ckpt + 2, snap = (size_t)h.nseg * 3, vrec = 1;
        GB_TRY(L.hist->ensure((ring + seg + vrec) * lev * sizeof(float2)));
        GB_TRY(L.snap->ensure(snap * lev * sizeof(float2)));
        h.ring = L.hist->as<float2>();
        h.seg = h.ring + ring * lev;
        h.vh_rec = h.seg + seg * lev;
        h.snap = L.snap->as<float2>();
    }
    GB_TRY(L.vh->ensure(lev * sizeof(float2)));
    h.vh = L.vh->as<float2>();
    if (adjoint) {
        GB_TRY(L.adj->ensure(3 * lev * sizeof(float2)));
        GB_TRY(L.wh->ensure(lev * sizeof(float2)));
        h.wring = L.adj->as<float2>();
        h.wh = L.wh->as<float2>();
    }
    return GBFWI_OK;
}

// forward over all launches, recording into seis (device, [B][nrec][2][nt])
int forward_pass(const Ctx &c, BatchHist &h, float *seis)
{
    gbfwi_mesh *m = c.m;
    const int nt = m->d.nt;
    const long long lev = (long long)c.B * c.NP;
    float2 *vh = h.vh;
    GB_CUDA(cudaMemsetAsync(vh, 0, lev * sizeof(float2), c.s));
    if (h.C == 0) {
        GB_CUDA(cudaMemsetAsync(h.full.base, 0, 2 * lev * sizeof(float2), c.s));
        SlotFn slot = [&](int k) { return h.full.at(k); };
        return fwd_range(c, MODE_FWD, 0, nt, slot, vh, seis, nullptr, 0, 0);
    }
    GB_CUDA(cudaMemsetAsync(h.ring, 0, 3 * lev * sizeof(float2), c.s));
    SlotFn slot = [&](int k) { return h.ring + (long long)(k % 3) * lev; };
    for (int sg = 0; sg < h.nseg; ++sg) {
        int n0 = sg * h.C, n1 = std::min(nt, n0 + h.C);
        float2 *sp = h.snap + (long long)sg * 3 * lev;
        GB_CUDA(cudaMemcpyAsync(sp, slot(n0), lev * sizeof(float2), cudaMemcpyDeviceToDevice, c.s));
        GB_CUDA(cudaMemcpyAsync(sp + lev, slot(n0 + 1), lev * sizeof(float2), cudaMemcpyDeviceToDevice, c.s));
        GB_CUDA(cudaMemcpyAsync(sp + 2 * lev, vh, lev * sizeof(float2), cudaMemcpyDeviceToDevice, c.s));
        GB_TRY(fwd_range(c, MODE_FWD, n0, n1, slot, vh, seis, nullptr, 0, 0));
    }
    return GBFWI_OK;
}

// adjoint over all launches; segments recomputed when checkpointed
int adjoint_pass(const Ctx &c, BatchHist &h, int mode, const float *sig, float *acc, long long acc_shot_stride,
                 long long acc_comp_stride)
{
    gbfwi_mesh *m = c.m;
    const int nt = m->d.nt;
    const long long lev = (long long)c.B * c.NP;
    float2 *wring = h.wring;
    float2 *wh = h.wh;
    GB_CUDA(cudaMemsetAsync(wring, 0, 3 * lev * sizeof(float2), c.s));
    GB_CUDA(cudaMemsetAsync(wh, 0, lev * sizeof(float2), c.s));
    if (h.C == 0) {
        SlotFn hist = [&](int k) { return h.full.at(k); };
        return adj_range(c, mode, 0, nt, wring, wh, hist, sig, acc, acc_shot_stride, acc_comp_stride);
    }
    for (int sg = h.nseg - 1; sg >= 0; --sg) {
        int n0 = sg * h.C, n1 = std::min(nt, n0 + h.C);
        float2 *sp = h.snap + (long long)sg * 3 * lev;
        History seg{h.seg, h.C + 2, n0, lev};
        GB_CUDA(cudaMemcpyAsync(seg.at(n0), sp, lev * sizeof(float2), cudaMemcpyDeviceToDevice, c.s));
        GB_CUDA(cudaMemcpyAsync(seg.at(n0 + 1), sp + lev, lev * sizeof(float2), cudaMemcpyDeviceToDevice, c.s));
        GB_CUDA(cudaMemcpyAsync(h.vh_rec, sp + 2 * lev, lev * sizeof(float2), cudaMemcpyDeviceToDevice, c.s));
        SlotFn slot = [&](int k) { return seg.at(k); };
        GB_TRY(fwd_range(c, MODE_FWD, n0, n1, slot, h.vh_rec, nullptr, nullptr, 0, 0));
        // adjoint launches whose correlation level k lies in [n0 + 1, n1]
        int j0 = nt - n1, j1 = nt - n0;
        GB_TRY(adj_range(c, mode, j0, j1, wring, wh, slot, sig, acc, acc_shot_stride, acc_comp_stride));
    }
    return GBFWI_OK;
}

// Run body() on the caller's stream s, or, with graphs enabled, replay a CUDA
// graph of it captured once on a private stream (the caller's stream may be
// the legacy default stream, which cannot be captured).
int run_pass(gbfwi_mesh *m, const std::string &key, cudaStream_t s, const std::function<int(cudaStream_t)> &body)
{
    if (!m->sch.use_graph) return body(s);
    for (auto &g : m->graphs)
        if (g.key == key) {
            GB_CUDA(cudaGraphLaunch(g.exec, s));
            gb_note_launches(g.kernels);
            return GBFWI_OK;
        }
    if (!m->cap_stream) GB_CUDA(cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
    // the capture stream must not run ahead of work already queued on s
    cudaEvent_t ready;
    GB_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    GB_CUDA(cudaEventRecord(ready, s));
    GB_CUDA(cudaStreamWaitEvent(m->cap_stream, ready, 0));
    GB_CUDA(cudaEventDestroy(ready));
    GB_CUDA(cudaStreamSynchronize(m->cap_stream));
    const long long before = gb_launches_so_far();
    GB_CUDA(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = body(m->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(m->cap_stream, &graph);
    // launches recorded during capture did not run: count them at replay
    const long long kernels = gb_launches_so_far() - before;
    gb_note_launches(-kernels);
    if (rc != GBFWI_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (rc == GBFWI_OK) {
            gb_set_last_cuda_error(ce, "cudaStreamEndCapture", __FILE__, __LINE__);
            rc = GBFWI_ECUDA;
        }
        return rc;
    }
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        gb_set_last_cuda_error(ce, "cudaGraphInstantiate", __FILE__, __LINE__);
        return GBFWI_ECUDA;
    }
    if (m->graphs.size() >= 16) {          // bounded cache
        cudaGraphExecDestroy(m->graphs.front().exec);
        m->graphs.erase(m->graphs.begin());
    }
    m->graphs.push_back({key, exec, kernels});
    GB_CUDA(cudaGraphLaunch(exec, s));
    gb_note_launches(kernels);
    return GBFWI_OK;
}

std::string pass_key(const char *what, const gbfwi_mesh *m, int B, int ckpt, std::initializer_list<const void *> ptrs)
{
    std::string k = what;
    k += "|" + std::to_string(m->sch.tile) + "|" + std::to_string(B) + "|" + std::to_string(ckpt);
    for (const void *p : ptrs) k += "|" + std::to_string((uintptr_t)p);
    return k;
}

}  // namespace

// ---------------------------------------------------------------------------
// misfit + gradient
// ---------------------------------------------------------------------------

extern "C" int gbfwi_adjoint_gradient(gbfwi_mesh *m, const int *shot_ids, int nshot, const float *d_obs,
                                      double *misfit, float *grad, int ckpt_every, void *stream)
{
    if (!m || !d_obs || !misfit || !grad) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(d_obs, misfit, grad));
    GB_TRY(check_shots(m, shot_ids, nshot));
    if (!m->have_model) return GBFWI_ENOMODEL;
    cudaStream_t s = (cudaStream_t)stream;
    const int tile = m->sch.tile;
    GB_TRY(gb_build_tile_lists(m, tile));
    const int nt = m->d.nt;
    const int ckpt = ckpt_every >= 0 ? ckpt_every : m->sch.ckpt_every;
    const long long NP = (long long)m->nz * m->pitch;
    const long long N = (long long)m->nz * m->nx;
    const int Bmax = std::min(m->sch.shots_per_launch, nshot);
    const size_t seis_shot = (size_t)m->nrec * 2 * nt;
    const int nbatch = (nshot + Bmax - 1) / Bmax;
    const int L = std::max(1, std::min(m->sch.streams, nbatch));

    // lanes: 0 = the mesh's own buffers on the caller's stream, 1.. = extra streams
    while ((int)m->lanes.size() < L - 1) m->lanes.push_back(new gbfwi_mesh::Lane());
    std::vector<LaneRef> lanes{lane0(m, s)};
    for (int l = 1; l < L; ++l) {
        gbfwi_mesh::Lane *ln = m->lanes[l - 1];
        if (!ln->st) GB_CUDA(cudaStreamCreateWithFlags(&ln->st, cudaStreamNonBlocking));
        lanes.push_back(
            LaneRef{&ln->hist, &ln->snap, &ln->vh, &ln->adj, &ln->wh, &ln->seis, &ln->batch, &ln->acc, ln->st});
    }
    std::vector<BatchHist> hs(L);
    for (int l = 0; l < L; ++l) {
        GB_TRY(alloc_hist(m, lanes[l], Bmax, ckpt, NP, hs[l], true));
        GB_TRY(lanes[l].seis->ensure(seis_shot * Bmax * sizeof(float)));
        GB_TRY(lanes[l].batch->ensure((size_t)Bmax * sizeof(int)));
        GB_TRY(lanes[l].acc->ensure((size_t)Bmax * 5 * NP * sizeof(float)));
    }
    // per-shot accumulators and misfit partials, reduced once in shot order at
    // the end: the result does not depend on batching or lanes
    GB_TRY(m->w_acc.ensure((size_t)nshot * 5 * NP * sizeof(float)));
    GB_TRY(m->w_grad.ensure((size_t)5 * NP * sizeof(float)));
    GB_TRY(m->w_shots.ensure((size_t)nshot * sizeof(int)));
    const int npart = kMisfitBlocks * nshot;
    GB_TRY(m->w_red.ensure((size_t)(npart + 8) * sizeof(double) + 4096));
    GB_TRY(m->w_flag.ensure(16));
    const void *obs_d = nullptr;
    GB_TRY(stage_in(m->w_obs, d_obs, seis_shot * nshot * sizeof(float), s, &obs_d));
    const bool dev_grad = gb_is_device_ptr(grad);
    float *grad_d = grad;
    if (!dev_grad) {
        GB_TRY(m->w_tmp.ensure((size_t)3 * N * sizeof(float)));
        grad_d = m->w_tmp.as<float>();
    }
    double *partial = m->w_red.as<double>();
    double *mis_d = partial + npart;
    int *flag = m->w_flag.as<int>();
    float *acc_all = m->w_acc.as<float>();
    GB_CUDA(cudaMemcpyAsync(m->w_shots.p, shot_ids, nshot * sizeof(int), cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaMemsetAsync(mis_d, 0, sizeof(double), s));
    GB_CUDA(cudaMemsetAsync(flag, 0, 16, s));
    float *tot = m->w_grad.as<float>();
    GB_CUDA(cudaMemsetAsync(tot, 0, 5 * NP * sizeof(float), s));
    m->timed_valid = false;
    if (m->timing) {
        while ((int)m->ev.size() < 4 * nbatch + 2 * L) {
            cudaEvent_t e;
            GB_CUDA(cudaEventCreate(&e));
            m->ev.push_back(e);
        }
        m->fwd_launches = m->adj_launches = 0;
    }
    GB_TRY(gb_prepare_step(MODE_FWD, tile));
    GB_TRY(gb_prepare_step(MODE_ADJ_G, tile));
    // fork the lanes off the caller's stream
    std::vector<cudaEvent_t> sync_ev(L);
    for (int l = 0; l < L; ++l) GB_CUDA(cudaEventCreateWithFlags(&sync_ev[l], cudaEventDisableTiming));
    GB_CUDA(cudaEventRecord(sync_ev[0], s));
    for (int l = 1; l < L; ++l) GB_CUDA(cudaStreamWaitEvent(lanes[l].st, sync_ev[0], 0));

    int rc = GBFWI_OK;
    for (int i0 = 0, bi = 0; i0 < nshot && rc == GBFWI_OK; i0 += Bmax, ++bi) {
        const int l = bi % L;
        const LaneRef &lr = lanes[l];
        BatchHist &h = hs[l];
        cudaStream_t ls = lr.st;
        const int B = std::min(Bmax, nshot - i0);
        auto step = [&]() -> int {
            auto mark = [&](int i) -> int {
                if (m->timing) GB_CUDA(cudaEventRecord(m->ev[i], ls));
                return GBFWI_OK;
            };
            // this batch's source ids at a fixed address, so captured passes replay for every batch
            GB_CUDA(cudaMemcpyAsync(lr.batch->p, m->w_shots.as<int>() + i0, B * sizeof(int),
                                    cudaMemcpyDeviceToDevice, ls));
            Ctx c{m, &m->lists[tile], tile, B, ls, lr.batch->as<int>(), NP};
            float *seis_d = lr.seis->as<float>();
            float *acc = lr.acc->as<float>();
            const std::string kf = pass_key("fwd", m, B, h.C, {lr.hist->p, lr.vh->p, lr.seis->p, lr.snap->p,
                                                               lr.batch->p});
            const std::string ka = pass_key("adj", m, B, h.C, {lr.hist->p, lr.seis->p, lr.snap->p, lr.adj->p,
                                                               lr.wh->p, lr.acc->p});
            GB_TRY(mark(4 * bi));
            GB_TRY(run_pass(m, kf, ls, [&](cudaStream_t cs) {
                Ctx cc = c;
                cc.s = cs;
                return forward_pass(cc, h, seis_d);
            }));
            GB_TRY(mark(4 * bi + 1));
            // residual r = s - d (in place), per-shot partial sums of r^2
            residual_kernel<<<dim3(kMisfitBlocks, B), 256, 0, ls>>>(seis_d, (const float *)obs_d + seis_shot * i0,
                                                                   (long long)seis_shot,
                                                                   partial + (long long)kMisfitBlocks * i0, flag);
            GB_LAUNCHED();
            GB_TRY(mark(4 * bi + 2));
            GB_TRY(run_pass(m, ka, ls, [&](cudaStream_t cs) -> int {
                Ctx cc = c;
                cc.s = cs;
                GB_CUDA(cudaMemsetAsync(acc, 0, (size_t)B * 5 * NP * sizeof(float), cs));
                return adjoint_pass(cc, h, MODE_ADJ_G, seis_d, acc, 5 * NP, NP);
            }));
            GB_TRY(mark(4 * bi + 3));
            GB_CUDA(cudaMemcpyAsync(acc_all + (long long)i0 * 5 * NP, acc, (size_t)B * 5 * NP * sizeof(float),
                                    cudaMemcpyDeviceToDevice, ls));
            m->fwd_launches += nt;
            m->adj_launches += (h.C == 0) ? nt : 2LL * nt;
            return GBFWI_OK;
        };
        rc = step();
    }
    // join the lanes back into the caller's stream (also after an error)
    for (int l = 1; l < L; ++l) {
        cudaEventRecord(sync_ev[l], lanes[l].st);
        cudaStreamWaitEvent(s, sync_ev[l], 0);
    }
    for (int l = 0; l < L; ++l) cudaEventDestroy(sync_ev[l]);
    if (rc != GBFWI_OK) return rc;
    misfit_finish<<<1, 32, 0, s>>>(partial, nshot, 0.5 * m->d.dt, mis_d);
    GB_LAUNCHED();
    acc_reduce<<<grid_for(5 * NP), 256, 0, s>>>(acc_all, nshot, 5, NP, tot);
    GB_LAUNCHED();
    const float dt = (float)m->d.dt;
    chain_kernel<<<grid_for(N), 256, 0, s>>>(tot, m->d_model.as<float>(), m->d_wx.as<float>(), m->d_wz.as<float>(),
                                             m->nx, m->nz, m->pitch, -dt * dt, grad_d);
    GB_LAUNCHED();
    finite_check<<<grid_for(3 * N), 256, 0, s>>>(grad_d, 3 * N, flag);
    GB_LAUNCHED();
    double mis_h = 0;
    int flag_h = 0;
    GB_CUDA(cudaMemcpyAsync(&mis_h, mis_d, sizeof(double), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(&flag_h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    GB_TRY(gb_take_status(m));
    if (m->timing) {
        double fm = 0, am = 0;
        for (int bi = 0; bi < nbatch; ++bi) {
            float a = 0, b = 0;
            GB_CUDA(cudaEventElapsedTime(&a, m->ev[4 * bi], m->ev[4 * bi + 1]));
            GB_CUDA(cudaEventElapsedTime(&b, m->ev[4 * bi + 2], m->ev[4 * bi + 3]));
            fm += a;
            am += b;
        }
        m->fwd_ms = fm;
        m->adj_ms = am;
        m->timed_valid = true;
    }
    if (flag_h || !std::isfinite(mis_h)) return gb_nonfinite("misfit");
    if (!dev_grad) {
        GB_CUDA(cudaMemcpyAsync(grad, grad_d, 3 * N * sizeof(float), cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
    }
    *misfit = mis_h;
    return GBFWI_OK;
}

// ---------------------------------------------------------------------------
// preconditioners P1..P4, smoothing, damping, inversion
// ---------------------------------------------------------------------------

// B0 = 1 / (S(H) + damp * median(S(H))) per parameter from the raw map Hd
// [3][N] (device); S1, S2 scratch [3][N].  Writes B0 (device or host).
static int b0_from_map(gbfwi_mesh *m, const float *Hd, float *S1, float *S2, double sigma, double damp, float *B0,
                       cudaStream_t s)
{
    const long long N = (long long)m->nx * m->nz;
    // smoothing tables (node coordinates along each axis, 5-sigma index ranges)
    std::vector<float> cx(m->nx), cz(m->nz);
    std::vector<int2> rx(m->nx), rz(m->nz);
    {
        std::vector<double> X((size_t)m->nx * m->nz), Z((size_t)m->nx * m->nz);
        gbfwi_node_coords(m, X.data(), Z.data());
        for (int i = 0; i < m->nx; ++i) cx[i] = (float)X[i];
        for (int i = 0; i < m->nz; ++i) cz[i] = (float)Z[(size_t)i * m->nx];
        auto ranges = [&](const std::vector<float> &c, std::vector<int2> &r) {
            int n = (int)c.size();
            for (int i = 0; i < n; ++i) {
                int lo = i, hi = i;
                while (lo > 0 && c[i] - c[lo - 1] <= 5.0 * sigma) --lo;
                while (hi < n - 1 && c[hi + 1] - c[i] <= 5.0 * sigma) ++hi;
                r[i] = make_int2(lo, hi);
            }
        };
        ranges(cx, rx);
        ranges(cz, rz);
    }
    std::vector<float> wxf(m->wx1.begin(), m->wx1.end()), wzf(m->wz1.begin(), m->wz1.end());
    GB_TRY(m->w_stage.ensure((size_t)(m->nx + m->nz) * (2 * sizeof(float) + sizeof(int2)) + 64));
    char *tb = m->w_stage.as<char>();
    float *dcx = (float *)tb, *dcz = dcx + m->nx, *dwx = dcz + m->nz, *dwz = dwx + m->nx;
    int2 *drx = (int2 *)(((uintptr_t)(dwz + m->nz) + 15) & ~(uintptr_t)15), *drz = drx + m->nx;
    GB_CUDA(cudaMemcpyAsync(dcx, cx.data(), m->nx * sizeof(float), cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaMemcpyAsync(dcz, cz.data(), m->nz * sizeof(float), cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaMemcpyAsync(dwx, wxf.data(), m->nx * sizeof(float), cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaMemcpyAsync(dwz, wzf.data(), m->nz * sizeof(float), cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaMemcpyAsync(drx, rx.data(), m->nx * sizeof(int2), cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaMemcpyAsync(drz, rz.data(), m->nz * sizeof(int2), cudaMemcpyHostToDevice, s));
    float inv2s2 = (float)(1.0 / (2.0 * sigma * sigma));
    smooth_axis<<<grid_for(3 * N), 256, 0, s>>>(Hd, S1, m->nx, m->nz, 0, dcx, dwx, drx, inv2s2);
    GB_LAUNCHED();
    smooth_axis<<<grid_for(3 * N), 256, 0, s>>>(S1, S2, m->nx, m->nz, 1, dcz, dwz, drz, inv2s2);
    GB_LAUNCHED();
    // medians of the smoothed maps (rank (N-1)/2)
    GB_TRY(m->w_red.ensure((1024 + 8) * sizeof(double) + 4096));
    unsigned *rstate = (unsigned *)(m->w_red.as<char>() + (1024 + 8) * sizeof(double));   // radix-select state
    unsigned *rhist = rstate + 4;
    float *med = (float *)(rhist + 256);
    GB_CUDA(cudaMemsetAsync(rhist, 0, 256 * sizeof(unsigned), s));
    for (int c = 0; c < 3; ++c) {
        radix_init<<<1, 32, 0, s>>>(rstate, (unsigned)((N - 1) / 2));
        for (int shift = 24; shift >= 0; shift -= 8) {
            radix_hist<<<grid_for(N), 256, 0, s>>>(S2 + c * N, N, rstate, shift, rhist);
            radix_pick<<<1, 32, 0, s>>>(rstate, rhist, shift, med + c);
        }
        GB_LAUNCHED();
    }
    const bool dev_b0 = gb_is_device_ptr(B0);
    float *B0d = dev_b0 ? B0 : S1;   // S1 is free after the second pass
    b0_kernel<<<grid_for(3 * N), 256, 0, s>>>(S2, med, N, (float)damp, B0d);
    GB_LAUNCHED();
    if (!dev_b0) GB_CUDA(cudaMemcpyAsync(B0, B0d, 3 * N * sizeof(float), cudaMemcpyDeviceToHost, s));
    return GBFWI_OK;
}

extern "C" int gbfwi_precond_diag(gbfwi_mesh *m, const int *shot_ids, int nshot, int kind, double sigma,
                                  double damp, float *H, float *B0, void *stream)
{
    if (!m || !B0 || kind < 1 || kind > 4 || !(sigma > 0) || !(damp >= 0)) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(H, B0));
    GB_TRY(check_shots(m, shot_ids, nshot));
    if (!m->have_model) return GBFWI_ENOMODEL;
    cudaStream_t s = (cudaStream_t)stream;
    const int tile = m->sch.tile;
    GB_TRY(gb_build_tile_lists(m, tile));
    const int nt = m->d.nt;
    const long long NP = (long long)m->nz * m->pitch;
    const long long N = (long long)m->nz * m->nx;
    const int Bmax = std::min(m->sch.shots_per_launch, nshot);
    const size_t seis_shot = (size_t)m->nrec * 2 * nt;
    const long long lev = (long long)Bmax * NP;
    const double dt = m->d.dt;

    GB_TRY(m->w_vh.ensure(lev * sizeof(float2)));
    GB_TRY(m->w_pc.ensure((size_t)Bmax * 4 * NP * sizeof(float)));
    GB_TRY(m->w_grad.ensure((size_t)5 * NP * sizeof(float)));
    GB_TRY(m->w_shots.ensure((size_t)nshot * sizeof(int)));
    BatchHist h;
    if (kind == 2 || kind == 4) {
        GB_TRY(alloc_hist(m, lane0(m, s), Bmax, m->sch.ckpt_every, NP, h, true));
        GB_TRY(m->w_seis.ensure(seis_shot * Bmax * sizeof(float)));
    } else {
        GB_TRY(m->w_hist.ensure((size_t)3 * lev * sizeof(float2)));
    }
    GB_CUDA(cudaMemcpyAsync(m->w_shots.p, shot_ids, nshot * sizeof(int), cudaMemcpyHostToDevice, s));
    float *tot = m->w_grad.as<float>();
    GB_CUDA(cudaMemsetAsync(tot, 0, 4 * NP * sizeof(float), s));
    for (int i0 = 0; i0 < nshot; i0 += Bmax) {
        int B = std::min(Bmax, nshot - i0);
        Ctx c{m, &m->lists[tile], tile, B, s, m->w_shots.as<int>() + i0, NP};
        float *acc = m->w_pc.as<float>();
        GB_CUDA(cudaMemsetAsync(acc, 0, (size_t)B * 4 * NP * sizeof(float), s));
        long long blev = (long long)B * NP;
        if (kind == 1 || kind == 3) {
            float2 *ring = m->w_hist.as<float2>();
            GB_CUDA(cudaMemsetAsync(ring, 0, 3 * blev * sizeof(float2), s));
            GB_CUDA(cudaMemsetAsync(m->w_vh.p, 0, blev * sizeof(float2), s));
            SlotFn slot = [&](int k) { return ring + (long long)(k % 3) * blev; };
            GB_TRY(fwd_range(c, MODE_FWD_PC, 0, nt, slot, m->w_vh.as<float2>(), nullptr, acc, 4 * NP, NP));
        } else {
            // receiver wavefield: adjoint recurrence driven by the synthetic data s(m0)
            float *seis_d = m->w_seis.as<float>();
            GB_TRY(forward_pass(c, h, seis_d));
            GB_TRY(adjoint_pass(c, h, MODE_ADJ_PC, seis_d, acc, 4 * NP, NP));
        }
        acc_reduce<<<grid_for(4 * NP), 256, 0, s>>>(acc, B, 4, NP, tot);
        GB_LAUNCHED();
    }
    // time-integral factors: forward mode S0 = sum a.a (x dt), S1..3 = sum of
    // products of undivided differences (x 1/dt); receiver mode S0 = sum of
    // (second difference) . a (x 1/dt)
    float f0 = (kind == 1 || kind == 3) ? (float)dt : (float)(1.0 / dt);
    float f1 = (float)(1.0 / dt);
    GB_TRY(m->w_tmp.ensure((size_t)9 * N * sizeof(float) + 4096));
    float *Hd = m->w_tmp.as<float>();
    float *S1 = Hd + 3 * N, *S2 = Hd + 6 * N;
    precond_finish<<<grid_for(N), 256, 0, s>>>(tot, m->d_model.as<float>(), m->d_wx.as<float>(),
                                               m->d_wz.as<float>(), m->nx, m->nz, m->pitch, kind, f0, f1, Hd);
    GB_LAUNCHED();

    GB_TRY(b0_from_map(m, Hd, S1, S2, sigma, damp, B0, s));
    if (H) {
        if (gb_is_device_ptr(H))
            GB_CUDA(cudaMemcpyAsync(H, Hd, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, s));
        else
            GB_CUDA(cudaMemcpyAsync(H, Hd, 3 * N * sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    GB_CUDA(cudaStreamSynchronize(s));
    GB_TRY(gb_take_status(m));
    return GBFWI_OK;
}

extern "C" int gbfwi_precond_from_hessian(gbfwi_mesh *m, const float *H, double sigma, double damp, float *B0,
                                          void *stream)
{
    if (!m || !H || !B0 || !(sigma > 0) || !(damp >= 0)) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(H, B0));
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = (long long)m->nx * m->nz;
    GB_TRY(m->w_tmp.ensure((size_t)9 * N * sizeof(float) + 4096));
    float *Hd = m->w_tmp.as<float>();
    float *S1 = Hd + 3 * N, *S2 = Hd + 6 * N;
    GB_CUDA(cudaMemcpyAsync(Hd, H, 3 * N * sizeof(float), cudaMemcpyDefault, s));
    GB_TRY(b0_from_map(m, Hd, S1, S2, sigma, damp, B0, s));
    GB_CUDA(cudaStreamSynchronize(s));
    return GBFWI_OK;
}
