// One time step of the 2-D isotropic elastic spectral-element scheme for a
// batch of shots (blockIdx.z), sm_103a.
//
// Scheme (Appendix A, Eqs. A6-A7, weak form; Newmark beta = 0, gamma = 1/2
// with implicit Stacey damping), state (u_{n+1}, vh_n = v_n + dt/2 a_n):
//   a_{n+1}  = (M + dt/2 C)^-1 (F_{n+1} - K u_{n+1} - C vh_n)
//   vh_{n+1} = vh_n + dt a_{n+1}
//   u_{n+2}  = u_{n+1} + dt vh_{n+1}
// The adjoint of the time stepping is the same recurrence run backwards, so
// the adjoint launches reuse this kernel with the residual as source
// (Eqs. A12-A15 in discrete form) and add the correlations of Eqs. A16-A18
// (gradient) or of Eqs. 5-8 / A21-A22 (preconditioners).
//
// Work decomposition: a CTA owns a tile of TX x TZ elements and the global
// nodes [4 ex0, 4 (ex0+TX)) x [4 ez0, 4 (ez0+TZ)) (the last tile of a row /
// column also owns the mesh's last node line).  It recomputes the element
// column to the left and the element row above the tile (halo elements), so
// every owned node receives all of its element contributions from this CTA:
// assembly is a fixed-order gather in shared memory, with no atomics and no
// colouring passes, and the result is bitwise reproducible.
//
// One thread computes one element: the 25-point tensor-product derivatives
// with the GLL derivative matrix held in constant memory (uniform operands),
// stress, and the weighted transposed products, all in registers.  Because
// the mesh elements are square, d/dx = (2/h) d/dxi, and the quadrature
// weight is w_i w_j (h/2)^2, the h factors cancel in the element force
// f_a(m,n) = sum_i D[i][m] tau_ax(i,n) + sum_j D[j][n] tau_az(m,j),
// tau = w_i w_j sigma_hat, sigma_hat built from derivatives in xi/eta.

#include "gbfwi_internal.h"

__constant__ float cD[GB_NG * GB_NG];   // D[i*5+k] = l_k'(xi_i)
__constant__ float cW[GB_NG * GB_NG];   // w_i w_j at [j*5+i]

int gb_upload_gll(const double *D, const double *w)
{
    float hD[25], hW[25];
    for (int i = 0; i < 25; ++i) hD[i] = (float)D[i];
    for (int j = 0; j < 5; ++j)
        for (int i = 0; i < 5; ++i) hW[j * 5 + i] = (float)(w[i] * w[j]);
    GB_CUDA(cudaMemcpyToSymbol(cD, hD, sizeof(hD)));
    GB_CUDA(cudaMemcpyToSymbol(cW, hW, sizeof(hW)));
    return GBFWI_OK;
}

namespace {

template <int NWXP>
__device__ __forceinline__ void load_patch(const float2 *__restrict__ win, int base, float (&px)[25],
                                           float (&pz)[25])
{
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            float2 v = win[base + j * NWXP + i];
            px[j * 5 + i] = v.x;
            pz[j * 5 + i] = v.y;
        }
}

// unscaled derivatives at local point (i, j): d/dxi and d/deta of both components
__device__ __forceinline__ void grad_at(const float (&px)[25], const float (&pz)[25], int i, int j,
                                        float &xx, float &xz, float &zx, float &zz)
{
    // xx = d ux/dxi, xz = d ux/deta, zx = d uz/dxi, zz = d uz/deta
    float a = 0.f, b = 0.f, c = 0.f, d = 0.f;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        a = fmaf(cD[i * 5 + k], px[j * 5 + k], a);
        c = fmaf(cD[i * 5 + k], pz[j * 5 + k], c);
        b = fmaf(cD[j * 5 + k], px[k * 5 + i], b);
        d = fmaf(cD[j * 5 + k], pz[k * 5 + i], d);
    }
    xx = a; xz = b; zx = c; zz = d;
}

// element nodal forces (K u restricted to one element) -> out[25]
template <int NWXP>
__device__ __forceinline__ void element_force(const float2 *__restrict__ sw, const float2 *__restrict__ slm,
                                              int base, float2 *__restrict__ out)
{
    float px[25], pz[25];
    load_patch<NWXP>(sw, base, px, pz);
    float txx[25], tzz[25], txz[25];
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            float xx, xz, zx, zz;
            grad_at(px, pz, i, j, xx, xz, zx, zz);
            float2 lm = slm[base + j * NWXP + i];
            float l2m = fmaf(2.f, lm.y, lm.x);
            float ww = cW[j * 5 + i];
            txx[j * 5 + i] = ww * fmaf(l2m, xx, lm.x * zz);
            tzz[j * 5 + i] = ww * fmaf(lm.x, xx, l2m * zz);
            txz[j * 5 + i] = ww * (lm.y * (xz + zx));
        }
#pragma unroll
    for (int n = 0; n < 5; ++n)
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            float fx = 0.f, fz = 0.f;
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                fx = fmaf(cD[i * 5 + m], txx[n * 5 + i], fx);
                fz = fmaf(cD[i * 5 + m], txz[n * 5 + i], fz);
            }
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                fx = fmaf(cD[j * 5 + n], txz[j * 5 + m], fx);
                fz = fmaf(cD[j * 5 + n], tzz[j * 5 + m], fz);
            }
            out[n * 5 + m] = make_float2(fx, fz);
        }
}

// Per local point products of the unscaled strains of two fields A and B,
// weighted by w_i w_j:
//   NC == 2 (gradient):     [div A div B, 2 exx exx' + 2 ezz ezz' + gam gam']
//   NC == 3 (preconditioner): [div A div B, exx exx' + ezz ezz', gam gam']
template <int NWXP, int NC>
__device__ __forceinline__ void element_products(const float2 *__restrict__ wa, const float2 *__restrict__ wb,
                                                 int base, float *__restrict__ out)
{
    float ax[25], az[25], bx[25], bz[25];
    load_patch<NWXP>(wa, base, ax, az);
    load_patch<NWXP>(wb, base, bx, bz);
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            float axx, axz, azx, azz, bxx, bxz, bzx, bzz;
            grad_at(ax, az, i, j, axx, axz, azx, azz);
            grad_at(bx, bz, i, j, bxx, bxz, bzx, bzz);
            float ww = cW[j * 5 + i];
            float da = axx + azz, db = bxx + bzz;
            float ga = axz + azx, gb = bxz + bzx;
            int q = (j * 5 + i) * NC;
            if (NC == 2) {
                out[q + 0] = ww * (da * db);
                out[q + 1] = ww * fmaf(2.f * axx, bxx, fmaf(2.f * azz, bzz, ga * gb));
            } else {
                out[q + 0] = ww * (da * db);
                out[q + 1] = ww * fmaf(axx, bxx, azz * bzz);
                out[q + 2] = ww * (ga * gb);
            }
        }
}

// same as above with A == B (forward preconditioner: squares)
template <int NWXP>
__device__ __forceinline__ void element_squares(const float2 *__restrict__ wa, int base, float *__restrict__ out)
{
    float ax[25], az[25];
    load_patch<NWXP>(wa, base, ax, az);
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            float axx, axz, azx, azz;
            grad_at(ax, az, i, j, axx, axz, azx, azz);
            float ww = cW[j * 5 + i];
            float da = axx + azz, ga = axz + azx;
            int q = (j * 5 + i) * 3;
            out[q + 0] = ww * (da * da);
            out[q + 1] = ww * fmaf(axx, axx, azz * azz);
            out[q + 2] = ww * (ga * ga);
        }
}

// window load: rows iz0.., node pairs from ix0 (even); out-of-mesh -> 0.
// op 0: dst = src;  op 1: dst -= src;  op 2: dst = src - src2
template <int NWZ, int NWXP, int NT>
__device__ __forceinline__ void load_window(float2 *__restrict__ dst, const float2 *__restrict__ src,
                                            const float2 *__restrict__ src2, int op, int ix0, int iz0,
                                            int nz, int pitch)
{
    constexpr int NP = NWXP / 2;
    for (int q = threadIdx.x; q < NWZ * NP; q += NT) {
        int r = q / NP, p = q - r * NP;
        int iz = iz0 + r, ix = ix0 + 2 * p;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        bool in = (iz >= 0) && (iz < nz) && (ix >= 0) && (ix < pitch);
        long long g = (long long)iz * pitch + ix;
        if (in) v = __ldg(reinterpret_cast<const float4 *>(src + g));
        float4 *d = reinterpret_cast<float4 *>(dst + r * NWXP + 2 * p);
        if (op == 0) {
            *d = v;
        } else if (op == 1) {
            float4 o = *d;
            *d = make_float4(o.x - v.x, o.y - v.y, o.z - v.z, o.w - v.w);
        } else {
            float4 v2 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (in) v2 = __ldg(reinterpret_cast<const float4 *>(src2 + g));
            *d = make_float4(v.x - v2.x, v.y - v2.y, v.z - v2.z, v.w - v2.w);
        }
    }
}

}  // namespace

template <int TX, int TZ, int MODE>
__global__ void __launch_bounds__((TX + 1) * (TZ + 1), 1) sem_step_kernel(const StepArgs a)
{
    constexpr int NE = (TX + 1) * (TZ + 1);
    constexpr int NT = NE;
    constexpr int NWZ = 4 * TZ + 5, NWXP = 4 * TX + 6;
    constexpr int OX = 4 * TX + 1, OZ = 4 * TZ + 1;
    constexpr int NC = (MODE == MODE_ADJ_G) ? 2 : ((MODE == MODE_FWD) ? 2 : 3);

    extern __shared__ float4 smem4[];
    float2 *sw = reinterpret_cast<float2 *>(smem4);      // field window [NWZ][NWXP]
    float2 *slm = sw + NWZ * NWXP;                         // (lambda, mu) window; later 2nd field
    float *sfl = reinterpret_cast<float *>(slm + NWZ * NWXP);   // element results [NE][25][NC]
    float2 *sF = reinterpret_cast<float2 *>(sfl + NE * 25 * NC); // source forces [OZ][OX]

    const int b = blockIdx.z;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    const int ex0 = blockIdx.x * TX, ez0 = blockIdx.y * TZ;
    const int ix0 = 4 * ex0 - 4, iz0 = 4 * ez0 - 4;
    const int pitch = a.pitch;
    const long long fo = (long long)b * a.fstride;   // shots of a field are fstride apart

    // owned node box
    const int ixe = (ex0 + TX >= a.nex) ? a.nx : 4 * (ex0 + TX);
    const int ize = (ez0 + TZ >= a.nez) ? a.nz : 4 * (ez0 + TZ);
    const int ow = ixe - 4 * ex0, oh = ize - 4 * ez0;

    // ---- phase 0: windows, zero source forces
    for (int q = threadIdx.x; q < OX * OZ; q += NT) sF[q] = make_float2(0.f, 0.f);
    load_window<NWZ, NWXP, NT>(sw, a.ucur + fo, nullptr, 0, ix0, iz0, a.nz, pitch);
    load_window<NWZ, NWXP, NT>(slm, a.lm, nullptr, 0, ix0, iz0, a.nz, pitch);
    __syncthreads();

    // ---- phase 1: records, element forces, source forces
    if (MODE == MODE_FWD || MODE == MODE_FWD_PC) {
        if (a.seis) {
            int rb = a.rec_tptr[tile], re = a.rec_tptr[tile + 1];
            for (int t = threadIdx.x; t < 2 * (re - rb); t += NT) {
                int r = a.rec_list[rb + (t >> 1)], c = t & 1;
                int2 e = a.rec_e[r];
                int base = (4 * (e.y - ez0 + 1)) * NWXP + 4 * (e.x - ex0 + 1);
                const float *w = a.recw + r * 25;
                float s = 0.f;
#pragma unroll
                for (int j = 0; j < 5; ++j)
#pragma unroll
                    for (int i = 0; i < 5; ++i) {
                        float2 v = sw[base + j * NWXP + i];
                        s = fmaf(w[j * 5 + i], c ? v.y : v.x, s);
                    }
                a.seis[(long long)b * a.seis_shot_stride + (long long)(r * 2 + c) * a.nt + a.trec] = s;
            }
        }
    }
    {
        int e = threadIdx.x;          // one element per thread
        int elx = e % (TX + 1), elz = e / (TX + 1);
        int ex = ex0 - 1 + elx, ez = ez0 - 1 + elz;
        if (ex >= 0 && ez >= 0 && ex < a.nex && ez < a.nez) {
            int base = 4 * elz * NWXP + 4 * elx;
            element_force<NWXP>(sw, slm, base, reinterpret_cast<float2 *>(sfl) + e * 25);
        }
    }
    {
        const int src_id = a.shot_map ? a.shot_map[b] : b;
        const int *gp = a.gptr + (a.per_shot_groups ? (long long)src_id * (a.ntiles + 1) : 0);
        int gb = gp[tile], ge = gp[tile + 1];
        const float *sig = a.sig + (long long)src_id * a.sig_shot_stride + a.tsig;
        for (int g = gb + threadIdx.x; g < ge; g += NT) {
            InjGroup G = a.groups[g];
            float fx = 0.f, fz = 0.f;
            for (int q = G.begin; q < G.end; ++q) {
                InjEntry E = a.entries[q];
                fx = fmaf(E.wx, sig[(long long)E.cx * a.sig_chan_stride], fx);
                fz = fmaf(E.wz, sig[(long long)E.cz * a.sig_chan_stride], fz);
            }
            sF[G.node] = make_float2(fx * a.sig_scale, fz * a.sig_scale);
        }
    }
    __syncthreads();

    // ---- phase 2: gather K u, Newmark update, pointwise accumulations
    const float dt = a.dt;
    const float2 *sf2 = reinterpret_cast<const float2 *>(sfl);
    for (int q = threadIdx.x; q < ow * oh; q += NT) {
        int oz = q / ow, ox = q - oz * ow;
        int ix = 4 * ex0 + ox, iz = 4 * ez0 + oz;
        int wxi = ox + 4, wzi = oz + 4;
        int elx1 = wxi >> 2, li1 = wxi & 3;
        int elz1 = wzi >> 2, lj1 = wzi & 3;
        float kx = 0.f, kz = 0.f;
#pragma unroll
        for (int cz = 0; cz < 2; ++cz) {
            int elz = cz == 0 ? elz1 - 1 : elz1, lj = cz == 0 ? 4 : lj1;
            if (cz == 0 && lj1 != 0) continue;
            int ez = ez0 - 1 + elz;
            if (ez < 0 || ez >= a.nez) continue;
#pragma unroll
            for (int cx = 0; cx < 2; ++cx) {
                int elx = cx == 0 ? elx1 - 1 : elx1, li = cx == 0 ? 4 : li1;
                if (cx == 0 && li1 != 0) continue;
                int ex = ex0 - 1 + elx;
                if (ex < 0 || ex >= a.nex) continue;
                float2 f = sf2[(elz * (TX + 1) + elx) * 25 + lj * 5 + li];
                kx += f.x;
                kz += f.y;
            }
        }
        float2 F = sF[oz * OX + ox];
        long long g = (long long)iz * pitch + ix;
        float2 v = a.vh[fo + g];
        bool edge = (ix == 0) | (ix == a.nx - 1) | (iz == 0) | (iz == a.nz - 1);
        float ax, az;
        if (edge) {
            float4 bd = a.bnd[g];
            ax = (F.x - kx - bd.x * v.x) * bd.z;
            az = (F.y - kz - bd.y * v.y) * bd.w;
        } else {
            float mi = a.minv[g];
            ax = (F.x - kx) * mi;
            az = (F.y - kz) * mi;
        }
        float2 vn = make_float2(fmaf(dt, ax, v.x), fmaf(dt, az, v.y));
        float2 uc = sw[wzi * NWXP + wxi];
        a.vh[fo + g] = vn;
        a.unext[fo + g] = make_float2(fmaf(dt, vn.x, uc.x), fmaf(dt, vn.y, uc.y));

        if (MODE == MODE_FWD_PC) {
            float *acc = a.acc + (long long)b * a.acc_shot_stride + g;
            acc[0] += fmaf(ax, ax, az * az);
        } else if (MODE == MODE_ADJ_G) {
            const long long ho = (long long)b * a.hstride;
            float2 uk = a.h0[ho + g];
            float *acc = a.acc + (long long)b * a.acc_shot_stride + g;
            const long long cs = a.acc_comp_stride;
            float wsum = a.wxs[ix] * a.wzs[iz];
            acc[2 * cs] += wsum * fmaf(uk.x, ax, uk.y * az);
            if (edge) {
                float4 w4 = a.bw[g];
                float vx = 0.5f * (v.x + vn.x), vz = 0.5f * (v.y + vn.y);
                acc[3 * cs] += fmaf(w4.x * uk.x, vx, w4.y * uk.y * vz);
                acc[4 * cs] += fmaf(w4.z * uk.x, vx, w4.w * uk.y * vz);
            }
        } else if (MODE == MODE_ADJ_PC) {
            const long long ho = (long long)b * a.hstride;
            float2 p0 = a.h0[ho + g], p1 = a.h1[ho + g], p2 = a.h2[ho + g];
            float fxa = (p0.x - p1.x) - (p1.x - p2.x);
            float fza = (p0.y - p1.y) - (p1.y - p2.y);
            float *acc = a.acc + (long long)b * a.acc_shot_stride + g;
            acc[0] += fmaf(fxa, ax, fza * az);
        }
    }
    if (MODE == MODE_FWD) return;
    __syncthreads();

    // ---- phase 3: second windows
    if (MODE == MODE_FWD_PC) {
        // sw <- u_{n+1} - u_n
        load_window<NWZ, NWXP, NT>(sw, a.uold + fo, nullptr, 1, ix0, iz0, a.nz, pitch);
    } else if (MODE == MODE_ADJ_G) {
        const long long ho = (long long)b * a.hstride;
        load_window<NWZ, NWXP, NT>(slm, a.h0 + ho, nullptr, 0, ix0, iz0, a.nz, pitch);
    } else {
        const long long ho = (long long)b * a.hstride;
        load_window<NWZ, NWXP, NT>(slm, a.h0 + ho, a.h1 + ho, 2, ix0, iz0, a.nz, pitch);
        load_window<NWZ, NWXP, NT>(sw, a.uold + fo, nullptr, 1, ix0, iz0, a.nz, pitch);
    }
    __syncthreads();

    // ---- phase 4: element products
    {
        int e = threadIdx.x;
        int elx = e % (TX + 1), elz = e / (TX + 1);
        int ex = ex0 - 1 + elx, ez = ez0 - 1 + elz;
        if (ex >= 0 && ez >= 0 && ex < a.nex && ez < a.nez) {
            int base = 4 * elz * NWXP + 4 * elx;
            if (MODE == MODE_FWD_PC)
                element_squares<NWXP>(sw, base, sfl + e * 25 * NC);
            else
                element_products<NWXP, NC>(sw, slm, base, sfl + e * 25 * NC);
        }
    }
    __syncthreads();

    // ---- phase 5: gather products into the accumulators
    const int c0 = (MODE == MODE_ADJ_G) ? 0 : 1;
    for (int q = threadIdx.x; q < ow * oh; q += NT) {
        int oz = q / ow, ox = q - oz * ow;
        int ix = 4 * ex0 + ox, iz = 4 * ez0 + oz;
        int wxi = ox + 4, wzi = oz + 4;
        int elx1 = wxi >> 2, li1 = wxi & 3;
        int elz1 = wzi >> 2, lj1 = wzi & 3;
        float s[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) s[c] = 0.f;
#pragma unroll
        for (int cz = 0; cz < 2; ++cz) {
            int elz = cz == 0 ? elz1 - 1 : elz1, lj = cz == 0 ? 4 : lj1;
            if (cz == 0 && lj1 != 0) continue;
            int ez = ez0 - 1 + elz;
            if (ez < 0 || ez >= a.nez) continue;
#pragma unroll
            for (int cx = 0; cx < 2; ++cx) {
                int elx = cx == 0 ? elx1 - 1 : elx1, li = cx == 0 ? 4 : li1;
                if (cx == 0 && li1 != 0) continue;
                int ex = ex0 - 1 + elx;
                if (ex < 0 || ex >= a.nex) continue;
                const float *p = sfl + ((elz * (TX + 1) + elx) * 25 + lj * 5 + li) * NC;
#pragma unroll
                for (int c = 0; c < NC; ++c) s[c] += p[c];
            }
        }
        long long g = (long long)iz * pitch + ix;
        float *acc = a.acc + (long long)b * a.acc_shot_stride + g;
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[(c0 + c) * a.acc_comp_stride] += s[c];
    }
}

// ---------------------------------------------------------------------------

template <int TX, int TZ>
static size_t step_smem(int mode)
{
    constexpr int NE = (TX + 1) * (TZ + 1);
    constexpr int NWZ = 4 * TZ + 5, NWXP = 4 * TX + 6;
    constexpr int OX = 4 * TX + 1, OZ = 4 * TZ + 1;
    int NC = (mode == MODE_FWD || mode == MODE_ADJ_G) ? 2 : 3;
    return (size_t)2 * NWZ * NWXP * sizeof(float2) + (size_t)NE * 25 * NC * sizeof(float) +
           (size_t)OX * OZ * sizeof(float2);
}

template <int TX, int TZ, int MODE>
static int launch_one(const StepArgs &a, int nbatch, cudaStream_t s)
{
    constexpr int NE = (TX + 1) * (TZ + 1);
    size_t smem = step_smem<TX, TZ>(MODE);
    static bool attr_done[64] = {};          // per device ordinal
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_done[dev]) {
        GB_CUDA(cudaFuncSetAttribute(sem_step_kernel<TX, TZ, MODE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_done[dev] = true;
    }
    dim3 grid((a.nex + TX - 1) / TX, (a.nez + TZ - 1) / TZ, nbatch);
    sem_step_kernel<TX, TZ, MODE><<<grid, NE, smem, s>>>(a);
    GB_CUDA(cudaGetLastError());
    return GBFWI_OK;
}

template <int TX, int TZ>
static int launch_mode(int mode, const StepArgs &a, int nbatch, cudaStream_t s)
{
    switch (mode) {
    case MODE_FWD: return launch_one<TX, TZ, MODE_FWD>(a, nbatch, s);
    case MODE_FWD_PC: return launch_one<TX, TZ, MODE_FWD_PC>(a, nbatch, s);
    case MODE_ADJ_G: return launch_one<TX, TZ, MODE_ADJ_G>(a, nbatch, s);
    case MODE_ADJ_PC: return launch_one<TX, TZ, MODE_ADJ_PC>(a, nbatch, s);
    }
    return GBFWI_EINVAL;
}

const TileShape kTiles[kNumTiles] = {{15, 7}, {7, 15}, {7, 7}, {15, 15}, {31, 3}};

int gb_launch_step(int mode, int tile, const StepArgs &a, int nbatch, cudaStream_t s)
{
    switch (tile) {
    case 0: return launch_mode<15, 7>(mode, a, nbatch, s);
    case 1: return launch_mode<7, 15>(mode, a, nbatch, s);
    case 2: return launch_mode<7, 7>(mode, a, nbatch, s);
    case 3: return launch_mode<15, 15>(mode, a, nbatch, s);
    case 4: return launch_mode<31, 3>(mode, a, nbatch, s);
    }
    return GBFWI_EINVAL;
}
