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
// no atomics, a fixed summation order, bitwise reproducible results.
//
// One thread computes one element: the 25-point tensor-product derivatives
// with the GLL derivative matrix held in constant memory (uniform operands),
// stress, and the weighted transposed products, all in registers.  Because
// the mesh elements are square, d/dx = (2/h) d/dxi, and the quadrature
// weight is w_i w_j (h/2)^2, the h factors cancel in the element force
// f_a(m,n) = sum_i D[i][m] tau_ax(i,n) + sum_j D[j][n] tau_az(m,j),
// tau = w_i w_j sigma_hat, sigma_hat built from derivatives in xi/eta.
//
// Assembly: in the forward and adjoint-gradient steps every element owns 16
// nodes of its patch and receives its neighbours' shares by warp shuffles
// (x) and one shared-memory exchange (z), then updates its own nodes
// (sem_step_kernel); the preconditioner steps sum into a shared node array
// in four colour passes (sem_pc_step_kernel).

#include "gbfwi_internal.h"
#include "sm100.h"

using sm100::bulk_g2s;
using sm100::mbar_arrive_expect_tx;
using sm100::mbar_init;
using sm100::mbar_wait_bounded;

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

// Per local point products of the unscaled strains of two fields A and B,
// weighted by w_i w_j:
//   NC == 2 (gradient):     [div A div B, 2 exx exx' + 2 ezz ezz' + gam gam']
//   NC == 3 (preconditioner): [div A div B, exx exx' + ezz ezz', gam gam']
template <int NWXP, int NC>
__device__ __forceinline__ void element_products(const float2 *__restrict__ wa, const float2 *__restrict__ wb,
                                                 int base, float (&out)[25 * NC])
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
__device__ __forceinline__ void element_squares(const float2 *__restrict__ wa, int base, float (&out)[75])
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

// Element nodal forces accumulated row by row of local points: the
// stresses of row j give the xi-part of the nodes of row j and the eta-part
// of every node, so one row of stresses is live at a time.
template <int NWXP>
__device__ __forceinline__ void element_force_rows(const float2 *__restrict__ sw, const float2 *__restrict__ slm,
                                                   int base, float2 (&f)[25])
{
    float px[25], pz[25];
    load_patch<NWXP>(sw, base, px, pz);
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        float txx[5], tzz[5], txz[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            float xx, xz, zx, zz;
            grad_at(px, pz, i, j, xx, xz, zx, zz);
            float2 lm = slm[base + j * NWXP + i];
            float l2m = fmaf(2.f, lm.y, lm.x);
            float ww = cW[j * 5 + i];
            txx[i] = ww * fmaf(l2m, xx, lm.x * zz);
            tzz[i] = ww * fmaf(lm.x, xx, l2m * zz);
            txz[i] = ww * (lm.y * (xz + zx));
        }
        // f(m, n) += D[j][n] (txz, tzz)(m, j) for every node; for n == j also
        // the xi-part sum_i D[i][m] (txx, txz)(i, j)
#pragma unroll
        for (int n = 0; n < 5; ++n)
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                float fx, fz;
                if (j == 0) {
                    fx = cD[n] * txz[m];
                    fz = cD[n] * tzz[m];
                } else {
                    fx = fmaf(cD[j * 5 + n], txz[m], f[n * 5 + m].x);
                    fz = fmaf(cD[j * 5 + n], tzz[m], f[n * 5 + m].y);
                }
                if (n == j) {
#pragma unroll
                    for (int i = 0; i < 5; ++i) {
                        fx = fmaf(cD[i * 5 + m], txx[i], fx);
                        fz = fmaf(cD[i * 5 + m], txz[i], fz);
                    }
                }
                f[n * 5 + m] = make_float2(fx, fz);
            }
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

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (16 B, zero-filled beyond src_bytes)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

// window of a float2 node field: rows iz0.., node pairs from ix0 (even)
template <int NWZ, int NWXP, int NT>
__device__ __forceinline__ void prefetch_window(float2 *dst, const float2 *src, int ix0, int iz0, int nz, int pitch)
{
    constexpr int NP = NWXP / 2;
    for (int q = threadIdx.x; q < NWZ * NP; q += NT) {
        int r = q / NP, p = q - r * NP;
        int iz = iz0 + r, ix = ix0 + 2 * p;
        bool in = (iz >= 0) && (iz < nz) && (ix >= 0) && (ix < pitch);
        const float2 *g = in ? src + (long long)iz * pitch + ix : src;
        cp_async16(dst + r * NWXP + 2 * p, g, in ? 16 : 0);
    }
}

// owned box of a float2 field: oh rows of ow nodes from (ixo, izo); smem row pitch OXP (even)
template <int OXP, int NT>
__device__ __forceinline__ void prefetch_owned2(float2 *dst, const float2 *src, int ixo, int izo, int ow, int oh,
                                                int pitch)
{
    const int np = (ow + 1) >> 1;
    for (int q = threadIdx.x; q < oh * np; q += NT) {
        int r = q / np, p = q - r * np;
        cp_async16(dst + r * OXP + 2 * p, src + (long long)(izo + r) * pitch + ixo + 2 * p, 16);
    }
}

// owned box of a float field; smem row pitch OXQ (multiple of 4)
template <int OXQ, int NT>
__device__ __forceinline__ void prefetch_owned1(float *dst, const float *src, int ixo, int izo, int ow, int oh,
                                                int pitch)
{
    const int nq = (ow + 3) >> 2;
    for (int q = threadIdx.x; q < oh * nq; q += NT) {
        int r = q / nq, p = q - r * nq;
        int ix = ixo + 4 * p;
        int bytes = max(0, min(16, (pitch - ix) * 4));
        cp_async16(dst + r * OXQ + 4 * p, src + (long long)(izo + r) * pitch + ix, bytes);
    }
}

// ---------------------------------------------------------------------------
// Forward and adjoint-gradient steps (MODE_FWD, MODE_ADJ_G): owner-computes assembly
// ---------------------------------------------------------------------------
// Each element owns the 16 nodes (i, j) in [0,4) x [0,4) of its patch (the
// last element of a mesh row / column also owns its i = 4 column / j = 4
// row), so the tile's owned nodes are partitioned among the element
// threads.  Assembly of the element vectors is then two exchanges instead
// of colour passes over a node-sum array:
//   x: the i = 4 column of every element goes to its right neighbour, the
//      next lane of the same warp (a warp holds whole rows of the extended
//      tile), by register shuffles;
//   z: the j = 4 row (after the x-step) goes to the element below through a
//      small shared buffer, after one barrier.
// Node (0, 0) of element (ex, ez) thus sums
//   [v(ex,ez) + v(ex-1,ez)(4,.)] + [v(ex,ez-1)(.,4) + v(ex-1,ez-1)(4,4)]
// in this order for every tile shape, so results are bitwise the same
// across tile shapes, batching and checkpointing.  The element thread then
// runs the Newmark update (and the correlation sums) of its own nodes, with
// 16-byte global accesses along node rows.

template <int TX, int TZ, int MODE>
struct StepShape {
    static_assert(MODE == MODE_FWD || MODE == MODE_ADJ_G, "forward and adjoint-gradient modes");
    static constexpr int NT = (TX + 1) * (TZ + 1);
    static constexpr int NWZ = 4 * TZ + 5, NWXP = 4 * TX + 6;
    static constexpr int WIN = NWZ * NWXP;
    static constexpr int OX = 4 * TX + 1, OZ = 4 * TZ + 1;
    static constexpr int OXP = 4 * TX + 2;                     // float2 row pitch of the source-force box
    static constexpr int NWIN = (MODE == MODE_ADJ_G) ? 3 : 2;   // field, (lambda, mu) / source forces, history
    static constexpr int NZB = (MODE == MODE_ADJ_G) ? 2 : 1;    // z-exchange buffers (force, correlation)
    static constexpr size_t ZB = (size_t)NT * 5 * sizeof(float2);
    static_assert((size_t)OZ * OXP <= (size_t)WIN, "source-force box fits the (lambda, mu) window");
    // half-step velocity of the standard owned nodes (4 TX x 4 TZ), staged in phase 0
    static constexpr int VXP = 4 * TX;
    static constexpr size_t VB = (size_t)4 * TZ * VXP * sizeof(float2);
    static constexpr int NCOPY = NWIN * NWZ + 4 * TZ;           // bulk row copies of phase 0
    static constexpr int MINB = ((MODE == MODE_FWD ? 512 : 384) / NT) > 0 ? (MODE == MODE_FWD ? 512 : 384) / NT : 1;
    static constexpr size_t bytes = (size_t)NWIN * WIN * sizeof(float2) + NZB * ZB + VB;
};

// x-step of the assembly: v(0, j) += left neighbour's v(4, j) (lane - 1)
__device__ __forceinline__ void assemble_x(float2 (&v)[25], bool has_left)
{
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const float rx = __shfl_up_sync(0xffffffffu, v[j * 5 + 4].x, 1);
        const float rz = __shfl_up_sync(0xffffffffu, v[j * 5 + 4].y, 1);
        if (has_left) {
            v[j * 5].x += rx;
            v[j * 5].y += rz;
        }
    }
}

template <int TX, int TZ, int MODE>
__global__ void __launch_bounds__(StepShape<TX, TZ, MODE>::NT, StepShape<TX, TZ, MODE>::MINB)
    sem_step_kernel(const StepArgs a)
{
    using S = StepShape<TX, TZ, MODE>;
    constexpr int NT = S::NT, NWXP = S::NWXP, NWZ = S::NWZ, WIN = S::WIN, OXP = S::OXP;

    extern __shared__ float4 smem4[];
    float2 *sw = reinterpret_cast<float2 *>(smem4);     // field window (u_{n+1} or w_{j+1})
    float2 *slm = sw + WIN;                              // (lambda, mu) window
    float2 *sF = slm;                                    // source forces of the owned box, after the forces
    float2 *su2 = slm + WIN;                             // forward-history window (MODE_ADJ_G)
    float2 *zb0 = sw + S::NWIN * WIN;                    // z-exchange of the forces [NT][5]
    float2 *zb1 = zb0 + NT * 5;                          // z-exchange of the correlation (MODE_ADJ_G)
    float2 *svh = zb0 + S::NZB * NT * 5;                 // [4 TZ][4 TX] owned half-step velocity
    __shared__ unsigned long long s_mbar;

    const int b = blockIdx.z;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    const int ex0 = blockIdx.x * TX, ez0 = blockIdx.y * TZ;
    const int ix0 = 4 * ex0 - 4, iz0 = 4 * ez0 - 4;
    const int pitch = a.pitch;
    const long long fo = (long long)b * a.fstride;

    const int ixo = 4 * ex0, izo = 4 * ez0;              // owned box origin
    // source injections of this tile (read ahead of their use)
    const int src_id = a.shot_map ? a.shot_map[b] : b;
    const int *gp = a.gptr + (a.per_shot_groups ? (long long)src_id * (a.ntiles + 1) : 0);
    const int gb = gp[tile], ge = gp[tile + 1];

    // ---- phase 0: bulk copies of the windows (rows inside the mesh; the rest
    // is never read) and of the owned velocity box, one row per copy
    {
        const int r_lo = max(0, -iz0), r_hi = min(NWZ, a.nz - iz0);
        const int cx0 = max(ix0, 0), cx1 = min(ix0 + NWXP, pitch);
        const unsigned wbytes = (unsigned)(cx1 - cx0) * (unsigned)sizeof(float2);
        const int vrows = min(4 * TZ, a.nz - izo);
        const unsigned vbytes = (unsigned)(min(ixo + S::VXP, pitch) - ixo) * (unsigned)sizeof(float2);
        if (threadIdx.x == 0) {
            mbar_init(&s_mbar, 1);
            mbar_arrive_expect_tx(&s_mbar, (unsigned)S::NWIN * (unsigned)(r_hi - r_lo) * wbytes +
                                               (unsigned)vrows * vbytes);
        }
        __syncthreads();
        for (int c = threadIdx.x; c < S::NCOPY; c += NT) {
            if (c < S::NWIN * NWZ) {
                const int w = c / NWZ, r = c - w * NWZ;
                const float2 *src = w == 0 ? a.ucur + fo : (w == 1 ? a.lm : a.h0 + (long long)b * a.hstride);
                float2 *dst = w == 0 ? sw : (w == 1 ? slm : su2);
                if (r >= r_lo && r < r_hi)
                    bulk_g2s(dst + r * NWXP + (cx0 - ix0), src + (long long)(iz0 + r) * pitch + cx0, wbytes, &s_mbar);
            } else {
                const int r = c - S::NWIN * NWZ;
                if (r < vrows)
                    bulk_g2s(svh + r * S::VXP, a.vh + fo + (long long)(izo + r) * pitch + ixo, vbytes, &s_mbar);
            }
        }
        const bool ok = mbar_wait_bounded(&s_mbar, 0);
        if (__syncthreads_or(!ok)) {
            // the copies did not complete within the bound: flag it, give the
            // ones in flight another bounded wait, and leave
            if (threadIdx.x == 0 && a.status) atomicExch(a.status, 1);
            mbar_wait_bounded(&s_mbar, 0);
            return;
        }
    }

    // ---- phase 1: records, element forces
    if (MODE == MODE_FWD && a.seis) {
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
    constexpr int R = 32 / (TX + 1);
    static_assert(R >= 1 && 32 % (TX + 1) == 0 && (TZ + 1) % (2 * R) == 0, "parity-grouped element rows");
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int elx = lane % (TX + 1);
    const int elz = (wid >> 1) * 2 * R + (wid & 1) + 2 * (lane / (TX + 1));
    const int ex = ex0 - 1 + elx, ez = ez0 - 1 + elz;
    const bool evalid = (ex >= 0) && (ez >= 0) && (ex < a.nex) && (ez < a.nez);
    const bool owns = evalid && elx >= 1 && elz >= 1;    // halo elements own no node of this tile
    const int ni = (ex == a.nex - 1) ? 5 : 4, nj = (ez == a.nez - 1) ? 5 : 4;
    const int ebase = 4 * elz * NWXP + 4 * elx;
    const int eslot = elz * (TX + 1) + elx;
    // element below in z (elz - 1) in the same extended-tile column
    const int bslot = eslot - (TX + 1);

    // owned-node data of the 16 standard nodes (i, j < 4) read from global
    // memory ahead of their use, 16 bytes at a time along node rows (the
    // extra column / row of the last element is read where it is used)
    float2 *vhb = a.vh + fo;
    float *accb = a.acc + (long long)b * a.acc_shot_stride;
    const long long cs = a.acc_comp_stride;
    const long long g00 = (long long)(4 * ez) * pitch + 4 * ex;   // node (0, 0) of the element
    float mip[16], amp[16];
    float2 f[25];
    if (evalid) {
        element_force_rows<NWXP>(sw, slm, ebase, f);
    } else {
#pragma unroll
        for (int q = 0; q < 25; ++q) f[q] = make_float2(0.f, 0.f);
    }
    if (owns) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long g = g00 + (long long)j * pitch;
            const float4 m4 = *reinterpret_cast<const float4 *>(a.minv + g);
            mip[4 * j + 0] = m4.x; mip[4 * j + 1] = m4.y; mip[4 * j + 2] = m4.z; mip[4 * j + 3] = m4.w;
            if (MODE == MODE_ADJ_G) {
                const float4 c4 = *reinterpret_cast<const float4 *>(accb + 2 * cs + g);
                amp[4 * j + 0] = c4.x; amp[4 * j + 1] = c4.y; amp[4 * j + 2] = c4.z; amp[4 * j + 3] = c4.w;
            }
        }
    }
    assemble_x(f, elx >= 1);
#pragma unroll
    for (int i = 0; i < 5; ++i) zb0[eslot * 5 + i] = f[20 + i];
    __syncthreads();                                     // windows read, z-row published

    // ---- sources (tiles with injections only): forces of the owned box
    if (ge > gb) {
        for (int q = threadIdx.x; q < S::OZ * OXP; q += NT) sF[q] = make_float2(0.f, 0.f);
        __syncthreads();
        const float *sig = a.sig + (long long)src_id * a.sig_shot_stride + a.tsig;
        for (int g = gb + threadIdx.x; g < ge; g += NT) {
            InjGroup G = a.groups[g];
            float fx = 0.f, fz = 0.f;
            for (int q = G.begin; q < G.end; ++q) {
                InjEntry E = a.entries[q];
                fx = fmaf(E.wx, sig[(long long)E.cx * a.sig_chan_stride], fx);
                fz = fmaf(E.wz, sig[(long long)E.cz * a.sig_chan_stride], fz);
            }
            int oz = G.node / S::OX, ox = G.node - oz * S::OX;
            sF[oz * OXP + ox] = make_float2(-fx * a.sig_scale, -fz * a.sig_scale);
        }
        __syncthreads();
    }

    // ---- phase 2: z-step of the forces, Newmark update of the owned nodes
    if (elz >= 1) {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float2 r = zb0[bslot * 5 + i];
            f[i].x += r.x;
            f[i].y += r.y;
        }
    }
    const float dt = a.dt;
    if (owns) {
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            float2 vrow[5];                              // new half-step velocity and displacement of the row
            float2 urow[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                if (!(i < ni && j < nj)) continue;
                const bool std16 = (i < 4) && (j < 4);
                const int q = j * 5 + i;
                const int ix = 4 * ex + i, iz = 4 * ez + j;
                const long long g = g00 + (long long)j * pitch + i;
                float2 k = f[q];
                if (ge > gb) {
                    const float2 F = sF[(4 * (elz - 1) + j) * OXP + 4 * (elx - 1) + i];
                    k.x += F.x;
                    k.y += F.y;
                }
                const float2 v = std16 ? svh[(4 * (elz - 1) + j) * S::VXP + 4 * (elx - 1) + i] : vhb[g];
                const bool edge = (ix == 0) | (ix == a.nx - 1) | (iz == 0) | (iz == a.nz - 1);
                float ax, az;
                if (edge) {
                    float4 bd = a.bnd[g];
                    ax = -(k.x + bd.x * v.x) * bd.z;
                    az = -(k.y + bd.y * v.y) * bd.w;
                } else {
                    const float mi = std16 ? mip[4 * j + i] : a.minv[g];
                    ax = -k.x * mi;
                    az = -k.y * mi;
                }
                const float2 vn = make_float2(fmaf(dt, ax, v.x), fmaf(dt, az, v.y));
                const float2 uc = sw[ebase + j * NWXP + i];
                vrow[i] = vn;
                urow[i] = make_float2(fmaf(dt, vn.x, uc.x), fmaf(dt, vn.y, uc.y));
                if (!std16) {
                    vhb[g] = vrow[i];
                    a.unext[fo + g] = urow[i];
                }
                if (MODE == MODE_ADJ_G) {
                    const float2 uk = su2[ebase + j * NWXP + i];
                    // u_k . a^w; the node's mass factor rho W_g enters once, in the chain rule
                    const float am = std16 ? amp[4 * j + i] : accb[2 * cs + g];
                    accb[2 * cs + g] = am + fmaf(uk.x, ax, uk.y * az);
                    if (edge) {
                        float4 w4 = a.bw[g];
                        float vx = 0.5f * (v.x + vn.x), vz = 0.5f * (v.y + vn.y);
                        accb[3 * cs + g] += fmaf(w4.x * uk.x, vx, w4.y * uk.y * vz);
                        accb[4 * cs + g] += fmaf(w4.z * uk.x, vx, w4.w * uk.y * vz);
                    }
                }
            }
            if (j < 4) {
                const long long g = g00 + (long long)j * pitch;
                *reinterpret_cast<float4 *>(vhb + g) = make_float4(vrow[0].x, vrow[0].y, vrow[1].x, vrow[1].y);
                *reinterpret_cast<float4 *>(vhb + g + 2) = make_float4(vrow[2].x, vrow[2].y, vrow[3].x, vrow[3].y);
                float2 *un = a.unext + fo + g;
                *reinterpret_cast<float4 *>(un) = make_float4(urow[0].x, urow[0].y, urow[1].x, urow[1].y);
                *reinterpret_cast<float4 *>(un + 2) = make_float4(urow[2].x, urow[2].y, urow[3].x, urow[3].y);
            }
        }
    }
    if constexpr (MODE == MODE_FWD) return;

    // ---- phase 3: element strain products, assembled like the forces
    {
        float pr[50];
        if (evalid) {
            element_products<NWXP, 2>(sw, su2, ebase, pr);
        } else {
#pragma unroll
            for (int q = 0; q < 50; ++q) pr[q] = 0.f;
        }
        float2 c[25];
#pragma unroll
        for (int q = 0; q < 25; ++q) c[q] = make_float2(pr[2 * q], pr[2 * q + 1]);
        // strain accumulators of the 16 standard nodes, read ahead of the exchange
        float4 a0p[4], a1p[4];
        if (owns) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long g = g00 + (long long)j * pitch;
                a0p[j] = *reinterpret_cast<const float4 *>(accb + g);
                a1p[j] = *reinterpret_cast<const float4 *>(accb + cs + g);
            }
        }
        assemble_x(c, elx >= 1);
#pragma unroll
        for (int i = 0; i < 5; ++i) zb1[eslot * 5 + i] = c[20 + i];
        __syncthreads();
        if (elz >= 1) {
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                const float2 r = zb1[bslot * 5 + i];
                c[i].x += r.x;
                c[i].y += r.y;
            }
        }
        if (owns) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long g = g00 + (long long)j * pitch;
                const float2 *cr = c + j * 5;
                *reinterpret_cast<float4 *>(accb + g) =
                    make_float4(a0p[j].x + cr[0].x, a0p[j].y + cr[1].x, a0p[j].z + cr[2].x, a0p[j].w + cr[3].x);
                *reinterpret_cast<float4 *>(accb + cs + g) =
                    make_float4(a1p[j].x + cr[0].y, a1p[j].y + cr[1].y, a1p[j].z + cr[2].y, a1p[j].w + cr[3].y);
            }
            // the extra column / row of the last element of a mesh row / column
#pragma unroll
            for (int j = 0; j < 5; ++j)
#pragma unroll
                for (int i = 0; i < 5; ++i)
                    if ((i == 4 || j == 4) && i < ni && j < nj) {
                        const long long g = g00 + (long long)j * pitch + i;
                        accb[g] += c[j * 5 + i].x;
                        accb[cs + g] += c[j * 5 + i].y;
                    }
        }
    }
}

// ---------------------------------------------------------------------------
// Preconditioner steps (MODE_FWD_PC, MODE_ADJ_PC; iteration 0 only)
// ---------------------------------------------------------------------------
// The forward step with the P1/P3 time integrals (Eqs. 5 and 7, A21) and
// the receiver-field step with the P2/P4 integrals (Eqs. 6 and 8, A22).
// Node sums are gathered in a shared node array over the window, the
// element contributions added in four passes by global element parity
// (4-colouring): deterministic and identical for every tile shape.

template <int TX, int TZ, int MODE>
struct PcShape {
    static_assert(MODE == MODE_FWD_PC || MODE == MODE_ADJ_PC, "preconditioner modes");
    static constexpr int NT = (TX + 1) * (TZ + 1);          // one thread per element of the extended tile
    static constexpr int NWZ = 4 * TZ + 5, NWXP = 4 * TX + 6;
    static constexpr int WIN = NWZ * NWXP;                    // float2 per window
    static constexpr int OX = 4 * TX + 1, OZ = 4 * TZ + 1;   // largest owned box
    static constexpr int OXP = 4 * TX + 2;                    // float2 row pitch of owned boxes
    static constexpr int OXQ = 4 * TX + 4;                    // float row pitch of owned boxes
    static constexpr int CW = OX <= 32 ? 32 : (OX <= 64 ? 64 : 128);   // owned-node columns per pass
    static constexpr int RPP = NT / CW;                       // owned-node rows per pass
    static constexpr int NWIN = 3;                            // field, (lambda, mu) / 2nd field, node sums
    static constexpr int WIN4 = (WIN + 3) / 4 * 4;            // 3rd node-sum plane (floats)
    static constexpr int MINB = (256 / NT) > 0 ? 256 / NT : 1;
    static constexpr size_t bytes = (size_t)NWIN * WIN * sizeof(float2) + (size_t)WIN4 * sizeof(float) +
                                    (size_t)OZ * OXP * sizeof(float2) + (size_t)OZ * OXQ * sizeof(float);
    static_assert(NT % CW == 0 && CW >= OX, "owned-node mapping");
};

template <int TX, int TZ, int MODE>
__global__ void __launch_bounds__(PcShape<TX, TZ, MODE>::NT, PcShape<TX, TZ, MODE>::MINB)
    sem_pc_step_kernel(const StepArgs a)
{
    using S = PcShape<TX, TZ, MODE>;
    constexpr int NT = S::NT, NWXP = S::NWXP, NWZ = S::NWZ, WIN = S::WIN;
    constexpr int OXP = S::OXP, OXQ = S::OXQ, CW = S::CW, RPP = S::RPP;

    extern __shared__ float4 smem4[];
    float2 *sw = reinterpret_cast<float2 *>(smem4);     // field window (u_{n+1} or w_{j+1})
    float2 *slm = sw + WIN;                              // (lambda, mu) window; 2nd field later
    float2 *sK = slm + WIN;                              // node sums over the window
    float *sK3 = reinterpret_cast<float *>(sw + S::NWIN * WIN);   // 3rd node sum
    float2 *svh = reinterpret_cast<float2 *>(sK3 + S::WIN4);       // owned half-step velocity
    float *sminv = reinterpret_cast<float *>(svh + S::OZ * OXP);

    const int b = blockIdx.z;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    const int ex0 = blockIdx.x * TX, ez0 = blockIdx.y * TZ;
    const int ix0 = 4 * ex0 - 4, iz0 = 4 * ez0 - 4;
    const int ixo = 4 * ex0, izo = 4 * ez0;              // owned box origin
    const int pitch = a.pitch;
    const long long fo = (long long)b * a.fstride;
    const int ixe = (ex0 + TX >= a.nex) ? a.nx : 4 * (ex0 + TX);
    const int ize = (ez0 + TZ >= a.nez) ? a.nz : 4 * (ez0 + TZ);
    const int ow = ixe - ixo, oh = ize - izo;

    // ---- phase 0: asynchronous prefetch of every input of this step
    prefetch_window<NWZ, NWXP, NT>(sw, a.ucur + fo, ix0, iz0, a.nz, pitch);
    prefetch_window<NWZ, NWXP, NT>(slm, a.lm, ix0, iz0, a.nz, pitch);
    prefetch_owned2<OXP, NT>(svh, a.vh + fo, ixo, izo, ow, oh, pitch);
    prefetch_owned1<OXQ, NT>(sminv, a.minv, ixo, izo, ow, oh, pitch);
    for (int q = threadIdx.x; q < WIN; q += NT) sK[q] = make_float2(0.f, 0.f);
    cp_async_wait_all();
    __syncthreads();

    // ---- phase 1: records, element forces accumulated by colour, sources
    if (MODE == MODE_FWD_PC && a.seis) {
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
    // Element of this thread.  A warp holds R = 32 / (TX + 1) rows of the
    // extended tile, all of one row parity (rows r, r + 2, ...), so its
    // elements take only two of the four colours below and it runs the
    // accumulation body in two of the four passes.
    constexpr int R = 32 / (TX + 1);
    static_assert(R >= 1 && 32 % (TX + 1) == 0 && (TZ + 1) % (2 * R) == 0, "parity-grouped element rows");
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int elx = lane % (TX + 1);
    const int elz = (wid >> 1) * 2 * R + (wid & 1) + 2 * (lane / (TX + 1));
    const bool evalid = (ex0 - 1 + elx >= 0) && (ez0 - 1 + elz >= 0) && (ex0 - 1 + elx < a.nex) &&
                        (ez0 - 1 + elz < a.nez);
    const int ebase = 4 * elz * NWXP + 4 * elx;
    // colour by global element parity: every node then sums its element
    // contributions in the same order whatever the tile shape
    const int colour = ((ex0 - 1 + elx) & 1) | (((ez0 - 1 + elz) & 1) << 1);
    {
        float2 f[25];
        if (evalid) element_force_rows<NWXP>(sw, slm, ebase, f);
#pragma unroll 1
        for (int pass = 0; pass < 4; ++pass) {
            if (evalid && colour == pass) {
#pragma unroll
                for (int j = 0; j < 5; ++j)
#pragma unroll
                    for (int i = 0; i < 5; ++i) {
                        float2 &k = sK[ebase + j * NWXP + i];
                        k.x += f[j * 5 + i].x;
                        k.y += f[j * 5 + i].y;
                    }
            }
            __syncthreads();
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
            int oz = G.node / S::OX, ox = G.node - oz * S::OX;
            float2 &k = sK[(oz + 4) * NWXP + ox + 4];      // K u - F
            k.x -= fx * a.sig_scale;
            k.y -= fz * a.sig_scale;
        }
    }
    __syncthreads();

    // ---- phase 2: Newmark update of the owned nodes, pointwise accumulations
    const float dt = a.dt;
    const int ox = threadIdx.x % CW;
    for (int oz = threadIdx.x / CW; oz < oh; oz += RPP) {
        if (ox >= ow) continue;
        const int ix = ixo + ox, iz = izo + oz;
        const int wq = (oz + 4) * NWXP + ox + 4;
        const long long g = (long long)iz * pitch + ix;
        float2 k = sK[wq];
        float2 v = svh[oz * OXP + ox];
        const bool edge = (ix == 0) | (ix == a.nx - 1) | (iz == 0) | (iz == a.nz - 1);
        float ax, az;
        if (edge) {
            float4 bd = a.bnd[g];
            ax = -(k.x + bd.x * v.x) * bd.z;
            az = -(k.y + bd.y * v.y) * bd.w;
        } else {
            float mi = sminv[oz * OXQ + ox];
            ax = -k.x * mi;
            az = -k.y * mi;
        }
        float2 vn = make_float2(fmaf(dt, ax, v.x), fmaf(dt, az, v.y));
        float2 uc = sw[wq];
        a.vh[fo + g] = vn;
        a.unext[fo + g] = make_float2(fmaf(dt, vn.x, uc.x), fmaf(dt, vn.y, uc.y));
        float *acc = a.acc + (long long)b * a.acc_shot_stride + g;
        if (MODE == MODE_FWD_PC) {
            acc[0] += fmaf(ax, ax, az * az);
        } else {
            const long long ho = (long long)b * a.hstride;
            float2 p0 = a.h0[ho + g], p1 = a.h1[ho + g], p2 = a.h2[ho + g];
            float fxa = (p0.x - p1.x) - (p1.x - p2.x);
            float fza = (p0.y - p1.y) - (p1.y - p2.y);
            acc[0] += fmaf(fxa, ax, fza * az);
        }
    }
    __syncthreads();

    // ---- phase 3: second windows and cleared node sums
    if (MODE == MODE_FWD_PC) {
        load_window<NWZ, NWXP, NT>(sw, a.uold + fo, nullptr, 1, ix0, iz0, a.nz, pitch);      // u_{n+1} - u_n
    } else {
        const long long ho = (long long)b * a.hstride;
        load_window<NWZ, NWXP, NT>(slm, a.h0 + ho, a.h1 + ho, 2, ix0, iz0, a.nz, pitch);     // u_{k+1} - u_k
        load_window<NWZ, NWXP, NT>(sw, a.uold + fo, nullptr, 1, ix0, iz0, a.nz, pitch);      // w_{j+1} - w_j
    }
    for (int q = threadIdx.x; q < WIN; q += NT) {
        sK[q] = make_float2(0.f, 0.f);
        sK3[q] = 0.f;
    }
    __syncthreads();

    // ---- phase 4: element products accumulated by colour
    {
        float pr[75];
        if (evalid) {
            if constexpr (MODE == MODE_FWD_PC)
                element_squares<NWXP>(sw, ebase, pr);
            else
                element_products<NWXP, 3>(sw, slm, ebase, pr);
        }
#pragma unroll 1
        for (int pass = 0; pass < 4; ++pass) {
            if (evalid && colour == pass) {
#pragma unroll
                for (int j = 0; j < 5; ++j)
#pragma unroll
                    for (int i = 0; i < 5; ++i) {
                        int q = ebase + j * NWXP + i, l = (j * 5 + i) * 3;
                        float2 &k = sK[q];
                        k.x += pr[l];
                        k.y += pr[l + 1];
                        sK3[q] += pr[l + 2];
                    }
            }
            __syncthreads();
        }
    }

    // ---- phase 5: accumulate into the global sums
    for (int oz = threadIdx.x / CW; oz < oh; oz += RPP) {
        if (ox >= ow) continue;
        const int ix = ixo + ox, iz = izo + oz;
        const int wq = (oz + 4) * NWXP + ox + 4;
        const long long g = (long long)iz * pitch + ix;
        float2 k = sK[wq];
        float *acc = a.acc + (long long)b * a.acc_shot_stride + g;
        const long long cs = a.acc_comp_stride;
        acc[cs] += k.x;
        acc[2 * cs] += k.y;
        acc[3 * cs] += sK3[wq];
    }
}

// ---------------------------------------------------------------------------
// launch
// ---------------------------------------------------------------------------

template <int TX, int TZ, int MODE>
static int prepare_one()
{
    static bool attr_done[64] = {};          // per device ordinal
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        if constexpr (MODE == MODE_FWD || MODE == MODE_ADJ_G)
            GB_CUDA(cudaFuncSetAttribute(sem_step_kernel<TX, TZ, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)StepShape<TX, TZ, MODE>::bytes));
        else
            GB_CUDA(cudaFuncSetAttribute(sem_pc_step_kernel<TX, TZ, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PcShape<TX, TZ, MODE>::bytes));
        attr_done[dev] = true;
    }
    return GBFWI_OK;
}

template <int TX, int TZ, int MODE>
static int launch_one(const StepArgs &a, int nbatch, cudaStream_t s)
{
    constexpr int NE = (TX + 1) * (TZ + 1);
    GB_TRY((prepare_one<TX, TZ, MODE>()));
    dim3 grid((a.nex + TX - 1) / TX, (a.nez + TZ - 1) / TZ, nbatch);
    if constexpr (MODE == MODE_FWD || MODE == MODE_ADJ_G)
        sem_step_kernel<TX, TZ, MODE><<<grid, NE, StepShape<TX, TZ, MODE>::bytes, s>>>(a);
    else
        sem_pc_step_kernel<TX, TZ, MODE><<<grid, NE, PcShape<TX, TZ, MODE>::bytes, s>>>(a);
    GB_LAUNCHED();
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

template <int TX, int TZ>
static int prepare_mode(int mode)
{
    switch (mode) {
    case MODE_FWD: return prepare_one<TX, TZ, MODE_FWD>();
    case MODE_FWD_PC: return prepare_one<TX, TZ, MODE_FWD_PC>();
    case MODE_ADJ_G: return prepare_one<TX, TZ, MODE_ADJ_G>();
    case MODE_ADJ_PC: return prepare_one<TX, TZ, MODE_ADJ_PC>();
    }
    return GBFWI_EINVAL;
}

int gb_prepare_step(int mode, int tile)
{
    switch (tile) {
    case 0: return prepare_mode<15, 7>(mode);
    case 1: return prepare_mode<7, 15>(mode);
    case 2: return prepare_mode<7, 7>(mode);
    case 3: return prepare_mode<15, 15>(mode);
    case 4: return prepare_mode<31, 3>(mode);
    }
    return GBFWI_EINVAL;
}

const TileShape kTiles[kNumTiles] = {{15, 7}, {7, 15}, {7, 7}, {15, 15}, {31, 3}};

int gb_launch_step(int mode, int tile, const StepArgs &a, int nbatch, cudaStream_t s)
{
    // 16-byte copies and accesses need 16-byte aligned rows and field bases
    if (a.pitch % 4 != 0 || a.fstride % 2 != 0 || a.hstride % 2 != 0 || a.acc_comp_stride % 4 != 0 ||
        a.acc_shot_stride % 4 != 0 || ((uintptr_t)a.ucur & 15) || ((uintptr_t)a.unext & 15) ||
        ((uintptr_t)a.vh & 15) || ((uintptr_t)a.minv & 15) || ((uintptr_t)a.acc & 15) || ((uintptr_t)a.h0 & 15))
        return GBFWI_EINVAL;
    switch (tile) {
    case 0: return launch_mode<15, 7>(mode, a, nbatch, s);
    case 1: return launch_mode<7, 15>(mode, a, nbatch, s);
    case 2: return launch_mode<7, 7>(mode, a, nbatch, s);
    case 3: return launch_mode<15, 15>(mode, a, nbatch, s);
    case 4: return launch_mode<31, 3>(mode, a, nbatch, s);
    }
    return GBFWI_EINVAL;
}
