// Full-history BFGS store, compact-form inverse-Hessian apply and the
// single-pass randomized SVD of the posterior covariance (sm_103a).
//
// Paper: Section 2.1 (Eqs. 1-3, Algorithm 1), Section 2.3 (Eq. 9,
// Algorithms 2-3, Eqs. 10-14).  The inverse Hessian after k pairs started
// from H0 = gamma B0 is applied in the compact form of Byrd, Nocedal &
// Schnabel (1994):
//   H = H0 + [S  H0 Y] [[R^-T (D + Y^T H0 Y) R^-1, -R^-T], [-R^-1, 0]] [S^T; Y^T H0]
// with R_ij = s_i^T y_j (i <= j), D = diag(s_i^T y_i).  It equals the
// recursion of Eq. 3 and the two-loop recursions of Algorithms 1-2.
//
// Layout: vectors are rows, S / Y / B0Y are [kmax][ld] FP32, blocks X / V
// are [p][ld] FP32, with the row pitch ld = n rounded up to 64 floats so
// that every row starts on a 256-byte boundary.  The n-long work is (a)
// split-K products A B^T on the tcgen05 tensor cores (exact three-part
// bfloat16 split, a fresh accumulator per 16-deep step, compensated sums
// within a split, a deterministic FP64 reduction over the splits;
// tc_products.cu), or compensated CUDA-core dot products for up to three
// columns, and (b) row combinations out = coef * rows on the tensor cores;
// the small matrices are FP64 (products spread over SMs, factorisations and
// solves in one CTA or one warp per right-hand side), and the small
// symmetric eigenproblems run as FP32 block Jacobi sweeps in one CTA.
//
// The low-rank part (Algorithm 3, gbfwi_lowrank_invhess): E = (B - B0) X,
// a rank-revealing orthonormal basis Q of E (pivoted Cholesky of E E^T and
// one CholeskyQR pass), Omega (Q X) = Q E by least squares, Omega = U L U^T,
// V = U^T Q, all carried out in the coordinates of W = [S, B0 Y] with the
// Gram matrix W^T W kept by the update (see basis_coords).
// gbfwi_lowrank_exact takes Q from W itself instead of probes.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gbfwi_internal.h"

struct gbfwi_bfgs {
    long long n = 0;
    long long ld = 0;          // row pitch of every [rows][n] block: n rounded up to 64
    int kmax = 0, k = 0;
    DevBuf S, Y, BY, B0;       // [kmax][n] x 3, [n]
    std::vector<double> SY;    // [kmax][kmax]: SY[i*kmax + j] = s_i^T y_j (i <= j)
    std::vector<double> YBY;   // [kmax][kmax]: y_i^T B0 y_j
    std::vector<double> SS, SB, BB;   // [kmax][kmax]: s_i^T s_j, s_i^T B0 y_j, (B0 y_i)^T (B0 y_j)
    DevBuf dSY, dYBY;          // device copies
    DevBuf dG;                 // [2k][2k] FP64: W^T W with W = [S, B0 Y] (rows s_i, then B0 y_i)
    DevBuf part;               // split-K partials
    DevBuf small;              // FP64 small matrices
    DevBuf coef;               // FP32 combination coefficients
    DevBuf X, E, Q, V;         // [p][n] blocks
    DevBuf stage;              // host staging
    DevBuf flag;
    DevBuf status;             // int: nonzero after a product kernel's bounded wait gave up
    DevBuf ex;                 // FP64 scratch of the low-rank decompositions
};

namespace {

// One term of a compensated FP32 dot product (Ogita, Rump & Oishi 2005,
// "Accurate sum and dot product", algorithm Dot2): the product is split
// exactly into pr + pe with an FMA, the running sum hi + pr exactly into
// s + se (Knuth's TwoSum), and the error terms are collected in lo.  The
// _rn intrinsics keep the compiler from contracting the products into FMAs,
// which would break the exact splits.  The result hi + lo is as accurate as
// an FP64-accumulated sum of the FP32 products up to a term in n eps^2.
__device__ __forceinline__ void dot2_term(float a, float b, float &hi, float &lo)
{
    const float pr = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -pr);
    const float sm = __fadd_rn(hi, pr);
    const float z = __fsub_rn(sm, hi);
    const float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(sm, z)), __fsub_rn(pr, z));
    hi = sm;
    lo = __fadd_rn(lo, __fadd_rn(se, pe));
}

// Products with kb <= 2 columns (dot products of the pair updates, the
// search direction): CTA (split, a) accumulates row a against the kb
// columns with compensated (Dot2) sums, then an FP64 tree over its threads;
// part[sx][a][b] is reduced over the splits by atb_reduce.
template <int KB>
__global__ void __launch_bounds__(256) atb_thin(const float *__restrict__ A, long long lda,
                                                const float *__restrict__ Bm, long long ldb,
                                                const float *__restrict__ w, long long n, long long chunk, int ka,
                                                double *__restrict__ part)
{
    __shared__ double red[KB][256];
    const int sx = blockIdx.x, a = blockIdx.y, t = threadIdx.x;
    const long long ib = (long long)sx * chunk, ie = min(n, ib + chunk);
    float hi[KB], lo[KB];
#pragma unroll
    for (int b = 0; b < KB; ++b) hi[b] = lo[b] = 0.f;
    const float *ar = A + (long long)a * lda;
    for (long long i = ib + t; i < ie; i += blockDim.x) {
        const float av = __ldg(ar + i);
#pragma unroll
        for (int b = 0; b < KB; ++b) {
            float bv = __ldg(Bm + (long long)b * ldb + i);
            if (w) bv *= __ldg(w + i);
            dot2_term(av, bv, hi[b], lo[b]);
        }
    }
#pragma unroll
    for (int b = 0; b < KB; ++b) red[b][t] = (double)hi[b] + (double)lo[b];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (t < h)
#pragma unroll
            for (int b = 0; b < KB; ++b) red[b][t] += red[b][t + h];
        __syncthreads();
    }
    if (t == 0)
#pragma unroll
        for (int b = 0; b < KB; ++b) part[((long long)sx * ka + a) * KB + b] = red[b][0];
}

__global__ void atb_reduce(const double *__restrict__ part, int nsplit, int nab, double *__restrict__ out,
                           long long ldo, int kb)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nab) return;
    double s = 0.0;
    for (int sx = 0; sx < nsplit; ++sx) s += part[(long long)sx * nab + q];
    int a = q / kb, b = q - a * kb;
    out[(long long)a * ldo + b] = s;
}

// Dot products of a new pair with the store (the update of the Gram
// matrices): CTA (split, a) takes row a of [S_0..S_{k1-1}, B0Y_0..B0Y_{k1-1}]
// against the three vectors (y, s, B0 y) with compensated (Dot2) sums, then
// an FP64 tree over its threads; part[sx][a][b] is reduced over the splits
// by atb_reduce.
__global__ void __launch_bounds__(256) pair_dots_kernel(const float *__restrict__ S, const float *__restrict__ BY,
                                                        long long ld, int k1, const float *__restrict__ y,
                                                        const float *__restrict__ sv, const float *__restrict__ by,
                                                        long long n, long long chunk, double *__restrict__ part)
{
    __shared__ double red[3][256];
    const int sx = blockIdx.x, a = blockIdx.y, t = threadIdx.x;
    const long long ib = (long long)sx * chunk, ie = min(n, ib + chunk);
    const float *ar = a < k1 ? S + (long long)a * ld : BY + (long long)(a - k1) * ld;
    float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
    for (long long i = ib + t; i < ie; i += blockDim.x) {
        const float av = __ldg(ar + i);
        dot2_term(av, __ldg(y + i), hi[0], lo[0]);
        dot2_term(av, __ldg(sv + i), hi[1], lo[1]);
        dot2_term(av, __ldg(by + i), hi[2], lo[2]);
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) red[b][t] = (double)hi[b] + (double)lo[b];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (t < h)
#pragma unroll
            for (int b = 0; b < 3; ++b) red[b][t] += red[b][t + h];
        __syncthreads();
    }
    if (t == 0)
#pragma unroll
        for (int b = 0; b < 3; ++b) part[((long long)sx * 2 * k1 + a) * 3 + b] = red[b][0];
}

// out[c][i] = sum_a coef[c][a] row_a[i] + beta * dw[i] * Xc[c][i]  for c in [c0, c0 + cn)
// rows a < k1 from A1, the rest from A2 (row stride lda)
template <int CB>
__global__ void __launch_bounds__(128) combine_kernel(const float *__restrict__ A1, const float *__restrict__ A2,
                                                      int k1, int ktot, long long lda,
                                                      const float *__restrict__ coef, int c0, int cn,
                                                      long long n, float *__restrict__ out, long long ldo,
                                                      const float *__restrict__ dw, const float *__restrict__ Xc,
                                                      long long ldx, float beta)
{
    extern __shared__ float4 cs4[];   // [ktot][CB/4]
    float *cs = reinterpret_cast<float *>(cs4);
    for (int q = threadIdx.x; q < ktot * CB; q += blockDim.x) {
        int a = q / CB, cc = q - a * CB;
        cs[q] = cc < cn ? coef[(long long)(c0 + cc) * ktot + a] : 0.f;
    }
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float acc[CB];
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) acc[cc] = 0.f;
        int a = 0;
        for (; a + 4 <= ktot; a += 4) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float *row = (a + u) < k1 ? A1 + (long long)(a + u) * lda : A2 + (long long)(a + u - k1) * lda;
                v[u] = __ldg(row + i);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 *c4 = cs4 + (a + u) * (CB / 4);
#pragma unroll
                for (int q = 0; q < CB / 4; ++q) {
                    float4 c = c4[q];
                    acc[4 * q + 0] = fmaf(c.x, v[u], acc[4 * q + 0]);
                    acc[4 * q + 1] = fmaf(c.y, v[u], acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(c.z, v[u], acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(c.w, v[u], acc[4 * q + 3]);
                }
            }
        }
        for (; a < ktot; ++a) {
            const float *row = a < k1 ? A1 + (long long)a * lda : A2 + (long long)(a - k1) * lda;
            float v = __ldg(row + i);
            const float4 *c4 = cs4 + a * (CB / 4);
#pragma unroll
            for (int q = 0; q < CB / 4; ++q) {
                float4 c = c4[q];
                acc[4 * q + 0] = fmaf(c.x, v, acc[4 * q + 0]);
                acc[4 * q + 1] = fmaf(c.y, v, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(c.z, v, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(c.w, v, acc[4 * q + 3]);
            }
        }
        float d = (beta != 0.f) ? beta * dw[i] : 0.f;
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) {
            if (cc < cn) {
                float r = acc[cc];
                if (beta != 0.f) r = fmaf(d, Xc[(long long)(c0 + cc) * ldx + i], r);
                out[(long long)(c0 + cc) * ldo + i] = r;
            }
        }
    }
}

__global__ void mul_kernel(const float *__restrict__ a, const float *__restrict__ b, long long n,
                           float *__restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] * b[i];
}

// Largest of the lanes' values (first index among equals; idx < 0: none),
// broadcast to the warp.  The values are compared through their IEEE bit
// patterns as signed 64-bit integers, which orders every non-negative double
// (and puts any negative one below them): integer compares and shuffles
// instead of FP64 compares in the pivot searches' serial steps.
__device__ __forceinline__ void warp_argmax_nonneg(double &v, int &idx)
{
    long long key = __double_as_longlong(v);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const long long ok = __shfl_down_sync(0xffffffffu, key, off);
        const int oi = __shfl_down_sync(0xffffffffu, idx, off);
        if (oi >= 0 && (idx < 0 || ok > key || (ok == key && oi < idx))) { key = ok; idx = oi; }
    }
    key = __shfl_sync(0xffffffffu, key, 0);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    v = __longlong_as_double(key);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Compact-form middle product for each column c of T ([2k][p], row stride
// p: rows 0..k-1 S^T x_c, rows k..2k-1 (B0 Y)^T x_c):
//   cv = R^-1 a, top = R^-T ((D + gamma Y^T B0 Y) cv - gamma t2)
//   coef[c] = [top, -gamma cv]
// i.e. coef[c] = M T_c with M the middle matrix of the compact form.  One
// warp per probe column c (block c): the k-long FP64 triangular solves and
// the Y^T B0 Y product, dot products split over the lanes; FP64 is spread
// over p SMs instead of one.  The solves are chains of dependent steps, so
// everything they read sits in shared memory (middle_smem_bytes): cv, d,
// the reciprocals of R's diagonal (formed once, in parallel: no division
// in the chains) and, when mats, R = S^T Y and Y^T B0 Y themselves (k x k
// each; otherwise they are read from global memory).  Outputs (either may
// be null): coef FP32 and coefd FP64, both [p][2k].
__host__ __device__ inline size_t middle_smem_bytes(int k, bool mats)
{
    return ((mats ? 2 * (size_t)k * k : 0) + 3 * (size_t)k) * sizeof(double);
}

__global__ void __launch_bounds__(32) middle_kernel(const double *__restrict__ T, const double *__restrict__ SYg,
                                                    const double *__restrict__ YBYg, int k, int kmax, int p,
                                                    double gamma, int mats, float *__restrict__ coef,
                                                    double *__restrict__ coefd)
{
    extern __shared__ double msm[];
    const int c = blockIdx.x, lane = threadIdx.x;
    if (c >= p) return;
    double *cv = msm, *d = cv + k, *rdiag = d + k;
    const double *SY = SYg, *YBY = YBYg;
    long long ls = kmax;                                // row stride of SY / YBY
    if (mats) {
        double *S1 = rdiag + k, *S2 = S1 + (size_t)k * k;
        for (int q = lane; q < k * k; q += 32) {
            const int i = q / k, j = q - i * k;
            S1[q] = __ldg(SYg + (long long)i * kmax + j);
            S2[q] = __ldg(YBYg + (long long)i * kmax + j);
        }
        SY = S1;
        YBY = S2;
        ls = k;
    }
    for (int i = lane; i < k; i += 32) rdiag[i] = 1.0 / __ldg(SYg + (long long)i * kmax + i);
    __syncwarp();
    // R cv = T_top (back substitution), R_ij = s_i^T y_j upper
    for (int i = k - 1; i >= 0; --i) {
        double s = 0.0;
        for (int j = i + 1 + lane; j < k; j += 32) s += SY[i * ls + j] * cv[j];
        s = warp_sum(s);
        if (lane == 0) cv[i] = (__ldg(T + (long long)i * p + c) - s) * rdiag[i];
        __syncwarp();
    }
    for (int i = 0; i < k; ++i) {
        double t = 0.0;
        for (int j = lane; j < k; j += 32) t += YBY[i * ls + j] * cv[j];
        t = warp_sum(t);
        if (lane == 0) d[i] = SY[i * ls + i] * cv[i] + gamma * t - gamma * __ldg(T + (long long)(k + i) * p + c);
    }
    __syncwarp();
    // R^T top = d (forward substitution); overwrite d with top
    for (int i = 0; i < k; ++i) {
        double s = 0.0;
        for (int j = lane; j < i; j += 32) s += SY[j * ls + i] * d[j];
        s = warp_sum(s);
        if (lane == 0) d[i] = (d[i] - s) * rdiag[i];
        __syncwarp();
    }
    for (int i = lane; i < k; i += 32) {
        const double top = d[i], bot = -gamma * cv[i];
        if (coef) {
            coef[(long long)c * 2 * k + i] = (float)top;
            coef[(long long)c * 2 * k + k + i] = (float)bot;
        }
        if (coefd) {
            coefd[(long long)c * 2 * k + i] = top;
            coefd[(long long)c * 2 * k + k + i] = bot;
        }
    }
}

// The same product with the solves column-oriented, for k <= 32 NJ: lane l
// owns the unknowns l + 32 t (t < NJ) in registers; step i of a triangular
// solve is one multiply by the precomputed reciprocal pivot on the owner
// lane, a shuffle of the result and one FMA per owned unknown, so the
// dependent chain per step is three FP64 operations instead of a warp
// reduction (five dependent FP64 adds).  Y^T B0 Y cv accumulates the same
// way over the broadcast cv_i.  Shared memory and outputs as middle_kernel.
template <int NJ>
__device__ __forceinline__ double pick_nj(const double (&v)[NJ], int t)
{
    double r = v[0];
#pragma unroll
    for (int q = 1; q < NJ; ++q)
        if (q == t) r = v[q];
    return r;
}

template <int NJ>
__global__ void __launch_bounds__(32) middle_col_kernel(const double *__restrict__ T, const double *__restrict__ SYg,
                                                        const double *__restrict__ YBYg, int k, int kmax, int p,
                                                        double gamma, int mats, float *__restrict__ coef,
                                                        double *__restrict__ coefd)
{
    extern __shared__ double msm[];
    const int c = blockIdx.x, lane = threadIdx.x;
    if (c >= p) return;
    double *rdiag = msm + 2 * k;                        // the layout of middle_kernel: cv, d, rdiag, R, YBY
    const double *SY = SYg, *YBY = YBYg;
    long long ls = kmax;
    if (mats) {
        double *S1 = rdiag + k, *S2 = S1 + (size_t)k * k;
        for (int q = lane; q < k * k; q += 32) {
            const int i = q / k, j = q - i * k;
            S1[q] = __ldg(SYg + (long long)i * kmax + j);
            S2[q] = __ldg(YBYg + (long long)i * kmax + j);
        }
        SY = S1;
        YBY = S2;
        ls = k;
    }
    for (int i = lane; i < k; i += 32) rdiag[i] = 1.0 / __ldg(SYg + (long long)i * kmax + i);
    __syncwarp();
    double x[NJ], cv[NJ], acc[NJ];
#pragma unroll
    for (int t = 0; t < NJ; ++t) {
        const int j = lane + 32 * t;
        x[t] = j < k ? __ldg(T + (long long)j * p + c) : 0.0;
        cv[t] = 0.0;
        acc[t] = 0.0;
    }
    // R cv = T_top (back substitution), R_ij = s_i^T y_j upper: cv_i final at step i
    for (int i = k - 1; i >= 0; --i) {
        const int ti = i >> 5, li = i & 31;
        const double v = __shfl_sync(0xffffffffu, pick_nj<NJ>(x, ti) * rdiag[i], li);
#pragma unroll
        for (int t = 0; t < NJ; ++t) {
            const int j = lane + 32 * t;
            if (t == ti && lane == li) cv[t] = v;
            if (j < i) x[t] = fma(-SY[j * ls + i], v, x[t]);
        }
    }
    // acc = Y^T B0 Y cv (column by column over the broadcast cv_i)
    for (int i = 0; i < k; ++i) {
        const double v = __shfl_sync(0xffffffffu, pick_nj<NJ>(cv, i >> 5), i & 31);
#pragma unroll
        for (int t = 0; t < NJ; ++t) {
            const int j = lane + 32 * t;
            if (j < k) acc[t] = fma(YBY[j * ls + i], v, acc[t]);
        }
    }
    // d = D cv + gamma (Y^T B0 Y cv - t2), then R^T top = d (forward substitution)
#pragma unroll
    for (int t = 0; t < NJ; ++t) {
        const int j = lane + 32 * t;
        x[t] = j < k ? SY[j * ls + j] * cv[t] + gamma * acc[t] - gamma * __ldg(T + (long long)(k + j) * p + c) : 0.0;
    }
    double top[NJ];
#pragma unroll
    for (int t = 0; t < NJ; ++t) top[t] = 0.0;
    for (int i = 0; i < k; ++i) {
        const int ti = i >> 5, li = i & 31;
        const double v = __shfl_sync(0xffffffffu, pick_nj<NJ>(x, ti) * rdiag[i], li);
#pragma unroll
        for (int t = 0; t < NJ; ++t) {
            const int j = lane + 32 * t;
            if (t == ti && lane == li) top[t] = v;
            if (j > i && j < k) x[t] = fma(-SY[i * ls + j], v, x[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < NJ; ++t) {
        const int j = lane + 32 * t;
        if (j >= k) continue;
        const double bot = -gamma * cv[t];
        if (coef) {
            coef[(long long)c * 2 * k + j] = (float)top[t];
            coef[(long long)c * 2 * k + k + j] = (float)bot;
        }
        if (coefd) {
            coefd[(long long)c * 2 * k + j] = top[t];
            coefd[(long long)c * 2 * k + k + j] = bot;
        }
    }
}

// out[i][j] = sum_l A(i, l) B(l, j), i < M, j < N, l < K, with A(i, l) =
// A[i ar + l ac] and B(l, j) = B[l br + j bc] (any transposition by the
// strides), FP64 accumulation in l order; one thread per output element,
// blocks (N / 32, M): the small FP64 products of the decompositions spread
// over the SMs (GB300 runs about two FP64 FMAs per clock per SM).  Outputs
// (either may be null): out FP64 and outf FP32, both with row stride ldo.
template <typename TA>
__global__ void __launch_bounds__(32) small_gemm_kernel(int M, int N, int K, const TA *__restrict__ A, long long ar,
                                                        long long ac, const double *__restrict__ B, long long br,
                                                        long long bc, double *__restrict__ out,
                                                        float *__restrict__ outf, long long ldo)
{
    const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y;
    if (j >= N || i >= M) return;
    const TA *a = A + (long long)i * ar;
    const double *b = B + (long long)j * bc;
    double acc = 0.0;
    for (int l = 0; l < K; ++l) acc = fma((double)a[(long long)l * ac], b[(long long)l * br], acc);
    if (out) out[(long long)i * ldo + j] = acc;
    if (outf) outf[(long long)i * ldo + j] = (float)acc;
}

// Block-cooperative cyclic Jacobi (FP32) for a symmetric p x p matrix A
// (row-major, scaled to |A|_F = 1, overwritten by the rotated matrix, its
// eigenvalues on the diagonal); U accumulates the eigenvectors as columns
// (must hold I on entry).  Round-robin pairing gives P/2 disjoint rotations
// per round (P = p rounded up to even); the pairing of every round is
// tabulated once.  A pair is rotated only while |a_pq| > 1e-7 sqrt(|a_pp
// a_qq|) (the relative threshold of Demmel & Veselic 1992, which also
// resolves small eigenvalues of a graded matrix) and |a_pq| > 4e-7 |A|_F
// (below that an entry is rounding noise of the largest eigenvalues:
// rotating it changes nothing at this precision); the sweeps stop after one
// without a rotation, or after max_sweeps.  The rotation annihilating
// a_pq, with |theta| <= pi/4 and tan 2 theta = 2 a_pq / (a_qq - a_pp), comes
// from the half-angle formulas: with d = a_qq - a_pp and rho = 1 / sqrt(d^2
// + 4 a_pq^2), cos 2 theta = |d| rho, c = sqrt((1 + cos 2 theta) / 2) and
// s = sign(d) a_pq rho / c: two reciprocal square roots and no division
// (the scaling keeps d^2 + 4 a_pq^2 in range for every rotated pair).
//
// Work split without index divisions: every warp forms the round's
// rotations itself in registers (lane l: the pairs l + 32 j, j < NJ; a
// warp's row pair comes from its owner lane by a shuffle), a barrier, then
// warp w rotates the 2 x 2 blocks (a pair of rows by a pair of columns, both
// sides in one pass, in place; blocks of two unrotated pairs are skipped) of
// the row pairs w, w + nwarps, .. against lane l's column pairs, and
// U <- U J (element (i, pair m) belongs to lane m mod 32 of warp
// i mod nwarps), a barrier.  P / 2 <= 32 NJ.  pairs: P (P - 1) shorts.
template <int NJ>
__device__ void block_jacobi(float *A, float *U, int p, short *pairs, int max_sweeps)
{
    const int t = threadIdx.x, nt = blockDim.x;
    const int lane = t & 31, warp = t >> 5, nw = nt >> 5;
    const float rel2 = 1e-14f, abs_tol = 4e-7f;   // (1e-7)^2; 4e-7 |A|_F with |A|_F = 1
    __shared__ int rotated;
    const int P = (p + 1) & ~1;
    const int npair = P / 2;
    // pairs[round][m] = (a, b), a < b, round-robin with element 0 fixed
    for (int q = t; q < (P - 1) * npair; q += nt) {
        const int round = q / npair, m = q - round * npair;
        const int a = m == 0 ? 0 : 1 + (m - 1 + round) % (P - 1);
        const int b = 1 + (P - 2 - m + round) % (P - 1);
        pairs[2 * q] = (short)min(a, b);
        pairs[2 * q + 1] = (short)max(a, b);
    }
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (t == 0) rotated = 0;
        __syncthreads();
        for (int round = 0; round < P - 1; ++round) {
            const short *pr = pairs + 2 * round * npair;
            float cr[NJ], sr[NJ];
            int pm[NJ], qm[NJ];
            bool any = false;
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                cr[j] = 1.f;
                sr[j] = 0.f;
                pm[j] = qm[j] = p;
                const int m = lane + 32 * j;
                if (m < npair) {
                    const int pp = pr[2 * m], qq = pr[2 * m + 1];
                    pm[j] = pp;
                    qm[j] = qq;
                    if (qq < p) {
                        const float apq = A[pp * p + qq];
                        const float app = A[pp * p + pp], aqq = A[qq * p + qq];
                        if (apq * apq > rel2 * fabsf(app * aqq) && fabsf(apq) > abs_tol) {
                            const float d = aqq - app, two = 2.f * apq;
                            const float rho = rsqrtf(fmaf(d, d, two * two));
                            const float x = fmaf(0.5f * fabsf(d), rho, 0.5f);      // c^2
                            const float rx = rsqrtf(x);                            // 1 / c
                            cr[j] = x * rx;
                            sr[j] = copysignf(1.f, d) * (apq * rho) * rx;
                            any = true;
                        }
                    }
                }
            }
            if (warp == 0 && any) rotated = 1;
            __syncthreads();                    // every rotation read its pair before any update
            for (int m1 = warp; m1 < npair; m1 += nw) {
                const int o = m1 & 31, j1 = m1 >> 5;
                float c1 = cr[0], s1 = sr[0];
                int p1 = pm[0], q1 = qm[0];
#pragma unroll
                for (int j = 1; j < NJ; ++j)
                    if (j == j1) { c1 = cr[j]; s1 = sr[j]; p1 = pm[j]; q1 = qm[j]; }
                c1 = __shfl_sync(0xffffffffu, c1, o);
                s1 = __shfl_sync(0xffffffffu, s1, o);
                p1 = __shfl_sync(0xffffffffu, p1, o);
                q1 = __shfl_sync(0xffffffffu, q1, o);
                const bool hq1 = q1 < p;
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const float c2 = cr[j], s2 = sr[j];
                    if (lane + 32 * j >= npair || (s1 == 0.f && s2 == 0.f)) continue;
                    const int p2 = pm[j], q2 = qm[j];
                    const bool hq2 = q2 < p;
                    float *r1 = A + p1 * p, *r2 = A + q1 * p;
                    const float a = r1[p2];
                    const float b = hq2 ? r1[q2] : 0.f;
                    const float cc = hq1 ? r2[p2] : 0.f;
                    const float d = (hq1 && hq2) ? r2[q2] : 0.f;
                    // rows (pair m1), then columns (pair m2)
                    const float ra = c1 * a - s1 * cc, rc = s1 * a + c1 * cc;
                    const float rb = c1 * b - s1 * d, rd = s1 * b + c1 * d;
                    r1[p2] = c2 * ra - s2 * rb;
                    if (hq2) r1[q2] = s2 * ra + c2 * rb;
                    if (hq1) r2[p2] = c2 * rc - s2 * rd;
                    if (hq1 && hq2) r2[q2] = s2 * rc + c2 * rd;
                }
            }
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                if (sr[j] == 0.f) continue;
                const int pp = pm[j], qq = qm[j];
                const float c = cr[j], sn = sr[j];
                for (int l = warp; l < p; l += nw) {
                    float *ur = U + l * p;
                    const float u = ur[pp], v = ur[qq];
                    ur[pp] = c * u - sn * v;
                    ur[qq] = sn * u + c * v;
                }
            }
            __syncthreads();
        }
        if (!rotated) break;
        __syncthreads();
    }
    __syncthreads();
}

// Rank-revealing basis of the probe block E [p][n] from its FP64 Gram matrix
// G = E E^T by diagonally pivoted Cholesky (the normal-equations form of QR
// with column pivoting on E): at step j the row of E with the largest
// remaining residual norm is taken, and the factorisation stops once that
// norm falls below tol times the largest row norm.  With the r selected rows
// E_s (permutation piv) and G_ss = R^T R, Q1 = R^-T E_s has orthonormal rows
// spanning them; the returned coef [r][p] gives Q1 = coef E (zero columns for
// the rows not taken).  An FP32 block carries ~1e-7 relative rounding, so
// directions far below the largest are noise: taking them would amplify
// that rounding by s_max / s_i.  With tol = 0 on a nearly orthonormal
// block's Gram matrix the kernel is one CholeskyQR pass (every row is taken;
// the pivoting only reorders them).  Each step's pivot takes one reciprocal
// square root (its reciprocal is kept for the inverse), so neither loop
// holds a division.  work: >= 3 p^2 + 2 p doubles.
__global__ void __launch_bounds__(512) gram_pivchol_kernel(const double *__restrict__ G, int p, double tol, double *work,
                                    double *__restrict__ coef, int *__restrict__ r_out, int *__restrict__ flag,
                                    int use_smem)
{
    extern __shared__ double smem_work[];
    if (use_smem) work = smem_work;
    const int t = threadIdx.x, nt = blockDim.x;
    const int tx = t & 31, ty = t >> 5;                 // 32 x 16 grid of the trailing updates (512 threads)
    const long long pp = (long long)p * p;
    double *A = work, *R = A + pp, *Ri = R + pp;
    int *piv = reinterpret_cast<int *>(Ri + pp);
    double *rinv = Ri + pp + p;                         // 1 / R_jj
    __shared__ int s_r, s_go;
    __shared__ double s_dinv, s_d0;
    if (tol == 0.0) {
        // CholeskyQR pass: a block already orthonormal to 1e-9 (far below
        // FP32 rounding) keeps its basis, coef = I
        __shared__ double s_dev[16];
        // largest deviation from I; a NaN sticks (it then fails the test
        // below, and the factorisation flags it)
        auto dmax = [](double a, double b) { return (b > a || b != b) ? b : a; };
        double dev = 0.0;
        for (long long q = t; q < pp; q += nt) {
            const long long i = q / p;
            dev = dmax(dev, fabs(G[q] - (q == i * p + i ? 1.0 : 0.0)));
        }
        for (int o = 16; o > 0; o >>= 1) dev = dmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
        if (tx == 0) s_dev[ty] = dev;
        __syncthreads();
        dev = 0.0;
        for (int w = 0; w < (nt >> 5); ++w) dev = dmax(dev, s_dev[w]);
        if (dev <= 1e-9) {
            for (long long q = t; q < pp; q += nt) {
                const long long i = q / p;
                coef[q] = q == i * p + i ? 1.0 : 0.0;
            }
            if (t == 0) *r_out = p;
            return;
        }
    }
    for (long long q = t; q < pp; q += nt) {
        A[q] = G[q];
        R[q] = 0.0;
    }
    for (int i = t; i < p; i += nt) piv[i] = i;
    if (t == 0) s_r = p;
    __syncthreads();
    for (int j = 0; j < p; ++j) {
        if (t < 32) {
            // largest remaining residual (first index among equals), warp 0
            int best = -1;
            double bv = 0.0;
            for (int k = j + t; k < p; k += 32) {
                const double d = A[(long long)piv[k] * p + piv[k]];
                if (best < 0 || __double_as_longlong(d) > __double_as_longlong(bv)) { bv = d; best = k; }
            }
            warp_argmax_nonneg(bv, best);
            if (best < 0) bv = -1.0;
            if (t == 0 && j == 0) {
                s_d0 = bv;
                if (!(bv > 0.0) || !isfinite(bv)) *flag = 1;
            }
            __syncwarp();
            const bool go = best >= 0 && bv > tol * tol * s_d0;
            if (go) {
                for (int i = t; i < j; i += 32) {  // the finished rows of R follow the swap
                    const double x = R[(long long)i * p + j];
                    R[(long long)i * p + j] = R[(long long)i * p + best];
                    R[(long long)i * p + best] = x;
                }
            }
            if (t == 0) {
                if (!go) {
                    s_r = j;
                    s_go = 0;
                } else {
                    const int tmp = piv[j];
                    piv[j] = piv[best];
                    piv[best] = tmp;
                    const double di = rsqrt(bv);
                    R[(long long)j * p + j] = bv * di;
                    rinv[j] = di;
                    s_dinv = di;
                    s_go = 1;
                }
            }
        }
        __syncthreads();
        if (!s_go) break;
        // row j of R, then the trailing update from it (one FP64 FMA per
        // element; neither touches row or column piv[j] of A)
        const int pj = piv[j];
        const double dinv = s_dinv;
        const double *Aj = A + (long long)pj * p;
        double *Rj = R + (long long)j * p;
        for (int k = j + 1 + t; k < p; k += nt) Rj[k] = Aj[piv[k]] * dinv;
        __syncthreads();
        for (int kk = j + 1 + ty; kk < p; kk += 16) {
            const double rk = Rj[kk];
            double *Ak = A + (long long)piv[kk] * p;
            for (int ll = j + 1 + tx; ll < p; ll += 32) Ak[piv[ll]] = fma(-rk, Rj[ll], Ak[piv[ll]]);
        }
        __syncthreads();
    }
    const int r = s_r;
    // R11^-1 (upper, r x r) by the column-oriented back substitution, one
    // barrier per step: at step i row i is final (B[i][c] / R[i][i]) and is
    // removed from the rows above; B (= I at the start) lives in A, free now
    for (int a = ty; a < r; a += 16)
        for (int c = tx; c < r; c += 32) {
            A[(long long)a * r + c] = a == c ? 1.0 : 0.0;
            Ri[(long long)a * r + c] = 0.0;            // the strict lower triangle stays zero
        }
    __syncthreads();
    for (int i = r - 1; i >= 0; --i) {
        const double rii = rinv[i];
        for (int a = ty; a <= i; a += 16)
            for (int c = tx; c < r; c += 32) {
                if (c < i) continue;
                const double xi = A[(long long)i * r + c] * rii;
                if (a == i)
                    Ri[(long long)i * r + c] = xi;
                else
                    A[(long long)a * r + c] -= R[(long long)a * p + i] * xi;
            }
        __syncthreads();
    }
    for (long long q = t; q < pp; q += nt) coef[q] = 0.0;
    __syncthreads();
    // coef[a][piv[b]] = (R11^-T)[a][b] = R11^-1[b][a]
    for (int q = t; q < r * r; q += nt) {
        const int a = q / r, b = q % r;
        coef[(long long)a * p + piv[b]] = Ri[(long long)b * r + a];
    }
    if (t == 0) *r_out = r;
}

// Eigenpairs of the Jacobi result (eigenvalues on the diagonal of Af,
// eigenvectors in the columns of Uf, r x r) ordered by |lambda| descending
// (the first index among equal magnitudes): lam[k] and coef [rank][r] = U^T,
// zero beyond r; the eigenvalues are the diagonal times scale.  Each
// eigenvalue's position is its count of larger ones, so every thread places
// its own.  A non-finite eigenvalue sets flag 4.
__device__ void select_eigenpairs(const float *Af, const float *Uf, int r, int rank, double scale, double *__restrict__ lam,
                                  float *__restrict__ coef, int *__restrict__ flag)
{
    const int t = threadIdx.x, nt = blockDim.x;
    for (int i = t; i < r; i += nt) {
        const float vi = fabsf(Af[(long long)i * r + i]);
        if (!isfinite(vi)) *flag = 4;
        int pos = 0;
        for (int j = 0; j < r; ++j) {
            const float vj = fabsf(Af[(long long)j * r + j]);
            pos += (vj > vi || (vj == vi && j < i)) ? 1 : 0;
        }
        if (pos < rank) {
            lam[pos] = (double)Af[(long long)i * r + i] * scale;
            for (int a = 0; a < r; ++a) coef[(long long)pos * r + a] = Uf[(long long)a * r + i];
        }
    }
    for (int q = t; q < (rank - min(rank, r)) * r; q += nt) coef[(long long)min(rank, r) * r + q] = 0.f;
    for (int k = r + t; k < rank; k += nt) lam[k] = 0.0;
}


// d_i = 1 / sqrt(G_ii) (0 for an empty row), G <- D G D: the pivoted
// Cholesky then compares directions, not the scales of S and B0 Y
// Omega from Omega (Q^T X) = Q^T E (Algorithm 3) in four steps, the FP64
// work spread over SMs where it is independent:
//   omega_system_kernel (block i): row i of the system N Omega^T = Bm^T:
//     square Q^T X: N = (Q^T X)^T, Bm^T = (Q^T E)^T; wide Q^T X (r < p): the
//     normal equations N = QX QX^T, Bm = QE QX^T;
//   lu_kernel (one CTA): N = P^T L U by partial pivoting (first row among
//     equal magnitudes), one barrier per elimination step; a zero pivot sets
//     flag 3 and is taken as 1;
//   lu_solve_kernel (block c): column c of Omega^T from its right-hand side;
//   then sym_kernel and eig_select_kernel.
__global__ void __launch_bounds__(32) omega_system_kernel(const double *__restrict__ QE,
                                                          const double *__restrict__ QX, long long ldq, int r, int p,
                                                          double *__restrict__ N, double *__restrict__ Bt)
{
    const int i = blockIdx.x, lane = threadIdx.x;
    if (i >= r) return;
    for (int j = 0; j < r; ++j) {
        if (r == p) {
            if (lane == 0) {
                N[(long long)i * r + j] = QX[(long long)j * ldq + i];
                Bt[(long long)i * r + j] = QE[(long long)j * ldq + i];
            }
            continue;
        }
        double nij = 0.0, bji = 0.0;
        for (int c = lane; c < p; c += 32) {
            const double xi = QX[(long long)i * ldq + c];
            nij += xi * QX[(long long)j * ldq + c];
            bji += QE[(long long)j * ldq + c] * xi;
        }
        nij = warp_sum(nij);
        bji = warp_sum(bji);
        if (lane == 0) {
            N[(long long)i * r + j] = nij;
            Bt[(long long)i * r + j] = bji;               // Bm^T[i][j] = Bm[j][i]
        }
    }
}

__global__ void __launch_bounds__(512) lu_kernel(double *__restrict__ M, double *__restrict__ L, int *__restrict__ perm,
                                                 int r, int *__restrict__ flag, int use_smem)
{
    extern __shared__ double lu_smem[];
    double *A = use_smem ? lu_smem : M;
    double *Ls = use_smem ? lu_smem + (size_t)r * r : L;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int a = ty; a < r; a += 16)
        for (int c = tx; c < r; c += 32) {
            if (use_smem) A[a * r + c] = M[(long long)a * r + c];
            Ls[a * r + c] = 0.0;
        }
    __syncthreads();
    for (int j = 0; j < r; ++j) {
        if (threadIdx.x < 32) {
            int best = -1;
            double bv = 0.0;
            for (int a = j + tx; a < r; a += 32) {
                const double v = fabs(A[a * r + j]);
                if (best < 0 || __double_as_longlong(v) > __double_as_longlong(bv)) { bv = v; best = a; }
            }
            warp_argmax_nonneg(bv, best);
            if (best < 0) bv = -1.0;
            if (best < 0) best = j;
            if (tx == 0) {
                if (!(bv > 0.0)) *flag = 3;
                perm[j] = best;
            }
            if (best != j)
                for (int c = tx; c < r; c += 32) {
                    const double x = A[j * r + c];
                    A[j * r + c] = A[best * r + c];
                    A[best * r + c] = x;
                    if (c < j) {
                        const double y = Ls[j * r + c];
                        Ls[j * r + c] = Ls[best * r + c];
                        Ls[best * r + c] = y;
                    }
                }
        }
        __syncthreads();
        double d = A[j * r + j];
        if (d == 0.0) d = 1.0;
        const double inv = 1.0 / d;
        for (int a = j + 1 + ty; a < r; a += 16) {
            const double l = A[a * r + j] * inv;
            for (int c = j + 1 + tx; c < r; c += 32) A[a * r + c] -= l * A[j * r + c];
            if (tx == 0) Ls[a * r + j] = l;
        }
        __syncthreads();
    }
    if (use_smem)
        for (int a = ty; a < r; a += 16)
            for (int c = tx; c < r; c += 32) {
                M[(long long)a * r + c] = A[a * r + c];
                L[(long long)a * r + c] = Ls[a * r + c];
            }
}

// (L and U staged in shared memory first when they fit: the solves are
// chains of dependent steps, each of which would otherwise wait on L2)
__global__ void __launch_bounds__(32) lu_solve_kernel(const double *__restrict__ U, const double *__restrict__ L,
                                                      const int *__restrict__ perm, const double *__restrict__ Bt,
                                                      int r, double *__restrict__ X, int use_smem)
{
    __shared__ double x[256], rd[256];
    extern __shared__ double lus_smem[];
    const int c = blockIdx.x, lane = threadIdx.x;
    if (c >= r) return;
    for (int i = lane; i < r; i += 32) {                 // reciprocal pivots, off the solve's chain
        const double d = U[(long long)i * r + i];
        rd[i] = d == 0.0 ? 1.0 : 1.0 / d;
    }
    if (use_smem) {
        double *Us = lus_smem, *Lsm = lus_smem + (size_t)r * r;
        for (int q = lane; q < r * r; q += 32) {
            Us[q] = U[q];
            Lsm[q] = L[q];
        }
        __syncwarp();
        U = Us;
        L = Lsm;
    }
    for (int i = lane; i < r; i += 32) x[i] = Bt[(long long)i * r + c];
    __syncwarp();
    if (lane == 0)
        for (int j = 0; j < r; ++j) {
            const int pj = perm[j];
            if (pj != j) {
                const double v = x[j];
                x[j] = x[pj];
                x[pj] = v;
            }
        }
    __syncwarp();
    for (int i = 1; i < r; ++i) {                        // L y = P b (unit lower)
        double sacc = 0.0;
        for (int j = lane; j < i; j += 32) sacc += L[(long long)i * r + j] * x[j];
        sacc = warp_sum(sacc);
        if (lane == 0) x[i] -= sacc;
        __syncwarp();
    }
    for (int i = r - 1; i >= 0; --i) {                   // U x = y
        double sacc = 0.0;
        for (int j = i + 1 + lane; j < r; j += 32) sacc += U[(long long)i * r + j] * x[j];
        sacc = warp_sum(sacc);
        if (lane == 0) x[i] = (x[i] - sacc) * rd[i];
        __syncwarp();
    }
    for (int i = lane; i < r; i += 32) X[(long long)i * r + c] = x[i];
}

__global__ void gram_scale_kernel(double *__restrict__ G, int m, double *__restrict__ d)
{
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double g = G[(long long)i * m + i];
        d[i] = g > 0.0 ? 1.0 / sqrt(g) : 0.0;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < m * m; q += blockDim.x) G[q] *= d[q / m] * d[q % m];
}

// c [r][m] <- c D (undo the column scaling of the Gram matrix)
__global__ void colscale_kernel(double *__restrict__ c, int r, int m, const double *__restrict__ d)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < r * m; q += gridDim.x * blockDim.x) c[q] *= d[q % m];
}

// T <- (T + T^T) / 2 in place, r x r, one CTA
__global__ void sym_kernel(double *__restrict__ T, int r)
{
    for (int q = threadIdx.x; q < r * r; q += blockDim.x) {
        const int i = q / r, j = q - i * r;
        if (j <= i) continue;
        const double v = 0.5 * (T[(long long)i * r + j] + T[(long long)j * r + i]);
        T[(long long)i * r + j] = v;
        T[(long long)j * r + i] = v;
    }
}

// Eigenpairs of a symmetric r x r matrix T (FP32 block Jacobi), ordered by
// |lambda| descending: lam[rank] and coef [rank][r] = U^T (zero rows
// beyond r).  r <= 32 * 2 NJ.  work: >= eig_work_doubles(r) doubles (or shared memory).
__host__ __device__ inline size_t eig_work_doubles(int r)
{
    return (size_t)r * r + ((size_t)r + 2) * (r + 2) / 4 + 16;
}

template <int NJ>
__global__ void __launch_bounds__(1024, 1) eig_select_kernel(const double *__restrict__ T, int r, int rank, double *work,
                                                          double *__restrict__ lam, float *__restrict__ coef,
                                                          int *__restrict__ flag, int use_smem)
{
    extern __shared__ double smem_work[];
    if (use_smem) work = smem_work;
    const int t = threadIdx.x, nt = blockDim.x;
    float *A0 = reinterpret_cast<float *>(work);
    float *Uf = A0 + (long long)r * r;
    short *pairs = reinterpret_cast<short *>(Uf + (long long)r * r);   // (r + 1)^2 shorts
    // |T|_F in FP64 (a non-finite T gives non-finite eigenvalues: flag 4)
    __shared__ double s_f[32];
    double f = 0.0;
    for (int q = t; q < r * r; q += nt) f += T[q] * T[q];
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if ((t & 31) == 0) s_f[t >> 5] = f;
    __syncthreads();
    f = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) f += s_f[w];
    const double fro = sqrt(f), sc = fro > 0.0 ? 1.0 / fro : 1.0;
    for (int q = t; q < r * r; q += nt) {
        A0[q] = (float)(T[q] * sc);
        Uf[q] = (q / r == q % r) ? 1.f : 0.f;
    }
    block_jacobi<NJ>(A0, Uf, r, pairs, 40);
    select_eigenpairs(A0, Uf, r, rank, fro > 0.0 ? fro : 1.0, lam, coef, flag);
}

__global__ void std_kernel(const float *__restrict__ V, long long ldv, const double *__restrict__ lam, int rank,
                           const float *__restrict__ B0, long long n, float eps, float *__restrict__ out)
{
    __shared__ float sl[256];
    for (int r = threadIdx.x; r < rank; r += blockDim.x) sl[r] = (float)lam[r];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float s = B0[i];
        for (int r = 0; r < rank; ++r) {
            float v = V[(long long)r * ldv + i];
            s = fmaf(sl[r] * v, v, s);
        }
        out[i] = sqrtf(eps * fmaxf(s, 0.f));
    }
}

// Philox4x32-10 (Salmon et al. 2011) + Box-Muller on 24-bit uniforms
__device__ __forceinline__ void philox10(unsigned c[4], unsigned k0, unsigned k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        unsigned hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        unsigned n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// element e = row * n + col of the [p][n] probe block (the counter is e / 4)
// is stored at X[row * ld + col]
__global__ void philox_normal_kernel(float *__restrict__ X, long long total, long long n, long long ld,
                                     unsigned long long seed)
{
    const float two_pi = 6.28318530717958647692f;
    const bool small = total + 4 < (1LL << 32);
    for (long long blk = blockIdx.x * (long long)blockDim.x + threadIdx.x; blk * 4 < total;
         blk += (long long)gridDim.x * blockDim.x) {
        unsigned c[4] = {(unsigned)(blk & 0xFFFFFFFFull), (unsigned)(blk >> 32), 0u, 0u};
        philox10(c, (unsigned)(seed & 0xFFFFFFFFull), (unsigned)(seed >> 32));
        // row and column of the first of the four elements, one division per
        // counter (32-bit when the block fits), then stepped along the row
        long long row, col;
        if (small) {
            const unsigned e0 = (unsigned)(blk * 4), nn = (unsigned)n;
            row = e0 / nn;
            col = e0 - (unsigned)row * nn;
        } else {
            row = (blk * 4) / n;
            col = blk * 4 - row * n;
        }
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
            float u1 = ((float)(c[2 * pr] >> 8) + 1.0f) * (1.0f / 16777216.0f);
            float u2 = (float)(c[2 * pr + 1] >> 8) * (1.0f / 16777216.0f);
            float rad = sqrtf(-2.0f * logf(u1));
            float sn, cn;
            sincosf(two_pi * u2, &sn, &cn);
            long long e = blk * 4 + 2 * pr;
            if (e < total) X[row * ld + col] = rad * cn;
            if (++col == n) { col = 0; ++row; }
            if (e + 1 < total) X[row * ld + col] = rad * sn;
            if (++col == n) { col = 0; ++row; }
        }
    }
}

// after the store's work has completed: GBFWI_ETIMEOUT (and the flag
// cleared) when a product kernel's bounded wait gave up since the last check
int take_status(gbfwi_bfgs *h)
{
    int st = 0;
    GB_CUDA(cudaMemcpy(&st, h->status.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) {
        GB_CUDA(cudaMemset(h->status.p, 0, sizeof(int)));
        return GBFWI_ETIMEOUT;
    }
    return GBFWI_OK;
}

int grid_n(long long n) { return (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 152 * 8); }

// splits of the one- and two-column products
long long thin_splits(long long n) { return std::min<long long>(304, std::max<long long>(1, (n + 4095) / 4096)); }

// FP64 split-K partials an (ka x kb) product of this store takes
size_t part_need(const gbfwi_bfgs *h, int ka, int kb)
{
    if (ka < 1 || kb < 1) return 0;
    if (kb <= 2) return (size_t)thin_splits(h->n) * ka * kb;
    const long long ns = gb_tc_atb_splits(ka, kb, h->n);
    return ns < 1 ? 0 : (size_t)ns * ka * kb;
}

// out[a][b] = sum_i A_a[i] B_b[i] -> out (device FP64, row stride ldo); the
// A rows a < ka1 come from A1, the rest from A2 (likewise B).  Rows have the
// store's pitch.  One or two columns from a single B block: compensated
// CUDA-core dot products; otherwise the tcgen05 product (gb_tc_atb).
int atb(gbfwi_bfgs *h, const float *A1, const float *A2, int ka1, int ka, const float *B1, const float *B2, int kb1,
        int kb, double *out, long long ldo, cudaStream_t s)
{
    if (ka == 0 || kb == 0) return GBFWI_OK;
    const long long n = h->n, ld = h->ld;
    if (kb <= 2 && kb1 >= kb) {
        const long long nsplit = thin_splits(n);
        const long long chunk = (n + nsplit - 1) / nsplit;
        const long long ns = (n + chunk - 1) / chunk;
        for (int blk = 0; blk < 2; ++blk) {
            const float *A = blk == 0 ? A1 : A2;
            const int kab = blk == 0 ? std::min(ka1, ka) : ka - ka1;
            if (kab <= 0) continue;
            if ((size_t)ns * kab * kb > h->part.bytes / sizeof(double)) return GBFWI_EINVAL;
            dim3 tg((unsigned)ns, (unsigned)kab);
            if (kb == 1)
                atb_thin<1><<<tg, 256, 0, s>>>(A, ld, B1, ld, nullptr, n, chunk, kab, h->part.as<double>());
            else
                atb_thin<2><<<tg, 256, 0, s>>>(A, ld, B1, ld, nullptr, n, chunk, kab, h->part.as<double>());
            GB_LAUNCHED();
            const int nab = kab * kb;
            atb_reduce<<<(nab + 255) / 256, 256, 0, s>>>(h->part.as<double>(), (int)ns, nab,
                                                         out + (blk == 0 ? 0 : (long long)ka1 * ldo), ldo, kb);
            GB_LAUNCHED();
        }
        return GBFWI_OK;
    }
    return gb_tc_atb(A1, A2, ka1, ka, B1, B2, kb1, kb, ld, n, h->part.as<double>(), h->part.bytes / sizeof(double),
                     out, ldo, h->status.as<int>(), s);
}

// out[c] = sum_a coef[c][a] row_a + beta * dw * Xc[c], c < nc; rows a < k1
// from A1, the rest from A2 (pitch ld); out and Xc with their own pitches
int combine(gbfwi_bfgs *h, const float *A1, const float *A2, int k1, int ktot, const float *coef, int nc,
            float *out, long long ldo, const float *dw, const float *Xc, long long ldx, float beta, cudaStream_t s)
{
    const long long n = h->n, ld = h->ld;
    if (ktot >= 1 && ktot <= 128)
        return gb_tc_combine(A1, A2, k1, ktot, ld, coef, nc, n, out, ldo, dw, Xc, ldx, beta, h->status.as<int>(), s);
    // no rows (out = beta dw Xc) or more than 128: CUDA-core combination
    for (int c0 = 0; c0 < nc; c0 += 64) {
        int cn = std::min(64, nc - c0);
        size_t smem = (size_t)std::max(ktot, 1) * 64 * sizeof(float);
        if (smem > 48 * 1024)
            GB_CUDA(cudaFuncSetAttribute(combine_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        combine_kernel<64><<<grid_n(n) / 2 + 1, 128, smem, s>>>(A1, A2, k1, ktot, ld, coef, c0, cn, n, out, ldo, dw,
                                                              Xc, ldx, beta);
        GB_LAUNCHED();
    }
    return GBFWI_OK;
}

// Copy a caller's [rows][n] block (host or device, contiguous rows) into a
// store buffer with the store's pitch.
int stage_rows(gbfwi_bfgs *h, DevBuf &buf, const float *user, int rows, cudaStream_t s)
{
    GB_TRY(buf.ensure((size_t)rows * h->ld * sizeof(float)));
    GB_CUDA(cudaMemcpy2DAsync(buf.p, h->ld * sizeof(float), user, h->n * sizeof(float), h->n * sizeof(float), rows,
                              cudaMemcpyDefault, s));
    return GBFWI_OK;
}

// Copy rows of a store buffer (pitch ld) out to a caller's contiguous block
int unstage_rows(gbfwi_bfgs *h, float *user, const float *dev, int rows, cudaStream_t s)
{
    GB_CUDA(cudaMemcpy2DAsync(user, h->n * sizeof(float), dev, h->ld * sizeof(float), h->n * sizeof(float), rows,
                              cudaMemcpyDefault, s));
    return GBFWI_OK;
}

// FP64 scratch of apply_dev (T = [S; B0 Y] X^T), placed first in `small`
size_t small_apply_doubles(const gbfwi_bfgs *h, int p) { return (size_t)2 * std::max(h->k, 1) * p + 64; }

// coef / coefd [q][2k] = (M T)^T for the q columns of T [2k][q] (middle_kernel)
int launch_middle(gbfwi_bfgs *h, const double *T, int q, double gamma, float *coef, double *coefd, cudaStream_t s)
{
    const int k = h->k;
    const int mats = middle_smem_bytes(k, true) <= 200 * 1024;
    const size_t bytes = middle_smem_bytes(k, mats);
    auto kern = k <= 32 ? middle_col_kernel<1> : k <= 64 ? middle_col_kernel<2> : k <= 128 ? middle_col_kernel<4>
                                                                                       : middle_kernel;
    if (bytes > 48 * 1024)
        GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    kern<<<q, 32, bytes, s>>>(T, h->dSY.as<double>(), h->dYBY.as<double>(), k, h->kmax, q, gamma, mats, coef, coefd);
    GB_LAUNCHED();
    return GBFWI_OK;
}

// Size the scratch buffers once per call so that nothing is reallocated
// while kernels queued earlier in the same call may still use it.
// shapes: the (ka, kb) of every product the call makes.
int reserve(gbfwi_bfgs *h, int p, bool lowrank, std::initializer_list<std::pair<int, int>> shapes)
{
    size_t part = 16;
    for (const auto &sh : shapes) part = std::max(part, part_need(h, sh.first, sh.second));
    GB_TRY(h->part.ensure(part * sizeof(double)));
    size_t pp = (size_t)p * p;
    size_t sm = small_apply_doubles(h, p) + (lowrank ? pp * 12 + 8 * (size_t)p + 64 : 0);
    sm = std::max(sm, (size_t)(4 * (h->k + 1) + 8));
    GB_TRY(h->small.ensure(sm * sizeof(double)));
    GB_TRY(h->coef.ensure(std::max<size_t>({pp, (size_t)p * 2 * std::max(h->k, 1), 16}) * sizeof(float)));
    return GBFWI_OK;
}

// Z = (H - minus_B0 gamma B0) X for X [p] rows of pitch ldx into Z (pitch
// ldz).  For p >= 3 the rows of X must be 16-byte aligned with ldx a
// multiple of 4 (a store buffer).
int apply_dev(gbfwi_bfgs *h, const float *Xd, long long ldx, int p, float *Zd, long long ldz, double gamma,
              int minus_B0, cudaStream_t s)
{
    const int k = h->k;
    float beta = minus_B0 ? 0.f : (float)gamma;
    if (k == 0) {
        if (beta == 0.f) {
            GB_CUDA(cudaMemset2DAsync(Zd, ldz * sizeof(float), 0, h->n * sizeof(float), p, s));
            return GBFWI_OK;
        }
        return combine(h, nullptr, nullptr, 0, 0, nullptr, p, Zd, ldz, h->B0.as<float>(), Xd, ldx, beta, s);
    }
    double *T = h->small.as<double>();
    // T = [S; B0 Y] X^T: rows 0..k-1 S^T x_c, rows k..2k-1 (B0 Y)^T x_c, one pass over X
    if (p <= 2 && ldx != h->ld) {
        // a caller's one or two vectors with their own pitch: thin products
        const long long n = h->n;
        const long long nsplit = thin_splits(n);
        const long long chunk = (n + nsplit - 1) / nsplit;
        const long long ns = (n + chunk - 1) / chunk;
        for (int blk = 0; blk < 2; ++blk) {
            const float *A = blk == 0 ? h->S.as<float>() : h->BY.as<float>();
            dim3 tg((unsigned)ns, (unsigned)k);
            if (p == 1)
                atb_thin<1><<<tg, 256, 0, s>>>(A, h->ld, Xd, ldx, nullptr, n, chunk, k, h->part.as<double>());
            else
                atb_thin<2><<<tg, 256, 0, s>>>(A, h->ld, Xd, ldx, nullptr, n, chunk, k, h->part.as<double>());
            GB_LAUNCHED();
            atb_reduce<<<(k * p + 255) / 256, 256, 0, s>>>(h->part.as<double>(), (int)ns, k * p,
                                                           T + (long long)blk * k * p, p, p);
            GB_LAUNCHED();
        }
    } else {
        GB_TRY(atb(h, h->S.as<float>(), h->BY.as<float>(), k, 2 * k, Xd, nullptr, p, p, T, p, s));
    }
    GB_TRY(launch_middle(h, T, p, gamma, h->coef.as<float>(), nullptr, s));
    return combine(h, h->S.as<float>(), h->BY.as<float>(), k, 2 * k, h->coef.as<float>(), p, Zd, ldz,
                   h->B0.as<float>(), Xd, ldx, beta, s);
}

}  // namespace

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------

extern "C" int gbfwi_bfgs_create(long long n, int kmax, const float *B0, gbfwi_bfgs **out)
{
    if (n < 1 || kmax < 1 || kmax > 4096 || !B0 || !out) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(B0));
    gbfwi_bfgs *h = new (std::nothrow) gbfwi_bfgs();
    if (!h) return GBFWI_ENOMEM;
    h->n = n;
    h->ld = (n + 63) / 64 * 64;
    h->kmax = kmax;
    const size_t store = (size_t)kmax * h->ld * sizeof(float);
    int rc = h->S.ensure(store);
    if (!rc) rc = h->Y.ensure(store);
    if (!rc) rc = h->BY.ensure(store);
    if (!rc) rc = h->B0.ensure((size_t)n * sizeof(float));
    if (!rc) rc = h->dSY.ensure((size_t)kmax * kmax * sizeof(double));
    if (!rc) rc = h->dYBY.ensure((size_t)kmax * kmax * sizeof(double));
    if (!rc) rc = h->flag.ensure(16);
    if (!rc) rc = h->status.ensure(16);
    if (rc) { delete h; return rc; }
    h->SY.assign((size_t)kmax * kmax, 0.0);
    h->YBY.assign((size_t)kmax * kmax, 0.0);
    h->SS.assign((size_t)kmax * kmax, 0.0);
    h->SB.assign((size_t)kmax * kmax, 0.0);
    h->BB.assign((size_t)kmax * kmax, 0.0);
    // the row padding stays zero
    if (cudaMemset(h->S.p, 0, store) != cudaSuccess || cudaMemset(h->Y.p, 0, store) != cudaSuccess ||
        cudaMemset(h->BY.p, 0, store) != cudaSuccess || cudaMemset(h->status.p, 0, 16) != cudaSuccess ||
        cudaMemcpy(h->B0.p, B0, (size_t)n * sizeof(float), cudaMemcpyDefault) != cudaSuccess) {
        gb_set_last_cuda_error(cudaGetLastError(), "initialise the BFGS store", __FILE__, __LINE__);
        delete h;
        return GBFWI_ECUDA;
    }
    *out = h;
    return GBFWI_OK;
}

extern "C" int gbfwi_bfgs_destroy(gbfwi_bfgs *h)
{
    delete h;
    return GBFWI_OK;
}

extern "C" int gbfwi_bfgs_count(const gbfwi_bfgs *h) { return h ? h->k : GBFWI_EINVAL; }

extern "C" int gbfwi_bfgs_update(gbfwi_bfgs *h, const float *s_, const float *y_, void *stream)
{
    if (!h || !s_ || !y_) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(s_, y_));
    if (h->k >= h->kmax) return GBFWI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = h->n, ld = h->ld;
    const int k = h->k;
    float *sk = h->S.as<float>() + (long long)k * ld;
    float *yk = h->Y.as<float>() + (long long)k * ld;
    float *byk = h->BY.as<float>() + (long long)k * ld;
    GB_CUDA(cudaMemcpyAsync(sk, s_, n * sizeof(float), cudaMemcpyDefault, s));
    GB_CUDA(cudaMemcpyAsync(yk, y_, n * sizeof(float), cudaMemcpyDefault, s));
    mul_kernel<<<grid_n(n), 256, 0, s>>>(h->B0.as<float>(), yk, n, byk);
    GB_LAUNCHED();
    // dots of the new pair with the store: rows [S_0..S_k, B0Y_0..B0Y_k]
    // against (y_k, s_k, B0 y_k), and y_k^T y_k; they extend S^T Y, Y^T B0 Y
    // and the Gram matrix W^T W of W = [S, B0 Y]
    const int k1 = k + 1;
    const long long nsplit = thin_splits(n);
    const long long chunk = (n + nsplit - 1) / nsplit;
    const long long ns = (n + chunk - 1) / chunk;
    GB_TRY(reserve(h, 1, false, {{k1, 1}}));
    GB_TRY(h->part.ensure(std::max(h->part.bytes, (size_t)ns * 6 * k1 * sizeof(double))));
    GB_TRY(h->small.ensure(std::max(h->small.bytes, (size_t)(6 * k1 + 8) * sizeof(double))));
    double *d1 = h->small.as<double>();          // [2 k1][3]
    double *d3 = d1 + 6 * k1;                    // [1]
    const float *S = h->S.as<float>(), *BY = h->BY.as<float>();
    pair_dots_kernel<<<dim3((unsigned)ns, (unsigned)(2 * k1)), 256, 0, s>>>(S, BY, ld, k1, yk, sk, byk, n, chunk,
                                                                          h->part.as<double>());
    GB_LAUNCHED();
    atb_reduce<<<(6 * k1 + 255) / 256, 256, 0, s>>>(h->part.as<double>(), (int)ns, 6 * k1, d1, 3, 3);
    GB_LAUNCHED();
    GB_TRY(atb(h, yk, nullptr, 1, 1, yk, nullptr, 1, 1, d3, 1, s));
    std::vector<double> hd(6 * k1 + 1);
    GB_CUDA(cudaMemcpyAsync(hd.data(), d1, hd.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    // hd[3 a + b]: a < k1 row s_a, a >= k1 row B0 y_(a - k1); b: y_k, s_k, B0 y_k
    double ys = hd[3 * k], ss = hd[3 * k + 1], yy = hd[6 * k1];
    if (!std::isfinite(ys) || !std::isfinite(ss) || !std::isfinite(yy)) return gb_nonfinite("BFGS pair dot product");
    if (!(ys > 1e-12 * std::sqrt(ss) * std::sqrt(yy))) return GBFWI_ECURV;
    for (double v : hd)
        if (!std::isfinite(v)) return gb_nonfinite("BFGS pair dot product");
    const int km = h->kmax;
    auto at = [km](std::vector<double> &A, int i, int j) -> double & { return A[(size_t)i * km + j]; };
    for (int i = 0; i <= k; ++i) {
        const double *sr = &hd[3 * i], *br = &hd[3 * (k1 + i)];
        at(h->SY, i, k) = sr[0];
        at(h->YBY, i, k) = at(h->YBY, k, i) = br[0];
        at(h->SS, i, k) = at(h->SS, k, i) = sr[1];
        at(h->SB, i, k) = sr[2];                     // s_i^T B0 y_k
        if (i < k) at(h->SB, k, i) = br[1];          // s_k^T B0 y_i
        at(h->BB, i, k) = at(h->BB, k, i) = br[2];
    }
    GB_CUDA(cudaMemcpyAsync(h->dSY.p, h->SY.data(), h->SY.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaMemcpyAsync(h->dYBY.p, h->YBY.data(), h->YBY.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    // W^T W for the k1 pairs: [[S^T S, S^T B0 Y], [(S^T B0 Y)^T, (B0 Y)^T B0 Y]]
    const int m1 = 2 * k1;
    std::vector<double> Gm((size_t)m1 * m1);
    for (int a = 0; a < k1; ++a)
        for (int b = 0; b < k1; ++b) {
            Gm[(size_t)a * m1 + b] = at(h->SS, a, b);
            Gm[(size_t)a * m1 + k1 + b] = at(h->SB, a, b);
            Gm[(size_t)(k1 + b) * m1 + a] = at(h->SB, a, b);
            Gm[(size_t)(k1 + a) * m1 + k1 + b] = at(h->BB, a, b);
        }
    GB_TRY(h->dG.ensure(Gm.size() * sizeof(double)));
    GB_CUDA(cudaMemcpyAsync(h->dG.p, Gm.data(), Gm.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    GB_CUDA(cudaStreamSynchronize(s));
    h->k = k + 1;
    return GBFWI_OK;
}

extern "C" int gbfwi_bfgs_apply(gbfwi_bfgs *h, const float *X, int p, float *Z, double gamma, int minus_B0,
                                void *stream)
{
    if (!h || !X || !Z || p < 1 || p > 256 || !(gamma > 0)) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(X, Z));
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = h->n, ld = h->ld;
    const int k = h->k;
    GB_TRY(reserve(h, p, false, {{2 * k, p}, {k, p}}));
    const float *Xd = X;
    long long ldx = n;
    if (p >= 3 || !gb_is_device_ptr(X)) {
        // a block goes to the tensor cores from a store buffer (aligned rows)
        GB_TRY(stage_rows(h, h->X, X, p, s));
        Xd = h->X.as<float>();
        ldx = ld;
    }
    const bool dev_out = gb_is_device_ptr(Z);
    float *Zd = Z;
    long long ldz = n;
    if (!dev_out) {
        GB_TRY(h->E.ensure((size_t)p * ld * sizeof(float)));
        Zd = h->E.as<float>();
        ldz = ld;
    }
    GB_TRY(apply_dev(h, Xd, ldx, p, Zd, ldz, gamma, minus_B0, s));
    if (!dev_out) {
        GB_TRY(unstage_rows(h, Z, Zd, p, s));
        GB_CUDA(cudaStreamSynchronize(s));
        GB_TRY(take_status(h));
    }
    return GBFWI_OK;
}

namespace {

// Sequential carve-up of the FP64 scratch of a decomposition
struct Arena {
    double *base;
    size_t off = 0;
    double *take(size_t n)
    {
        double *q = base + off;
        off += (n + 7) / 8 * 8;          // keep every piece 64-byte aligned
        return q;
    }
};

// FP64 scratch doubles of a decomposition with p probes (or basis rows) and m = 2k
size_t lowrank_doubles(int p, int m)
{
    const size_t P = (size_t)std::max(p, m), pm = P * (size_t)m, pp = P * P;
    return 12 * pm + 20 * pp + (size_t)m * m + 16 * P + 1024;
}

// out (M x N, row stride ldo) = A(i, l) B(l, j) over K, see small_gemm_kernel
template <typename TA>
int gemm(int M, int N, int K, const TA *A, long long ar, long long ac, const double *B, long long br, long long bc,
         double *out, float *outf, long long ldo, cudaStream_t s)
{
    if (M < 1 || N < 1) return GBFWI_OK;
    small_gemm_kernel<TA><<<dim3((unsigned)((N + 31) / 32), (unsigned)M), 32, 0, s>>>(M, N, K, A, ar, ac, B, br, bc,
                                                                                    out, outf, ldo);
    GB_LAUNCHED();
    return GBFWI_OK;
}

int launch_pivchol(const double *G, int p, double tol, double *work, double *coef, int *r_out, int *flag,
                   cudaStream_t s)
{
    const size_t ws = (3 * (size_t)p * p + 2 * (size_t)p) * sizeof(double);
    const int use_smem = ws <= 200 * 1024;
    if (use_smem)
        GB_CUDA(cudaFuncSetAttribute(gram_pivchol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws));
    gram_pivchol_kernel<<<1, 512, use_smem ? ws : 0, s>>>(G, p, tol, work, coef, r_out, flag, use_smem);
    GB_LAUNCHED();
    return GBFWI_OK;
}

int launch_eig(const double *T, int r, int rank, double *work, double *lam, float *coef, int *flag, cudaStream_t s)
{
    const size_t we = eig_work_doubles(r) * sizeof(double);
    const int use_smem = we <= 200 * 1024;
    const int npair = (r + 1) / 2;
    auto kern = npair <= 32 ? eig_select_kernel<1> : npair <= 64 ? eig_select_kernel<2> : eig_select_kernel<4>;
    if (use_smem) GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)we));
    kern<<<1, 1024, use_smem ? we : 0, s>>>(T, r, rank, work, lam, coef, flag, use_smem);
    GB_LAUNCHED();
    return GBFWI_OK;
}

// Every block of the decompositions lies in the span of the rows of W =
// [S, B0 Y] (m = 2k rows): E = (B - B0) X = C W with C = (M W^T X)^T, M the
// middle matrix of the compact form (gamma = 1), and so does every basis
// built from E.  The decompositions therefore carry their bases as FP64
// coordinates T ([r][m], basis = T W) and form every Gram matrix and
// projection from G = W^T W (kept by the update), W^T X and M in FP64:
//   E E^T = C G C^T,  Q Q^T = T G T^T,  Q E^T = T G C^T,  Q X^T = T (W^T X),
//   Q (B - B0) Q^T = (G T^T)^T M (G T^T).
// The n-long work is the one product W^T X and the final combination
// V = (U^T T) W; the FP32 rounding of E, of the basis and of its
// re-orthogonalisations never happens.
//
// The orthonormal basis of a block with coordinates Cb ([q][m]) and Gram
// matrix Gb = Cb G Cb^T: rank-revealing pivoted Cholesky of Gb (rows kept
// while their residual norm is >= tol of the largest), T1 = coef1 Cb, then
// one CholeskyQR pass in FP64 (pivoted Cholesky of T1 G T1^T with tol 0),
// Tq = coef2 T1.  Returns r through *r_host after one synchronisation;
// r_dev[1] holds the second pass's count (equal to r unless that Gram
// matrix lost definiteness, checked at the end).
int basis_coords(gbfwi_bfgs *h, const double *Gb, const double *Cb, int q, int m, double tol, const double *colscale,
                 Arena &ar, double *&Tq, int &r, int *r_dev, int *flag, cudaStream_t s)
{
    const double *G = h->dG.as<double>();
    const size_t P = (size_t)std::max(q, m);
    double *work = ar.take(3 * P * P + 2 * P);
    double *c1 = ar.take(P * P), *c2 = ar.take(P * P), *Gq = ar.take(P * P);
    double *T1 = ar.take(P * m), *P2 = ar.take(P * m);
    Tq = ar.take(P * m);
    GB_TRY(launch_pivchol(Gb, q, tol, work, c1, r_dev, flag, s));
    GB_CUDA(cudaMemcpyAsync(&r, r_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    GB_TRY(take_status(h));
    if (r < 1) return GBFWI_OK;
    if (colscale) {
        // Cb = D (identity coordinates, scaled Gram matrix): T1 = coef1 D
        GB_CUDA(cudaMemcpyAsync(T1, c1, (size_t)r * m * sizeof(double), cudaMemcpyDeviceToDevice, s));
        colscale_kernel<<<std::max(1, (r * m + 255) / 256), 256, 0, s>>>(T1, r, m, colscale);
        GB_LAUNCHED();
    } else {
        GB_TRY(gemm(r, m, q, c1, q, 1, Cb, m, 1, T1, nullptr, m, s));          // T1 = coef1 Cb
    }
    GB_TRY(gemm(r, m, m, T1, m, 1, G, m, 1, P2, nullptr, m, s));               // P2 = T1 G
    GB_TRY(gemm(r, r, m, P2, m, 1, T1, 1, m, Gq, nullptr, r, s));              // Gq = P2 T1^T
    GB_TRY(launch_pivchol(Gq, r, 0.0, work, c2, r_dev + 1, flag, s));
    GB_TRY(gemm(r, m, r, c2, r, 1, T1, m, 1, Tq, nullptr, m, s));              // Tq = coef2 T1
    return GBFWI_OK;
}

// The Rayleigh-Ritz matrix of the basis Tq W, Q (B - B0) Q^T = Y^T M Y with
// Y = G Tq^T ([m][r]), symmetrised into Cm [r][r]
int rayleigh_ritz(gbfwi_bfgs *h, const double *Tq, int r, int m, Arena &ar, double *Cm, cudaStream_t s)
{
    const double *G = h->dG.as<double>();
    double *Yc = ar.take((size_t)m * r), *CdY = ar.take((size_t)r * m);
    GB_TRY(gemm(m, r, m, G, m, 1, Tq, 1, m, Yc, nullptr, r, s));               // Y = G Tq^T
    GB_TRY(launch_middle(h, Yc, r, 1.0, nullptr, CdY, s));                      // (M Y)^T
    GB_TRY(gemm(r, r, m, CdY, m, 1, Yc, r, 1, Cm, nullptr, r, s));             // Y^T M Y
    sym_kernel<<<1, 256, 0, s>>>(Cm, r);
    GB_LAUNCHED();
    return GBFWI_OK;
}

// V = (U^T Tq) W for the first `rank` eigenvectors (coef = U^T, [rank][r];
// rows beyond r are zero), then the posterior std (Eq. 14) and the copies out
int finish_lowrank(gbfwi_bfgs *h, const double *Tq, int r, int rank, const double *lam, double eps_prior, float *V,
                   double *lambda, float *std_out, Arena &ar, const int *flag, const int *r_dev, cudaStream_t s)
{
    const long long n = h->n, ld = h->ld;
    const int k = h->k, m = 2 * k;
    float *F = reinterpret_cast<float *>(ar.take(((size_t)rank * m + 1) / 2));
    GB_TRY(gemm(rank, m, r, h->coef.as<float>(), r, 1, Tq, m, 1, (double *)nullptr, F, m, s));
    GB_TRY(h->E.ensure((size_t)std::max(rank, 1) * ld * sizeof(float)));
    GB_TRY(h->Q.ensure((size_t)ld * sizeof(float)));
    const bool devV = V && gb_is_device_ptr(V);
    float *Vd = devV ? V : h->E.as<float>();
    const long long ldv = devV ? n : ld;
    GB_TRY(combine(h, h->S.as<float>(), h->BY.as<float>(), k, m, F, rank, Vd, ldv, nullptr, nullptr, 0, 0.f, s));
    if (std_out) {
        const bool devS = gb_is_device_ptr(std_out);
        float *Sd = devS ? std_out : h->Q.as<float>();
        std_kernel<<<grid_n(n), 256, 0, s>>>(Vd, ldv, lam, rank, h->B0.as<float>(), n, (float)eps_prior, Sd);
        GB_LAUNCHED();
        if (!devS) GB_CUDA(cudaMemcpyAsync(std_out, Sd, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    if (V && !devV) GB_TRY(unstage_rows(h, V, Vd, rank, s));
    if (lambda)
        GB_CUDA(cudaMemcpyAsync(lambda, lam, rank * sizeof(double),
                                gb_is_device_ptr(lambda) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    int fl[3] = {0, 0, 0};
    GB_CUDA(cudaMemcpyAsync(fl, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(fl + 1, r_dev + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    GB_TRY(take_status(h));
    int flag_h = fl[0];
    if (!flag_h && fl[1] != r) flag_h = 2;            // the CholeskyQR pass lost a row
    if (flag_h) {
        static const char *stage[] = {"", "Gram matrix of the block", "Cholesky pivot of the basis Gram matrix",
                                      "singular Q^T X", "eigenvalues of the projected matrix"};
        return gb_nonfinite(stage[flag_h >= 1 && flag_h <= 4 ? flag_h : 0]);
    }
    return GBFWI_OK;
}

// The randomized eigendecomposition of B_{n+1} - B0 (Algorithm 3): probes
// X (given, or Philox normals), E = (B - B0) X, a rank-revealing orthonormal
// basis Q of E's rows; then either the single pass of Algorithm 3 (Omega
// from Omega (Q^T X) = Q^T E) or, two_pass, the Rayleigh-Ritz second pass
// C = Q (B - B0) Q^T.  Eigenpairs, V = U^T Q and the posterior std follow.
// All of it in the coordinates of W = [S, B0 Y] (see basis_coords).
int lowrank_randomized(gbfwi_bfgs *h, const float *X, int p, int rank, unsigned long long seed, double eps_prior,
                       float *V, double *lambda, float *std_out, bool two_pass, cudaStream_t s)
{
    const long long n = h->n, ld = h->ld;
    const int k = h->k, m = 2 * k;
    if (k < 1) return gb_nonfinite("probe block E = (B - B0) X is zero or not finite");
    // the probe block in a store buffer (aligned rows for the tensor cores)
    if (X) {
        GB_TRY(stage_rows(h, h->X, X, p, s));
    } else {
        GB_TRY(h->X.ensure((size_t)p * ld * sizeof(float)));
        philox_normal_kernel<<<grid_n((p * n + 3) / 4), 256, 0, s>>>(h->X.as<float>(), (long long)p * n, n, ld, seed);
        GB_LAUNCHED();
    }
    const float *Xd = h->X.as<float>();
    GB_TRY(reserve(h, p, false, {{m, p}}));
    GB_TRY(h->ex.ensure(lowrank_doubles(p, m) * sizeof(double)));
    Arena ar{h->ex.as<double>()};
    const size_t pm = (size_t)p * m, pp = (size_t)p * p;
    double *Z = ar.take(pm), *Cd = ar.take(pm), *Pm = ar.take(pm), *Ge = ar.take(pp);
    double *lam = ar.take((size_t)p + 2);
    int *rdev = reinterpret_cast<int *>(ar.take(2));
    int *flag = h->flag.as<int>();
    const double *G = h->dG.as<double>();
    GB_CUDA(cudaMemsetAsync(flag, 0, 16, s));
    // 1. Z = W^T X (one pass over S, B0 Y and X), C = (M Z)^T: E = C W
    GB_TRY(atb(h, h->S.as<float>(), h->BY.as<float>(), k, m, Xd, nullptr, p, p, Z, p, s));
    GB_TRY(launch_middle(h, Z, p, 1.0, nullptr, Cd, s));
    // 2. E E^T = C G C^T, the basis coordinates Tq
    GB_TRY(gemm(p, m, m, Cd, m, 1, G, m, 1, Pm, nullptr, m, s));               // P = C G
    GB_TRY(gemm(p, p, m, Pm, m, 1, Cd, 1, m, Ge, nullptr, p, s));              // E E^T = P C^T
    double *Tq = nullptr;
    int r = 0;
    GB_TRY(basis_coords(h, Ge, Cd, p, m, 1e-4, nullptr, ar, Tq, r, rdev, flag, s));
    if (r < 1) return gb_nonfinite("probe block E = (B - B0) X is zero or not finite");
    double *work = ar.take(4 * pp + 4 * (size_t)p);
    double *Om = ar.take(pp);
    if (!two_pass) {
        // 3. [Q^T E, Q^T X] (Q E^T = Tq P^T, Q X^T = Tq Z), Omega by least squares
        double *QEX = ar.take(2 * pp), *A = ar.take(pp), *Bm = ar.take(pp), *R2 = ar.take(pp);
        GB_TRY(gemm(r, p, m, Tq, m, 1, Pm, 1, m, QEX, nullptr, 2 * p, s));
        GB_TRY(gemm(r, p, m, Tq, m, 1, Z, p, 1, QEX + p, nullptr, 2 * p, s));
        int *perm = reinterpret_cast<int *>(work + pp);
        omega_system_kernel<<<r, 32, 0, s>>>(QEX, QEX + p, 2 * p, r, p, A, Bm);
        GB_LAUNCHED();
        const size_t wl = (size_t)2 * r * r * sizeof(double);
        const int lu_smem = wl <= 200 * 1024;
        if (lu_smem) GB_CUDA(cudaFuncSetAttribute(lu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wl));
        lu_kernel<<<1, 512, lu_smem ? wl : 0, s>>>(A, R2, perm, r, flag, lu_smem);
        GB_LAUNCHED();
        if (lu_smem) GB_CUDA(cudaFuncSetAttribute(lu_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wl));
        lu_solve_kernel<<<r, 32, lu_smem ? wl : 0, s>>>(A, R2, perm, Bm, r, Om, lu_smem);
        GB_LAUNCHED();
        sym_kernel<<<1, 512, 0, s>>>(Om, r);
        GB_LAUNCHED();
    } else {
        // 3. second pass: the Rayleigh-Ritz matrix Q (B - B0) Q^T
        GB_TRY(rayleigh_ritz(h, Tq, r, m, ar, Om, s));
    }
    GB_TRY(launch_eig(Om, r, rank, work, lam, h->coef.as<float>(), flag, s));
    return finish_lowrank(h, Tq, r, rank, lam, eps_prior, V, lambda, std_out, ar, flag, rdev, s);
}

}  // namespace

extern "C" int gbfwi_lowrank_invhess(gbfwi_bfgs *h, const float *X, int p, int rank, unsigned long long seed,
                                     double eps_prior, float *V, double *lambda, float *std_out, void *stream)
{
    if (!h || p < 1 || p > 256 || rank < 1 || rank > p || !(eps_prior > 0)) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(X, V, lambda, std_out));
    return lowrank_randomized(h, X, p, rank, seed, eps_prior, V, lambda, std_out, false, (cudaStream_t)stream);
}

extern "C" int gbfwi_lowrank_twopass(gbfwi_bfgs *h, const float *X, int p, int rank, unsigned long long seed,
                                     double eps_prior, float *V, double *lambda, float *std_out, void *stream)
{
    if (!h || p < 1 || p > 256 || rank < 1 || rank > p || !(eps_prior > 0)) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(X, V, lambda, std_out));
    return lowrank_randomized(h, X, p, rank, seed, eps_prior, V, lambda, std_out, true, (cudaStream_t)stream);
}

extern "C" int gbfwi_lowrank_exact(gbfwi_bfgs *h, int rank, double eps_prior, float *V, double *lambda,
                                   float *std_out, void *stream)
{
    if (!h || !(eps_prior > 0)) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(V, lambda, std_out));
    const int k = h->k;
    if (k < 1 || k > 128) return GBFWI_EINVAL;
    const int m = 2 * k;
    if (rank < 1 || rank > m) return GBFWI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t mm = (size_t)m * m;
    GB_TRY(reserve(h, m, false, {}));
    GB_TRY(h->ex.ensure(lowrank_doubles(m, m) * sizeof(double)));
    Arena ar{h->ex.as<double>()};
    double *Gs = ar.take(mm), *d = ar.take(m), *lam = ar.take((size_t)m + 2);
    int *rdev = reinterpret_cast<int *>(ar.take(2));
    int *flag = h->flag.as<int>();
    GB_CUDA(cudaMemsetAsync(flag, 0, 16, s));
    // 1. rank-revealing basis of W = [S, B0 Y]: pivoted Cholesky of the
    //    column-scaled Gram matrix D W^T W D (d_i = 1 / |w_i|), coordinates
    //    coef1 D, then a CholeskyQR pass (no n-long work: G is kept by the update)
    GB_CUDA(cudaMemcpyAsync(Gs, h->dG.p, mm * sizeof(double), cudaMemcpyDeviceToDevice, s));
    gram_scale_kernel<<<1, 256, 0, s>>>(Gs, m, d);
    GB_LAUNCHED();
    double *Tq = nullptr;
    int r = 0;
    GB_TRY(basis_coords(h, Gs, nullptr, m, m, 1e-4, d, ar, Tq, r, rdev, flag, s));
    if (r < 1) return gb_nonfinite("BFGS pairs S, B0 Y are zero or not finite");
    // 2. T = Q (B - B0) Q^T = C M C^T with C = Q W^T = Tq G, its eigenpairs, V = U^T Q
    double *work = ar.take(4 * mm + 4 * (size_t)m), *T = ar.take(mm);
    GB_TRY(rayleigh_ritz(h, Tq, r, m, ar, T, s));
    GB_TRY(launch_eig(T, r, rank, work, lam, h->coef.as<float>(), flag, s));
    return finish_lowrank(h, Tq, r, rank, lam, eps_prior, V, lambda, std_out, ar, flag, rdev, s);
}
