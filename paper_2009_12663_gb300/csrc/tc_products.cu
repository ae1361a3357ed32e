// Tensor-core products of the compact BFGS apply and the randomized SVD
// (sm_103a): the tall-skinny [S B0Y]^T X-type products and the row
// combinations [S B0Y] (M W)-type of the compact form of the inverse
// Hessian (Section 2.3, Eq. 9, Algorithms 2-3; Byrd, Nocedal & Schnabel
// 1994), and the Gram / projection products of Algorithm 3.
//
// Precision.  Every operand is FP32.  Each value x is split exactly into
// three bfloat16 parts, x = x1 + x2 + x3 (x1 = bf16(x), x2 = bf16(x - x1),
// x3 = x - x1 - x2: 8 significant bits each, 24 in all), and a product is
// taken as the six terms x_i y_j with i + j <= 4 on the tensor cores, small
// terms first; the dropped x2 y3, x3 y2, x3 y3 are below 2^-23 of |x y|, so a
// product is as accurate as an FP32 product (the splitting of Ootomo &
// Yokota (2022) carried to three bfloat16 parts, which is exact where two
// TF32 parts are not).  The tensor core keeps about 24 bits below the largest
// term of an MMA and truncates the rest (measured on sm_103a for mma.sync and
// for tcgen05.mma), so its accumulation never spans more than one 16-deep K
// step: each step's six part products go into a fresh TMEM accumulator, the
// step sums are added in FP32, and the long sums over n of the split-K
// products are carried in compensated FP32 pairs (TwoSum of Knuth) and
// reduced over the splits in FP64.
//
// Machinery (sm_100 family, inline PTX in sm100.h): operands arrive in
// shared memory by 2-D tensor-map loads (cp.async.bulk.tensor, zero past n)
// or one bulk copy per row, completing on mbarriers; the split parts are
// written into K-major 128-byte-swizzled planes read by tcgen05.mma (one
// issuing thread, accumulators in tensor memory), whose completion is
// committed to an mbarrier; the accumulators come back with tcgen05.ld.
// Rows are vectors of length n with a row stride ld (a multiple of 64
// floats, rows 256-byte aligned, readable up to the pitch).

#include <algorithm>
#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "gbfwi_internal.h"
#include "sm100.h"

namespace {

// two floats -> packed bfloat16 pair (round to nearest even), lo_col in the
// lower half
__device__ __forceinline__ unsigned pack_bf16(float lo_col, float hi_col)
{
    unsigned r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi_col), "f"(lo_col));
    return r;
}

// exact three-part bfloat16 split of the pair (u, v): u = u1 + u2 + u3 with
// the parts packed as (u_i, v_i) in p[i]
__device__ __forceinline__ void split3(float u, float v, unsigned (&p)[3])
{
    p[0] = pack_bf16(u, v);
    const float ur = __fsub_rn(u, __uint_as_float(p[0] << 16));
    const float vr = __fsub_rn(v, __uint_as_float(p[0] & 0xffff0000u));
    p[1] = pack_bf16(ur, vr);
    const float ur2 = __fsub_rn(ur, __uint_as_float(p[1] << 16));
    const float vr2 = __fsub_rn(vr, __uint_as_float(p[1] & 0xffff0000u));
    p[2] = pack_bf16(ur2, vr2);
}

// s + e += x, keeping s + e exact up to the rounding of e (TwoSum)
__device__ __forceinline__ void two_sum_add(float &s, float &e, float x)
{
    const float t = __fadd_rn(s, x);
    const float z = __fsub_rn(t, s);
    const float r = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z));
    s = t;
    e = __fadd_rn(e, r);
}

// row q of an operand made of two row blocks: q < k1 from P1, else P2
__device__ __forceinline__ const float *row_of(const float *P1, const float *P2, int k1, int q, long long ld)
{
    return q < k1 ? P1 + (long long)q * ld : P2 + (long long)(q - k1) * ld;
}

// ---------------------------------------------------------------------------
// split-K product on the 5th-generation tensor cores (tcgen05):
// part[sx][p sp + q sq] = sum_{i in split sx} P_p[i] Q_q[i]
// CTA tile: 128 P rows (the MMA's M, accumulator lane) x 64 Q rows (N);
// K steps of 64 through a two-stage ring of raw FP32 rows filled by bulk
// copies (one 256-byte row per copy, completing on an mbarrier).  Every
// staged element is split once into its three bfloat16 parts, written into
// three K-major 128-byte-swizzled planes per operand; per 16-deep K step one
// thread issues the six part products (smallest first) into a fresh TMEM
// accumulator (M 128, N 64), four steps per stage into four accumulators;
// the accumulator set of the previous stage is added in FP32 and folded into
// compensated FP32 pairs (TwoSum) while the tensor core works on the current
// one.  Two
// accumulator sets of 4 x 64 columns fill the 512 TMEM columns (one CTA per
// SM).  Elements at i >= n are taken as zero (rows are read to the 64-float
// row pitch).
// ---------------------------------------------------------------------------

constexpr int T5_M = 128, T5_N = 64, T5_K = 64, T5_THREADS = 256;
constexpr size_t T5_PLANE_P = (size_t)T5_M * 128;                 // bytes of one bfloat16 part plane of P
constexpr size_t T5_PLANE_Q = (size_t)T5_N * 128;
constexpr size_t T5_RAW = (size_t)(T5_M + T5_N) * T5_K * sizeof(float);   // one raw FP32 stage
constexpr size_t T5_SMEM = 1024 + 3 * (T5_PLANE_P + T5_PLANE_Q) + 2 * T5_RAW;

// 2-D tensor maps of the operand row blocks for single-tile products (P at
// most 128 rows, Q at most 64): map b covers rows [0, h[b]) of its block,
// landing at raw rows off[b]; elements at i >= n are filled with zeros
struct Tc05Maps {
    CUtensorMap m[4];    // P1, P2, Q1, Q2
    int h[4];            // box rows (0: block absent)
    int off[4];
    int use;             // 1: tensor-map loads, 0: one bulk copy per row
};

__global__ void __launch_bounds__(T5_THREADS, 1)
    atb_tc05_kernel(const __grid_constant__ Tc05Maps maps, const float *__restrict__ P1, const float *__restrict__ P2, int kp1, int kp,
                    const float *__restrict__ Q1, const float *__restrict__ Q2, int kq1, int kq, long long ld,
                    long long n, long long chunk, double *__restrict__ part, long long split_stride, long long sp,
                    long long sq, int *__restrict__ status)
{
    using namespace sm100;
    extern __shared__ unsigned char t5_smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)t5_smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *planeP = base;                                   // [3][128 rows][128 B]
    unsigned char *planeQ = base + 3 * T5_PLANE_P;                  // [3][64 rows][128 B]
    float *raw = reinterpret_cast<float *>(planeQ + 3 * T5_PLANE_Q);   // [2][192 rows][64]
    __shared__ unsigned long long mbar_raw[2], mbar_mma[2];
    __shared__ unsigned tslot;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sx = blockIdx.z;
    const int p0 = blockIdx.y * T5_M, q0 = blockIdx.x * T5_N;
    const int np = min(T5_M, kp - p0), nq = min(T5_N, kq - q0);
    const long long ib = (long long)sx * chunk;
    const long long ie = min(n, ib + chunk);
    const int nk = (int)((ie - ib + T5_K - 1) / T5_K);

    if (warp == 0) tmem_alloc(&tslot, 512);
    if (tid == 0) {
        mbar_init(&mbar_raw[0], 1);
        mbar_init(&mbar_raw[1], 1);
        mbar_init(&mbar_mma[0], 1);
        mbar_init(&mbar_mma[1], 1);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const unsigned tbase = tslot;

    // stage kt: P rows to raw rows [0, np), Q rows to [128, 128 + nq), by up to
    // four tensor-map loads or one bulk copy per row
    auto issue = [&](int kt) {
        float *buf = raw + (size_t)(kt & 1) * (T5_M + T5_N) * T5_K;
        const long long i0 = ib + (long long)kt * T5_K;
        if (maps.use) {
            if (tid == 0) {
                mbar_arrive_expect_tx(&mbar_raw[kt & 1],
                                      (unsigned)(maps.h[0] + maps.h[1] + maps.h[2] + maps.h[3]) * T5_K * sizeof(float));
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (maps.h[b] > 0) tma_load_2d(buf + (size_t)maps.off[b] * T5_K, &maps.m[b], (int)i0, 0, &mbar_raw[kt & 1]);
            }
            return;
        }
        if (tid == 0) mbar_arrive_expect_tx(&mbar_raw[kt & 1], (unsigned)(np + nq) * T5_K * sizeof(float));
        for (int r = tid; r < np + nq; r += T5_THREADS) {
            const bool isp = r < np;
            const float *src = isp ? row_of(P1, P2, kp1, p0 + r, ld) + i0 : row_of(Q1, Q2, kq1, q0 + r - np, ld) + i0;
            float *dst = buf + (size_t)(isp ? r : T5_M + r - np) * T5_K;
            bulk_g2s(dst, src, T5_K * sizeof(float), &mbar_raw[kt & 1]);
        }
    };
    issue(0);
    if (nk > 1) issue(1);

    constexpr unsigned idesc = idesc_bf16_f32(T5_M, T5_N);
    const int m = 32 * (warp & 3) + lane;                // accumulator row (TMEM lane) of this thread
    const int c0 = 32 * (warp >> 2);                     // its 32 of the 64 accumulator columns
    const unsigned tl = tbase + ((unsigned)(32 * (warp & 3)) << 16);
    float S[32], E[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) S[j] = E[j] = 0.f;

    // fold accumulator set `set` into the compensated pairs: the four 16-deep
    // step sums (each from a fresh accumulator, so the tensor core's
    // truncation never spans more than one step) are added in FP32 and the
    // result folded by TwoSum; warps whose 32 rows are all beyond np skip it
    const bool folds = 32 * (warp & 3) < np;
    auto fold = [&](int set) {
        if (!folds) return;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[4][16];
            const unsigned tc = tl + set * 256 + c0 + 16 * h;
            tmem_ld16x4(tc, tc + 64, tc + 128, tc + 192, v);
#pragma unroll
            for (int j = 0; j < 16; ++j)
                two_sum_add(S[16 * h + j], E[16 * h + j], (v[0][j] + v[1][j]) + (v[2][j] + v[3][j]));
        }
    };

    bool ok = true;
    int kfail = nk;                                      // first stage whose wait gave up
    for (int kt = 0; kt < nk; ++kt) {
        // stage kt landed; the MMAs of stage kt - 1 have released the planes
        // (each thread waits itself; a bound that ran out is agreed on at the
        // barrier below, before anything reads what was written)
        bool w = mbar_wait_bounded(&mbar_raw[kt & 1], (kt >> 1) & 1);
        if (kt > 0) w = w && mbar_wait_bounded(&mbar_mma[(kt - 1) & 1], ((kt - 1) >> 1) & 1);
        fence_after_sync();
        // split: the np + nq present rows x 8 chunks of 8 elements, each into
        // three 16-byte part chunks (elements at i >= ie zeroed in the last stage)
        {
            const float *src = raw + (size_t)(kt & 1) * (T5_M + T5_N) * T5_K;
            const long long i0 = ib + (long long)kt * T5_K;
            const bool tail = i0 + T5_K > ie;
            for (int item = tid; item < 8 * (np + nq); item += T5_THREADS) {
                const int rr0 = item >> 3, c = item & 7;
                const bool isp = rr0 < np;
                const int rr = isp ? rr0 : rr0 - np;
                const float *row = src + (size_t)(isp ? rr : T5_M + rr) * T5_K + 8 * c;
                const float4 x0 = *reinterpret_cast<const float4 *>(row);
                const float4 x1 = *reinterpret_cast<const float4 *>(row + 4);
                float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                if (tail) {
                    const long long ic = i0 + 8 * c;
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        if (ic + e >= ie) x[e] = 0.f;
                }
                unsigned pr[3][4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    unsigned s3[3];
                    split3(x[2 * h], x[2 * h + 1], s3);
                    pr[0][h] = s3[0];
                    pr[1][h] = s3[1];
                    pr[2][h] = s3[2];
                }
                unsigned char *pl = isp ? planeP : planeQ;
                const size_t pstride = isp ? T5_PLANE_P : T5_PLANE_Q;
                const unsigned off = k128_offset(rr, 8 * c);
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    *reinterpret_cast<uint4 *>(pl + q * pstride + off) = make_uint4(pr[q][0], pr[q][1], pr[q][2], pr[q][3]);
            }
        }
        fence_async_smem();
        fence_before_sync();
        if (__syncthreads_or(!w)) {                      // planes ready; raw stage kt & 1 free
            ok = false;
            kfail = kt;
            break;
        }
        if (kt + 2 < nk) issue(kt + 2);
        if (tid == 0) {
            fence_after_sync();
            const unsigned dset = tbase + (unsigned)((kt & 1) * 256);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                unsigned long long a[3], b[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    a[q] = sdesc_k128(planeP + q * T5_PLANE_P) + 2 * kk;
                    b[q] = sdesc_k128(planeQ + q * T5_PLANE_Q) + 2 * kk;
                }
                const unsigned d = dset + kk * 64;
                // the six terms a_i b_j, i + j <= 2 (parts 0 largest), smallest first
                sm100::mma_bf16(d, a[2], b[0], idesc, false);
                sm100::mma_bf16(d, a[0], b[2], idesc, true);
                sm100::mma_bf16(d, a[1], b[1], idesc, true);
                sm100::mma_bf16(d, a[1], b[0], idesc, true);
                sm100::mma_bf16(d, a[0], b[1], idesc, true);
                sm100::mma_bf16(d, a[0], b[0], idesc, true);
            }
            mma_commit(&mbar_mma[kt & 1]);
        }
        if (kt > 0) fold((kt - 1) & 1);                  // overlaps the MMAs of stage kt
    }
    if (ok && nk > 0) {
        ok = __syncthreads_and(mbar_wait_bounded(&mbar_mma[(nk - 1) & 1], ((nk - 1) >> 1) & 1));
        if (!ok) kfail = nk;
        if (ok) {
            fence_after_sync();
            fold((nk - 1) & 1);
        }
    }
    if (ok) {
        if (m < np) {
            double *dst = part + (long long)sx * split_stride + (long long)(p0 + m) * sp;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (c0 + j < nq) dst[(long long)(q0 + c0 + j) * sq] = (double)S[j] + (double)E[j];
        }
    } else {
        if (tid == 0 && status) atomicExch(status, 1);
        // give the copies and MMAs still in flight a bounded wait before the
        // shared memory and the accumulators are released
        for (int st = kfail; st < min(nk, kfail + 2); ++st) mbar_wait_bounded(&mbar_raw[st & 1], (st >> 1) & 1);
        if (kfail > 0) mbar_wait_bounded(&mbar_mma[(kfail - 1) & 1], ((kfail - 1) >> 1) & 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, 512);
}

__global__ void split_reduce_kernel(const double *__restrict__ part, int nsplit, int ka, int kb,
                                    double *__restrict__ out, long long ldo)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= ka * kb) return;
    double s = 0.0;
    for (int sx = 0; sx < nsplit; ++sx) s += part[(long long)sx * ka * kb + q];
    const int a = q / kb, b = q - a * kb;
    out[(long long)a * ldo + b] = s;
}

// ---------------------------------------------------------------------------
// row combination on the 5th-generation tensor cores (tcgen05):
// out[c][i] = sum_a coef[c][a] R_a[i] + beta dw[i] Xc[c][i], c in
// [64 blockIdx.y, + 64), a < ktot <= 128.  The MMA's M is a tile of 128
// columns i, N the 64 outputs c, K the rows a: persistent CTAs walk over the
// column tiles; a tile's rows arrive by tensor-map loads (one per row block,
// zero past n) or one bulk copy per row, are split into three bfloat16 parts
// and transposed into K-major 128-byte-swizzled planes (two 64-row K
// blocks); coef is split once per CTA.  Per 16-row K step one thread issues
// the six part products into a fresh TMEM accumulator (up to 8 x 64
// columns); the step sums are added pairwise in FP32.
// ---------------------------------------------------------------------------

constexpr int C5_M = 128, C5_N = 64, C5_KB = 64, C5_THREADS = 256;
constexpr size_t C5_APLANE = (size_t)C5_M * 128;                 // bytes of one A part plane (one K block)
constexpr size_t C5_BPLANE = (size_t)C5_N * 128;
constexpr size_t C5_RAW = (size_t)128 * C5_M * sizeof(float);    // rows a x 128 columns
constexpr size_t C5_SMEM = 1024 + 6 * C5_APLANE + 6 * C5_BPLANE + C5_RAW;

struct Cb5Maps {
    CUtensorMap m[2];    // R1, R2
    int h[2];            // box rows (0: block absent)
    int use;
};

__global__ void __launch_bounds__(C5_THREADS, 1)
    combine_tc05_kernel(const __grid_constant__ Cb5Maps maps, const float *__restrict__ R1,
                        const float *__restrict__ R2, int k1, int ktot, long long ldr, const float *__restrict__ coef,
                        int nc, long long n, float *__restrict__ out, long long ldo, const float *__restrict__ dw,
                        const float *__restrict__ Xc, long long ldx, float beta, int *__restrict__ status)
{
    using namespace sm100;
    extern __shared__ unsigned char c5_smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)c5_smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *planeA = base;                                  // [kb 2][part 3][128 rows i][128 B]
    unsigned char *planeB = base + 6 * C5_APLANE;                  // [kb 2][part 3][64 rows c][128 B]
    float *raw = reinterpret_cast<float *>(planeB + 6 * C5_BPLANE);   // [ktot rows a][128]
    __shared__ unsigned long long mbar_raw, mbar_mma;
    __shared__ unsigned tslot;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = blockIdx.y * C5_N;
    const int ncl = min(C5_N, nc - c0);
    const int nks = (ktot + 15) / 16;                    // 16-row K steps
    const long long ntiles = (n + C5_M - 1) / C5_M;

    if (warp == 0) tmem_alloc(&tslot, 512);
    if (tid == 0) {
        mbar_init(&mbar_raw, 1);
        mbar_init(&mbar_mma, 1);
    }
    // coef split once: B[c][a], zero beyond ncl rows and ktot columns
    for (int item = tid; item < C5_N * 16; item += C5_THREADS) {
        const int c = item >> 4, q = item & 15;          // 16 chunks of 8 along a (two K blocks)
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int a = 8 * q + e;
            x[e] = (c < ncl && a < ktot) ? coef[(long long)(c0 + c) * ktot + a] : 0.f;
        }
        unsigned pr[3][4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            unsigned s3[3];
            split3(x[2 * h], x[2 * h + 1], s3);
            pr[0][h] = s3[0];
            pr[1][h] = s3[1];
            pr[2][h] = s3[2];
        }
        const int kb = q >> 3;
        const unsigned off = k128_offset(c, 8 * (q & 7));
#pragma unroll
        for (int pt = 0; pt < 3; ++pt)
            *reinterpret_cast<uint4 *>(planeB + (kb * 3 + pt) * C5_BPLANE + off) =
                make_uint4(pr[pt][0], pr[pt][1], pr[pt][2], pr[pt][3]);
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const unsigned tbase = tslot;

    auto issue = [&](long long tile) {
        const long long i0 = tile * C5_M;
        if (maps.use) {
            if (tid == 0) {
                mbar_arrive_expect_tx(&mbar_raw, (unsigned)(maps.h[0] + maps.h[1]) * C5_M * sizeof(float));
                if (maps.h[0] > 0) tma_load_2d(raw, &maps.m[0], (int)i0, 0, &mbar_raw);
                if (maps.h[1] > 0) tma_load_2d(raw + (size_t)maps.h[0] * C5_M, &maps.m[1], (int)i0, 0, &mbar_raw);
            }
            return;
        }
        const long long iend = min(i0 + C5_M, ldr);      // rows are readable to their pitch
        const unsigned bytes = (unsigned)(iend - i0) * sizeof(float);
        if (tid == 0) mbar_arrive_expect_tx(&mbar_raw, (unsigned)ktot * bytes);
        for (int a = tid; a < ktot; a += C5_THREADS)
            bulk_g2s(raw + (size_t)a * C5_M, row_of(R1, R2, k1, a, ldr) + i0, bytes, &mbar_raw);
    };

    constexpr unsigned idesc = idesc_bf16_f32(C5_M, C5_N);
    const int i_loc = 32 * (warp & 3) + lane;            // accumulator row (TMEM lane): column i0 + i_loc
    const int cw = 32 * (warp >> 2);                     // this thread's 32 of the 64 outputs
    const unsigned tl = tbase + ((unsigned)(32 * (warp & 3)) << 16);
    bool ok = true;
    int it = 0;
    int inflight = -1;                                   // iteration whose rows are being copied
    if (blockIdx.x < ntiles) {
        issue(blockIdx.x);
        inflight = 0;
    }
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const long long i0 = tile * C5_M;
        bool w = mbar_wait_bounded(&mbar_raw, it & 1);
        fence_after_sync();
        // split + transpose: item = (column i, chunk of 8 rows a)
        for (int item = tid; item < C5_M * 16; item += C5_THREADS) {
            const int i = item & (C5_M - 1), q = item >> 7;   // lanes take consecutive columns
            if (8 * q >= nks * 16) continue;
            float x[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int a = 8 * q + e;
                x[e] = (a < ktot && i0 + i < n) ? raw[(size_t)a * C5_M + i] : 0.f;
            }
            unsigned pr[3][4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                unsigned s3[3];
                split3(x[2 * h], x[2 * h + 1], s3);
                pr[0][h] = s3[0];
                pr[1][h] = s3[1];
                pr[2][h] = s3[2];
            }
            const int kb = q >> 3;
            const unsigned off = k128_offset(i, 8 * (q & 7));
#pragma unroll
            for (int pt = 0; pt < 3; ++pt)
                *reinterpret_cast<uint4 *>(planeA + (kb * 3 + pt) * C5_APLANE + off) =
                    make_uint4(pr[pt][0], pr[pt][1], pr[pt][2], pr[pt][3]);
        }
        fence_async_smem();
        fence_before_sync();
        if (__syncthreads_or(!w)) {                      // planes ready, raw consumed
            ok = false;
            break;
        }
        inflight = -1;
        if (tile + gridDim.x < ntiles) {
            issue(tile + gridDim.x);
            inflight = it + 1;
        }
        if (tid == 0) {
            fence_after_sync();
            for (int ks = 0; ks < nks; ++ks) {
                const int kb = ks >> 2, kk = ks & 3;
                unsigned long long ad[3], bd[3];
#pragma unroll
                for (int pt = 0; pt < 3; ++pt) {
                    ad[pt] = sdesc_k128(planeA + (kb * 3 + pt) * C5_APLANE) + 2 * kk;
                    bd[pt] = sdesc_k128(planeB + (kb * 3 + pt) * C5_BPLANE) + 2 * kk;
                }
                const unsigned d = tbase + ks * 64;
                sm100::mma_bf16(d, ad[2], bd[0], idesc, false);
                sm100::mma_bf16(d, ad[0], bd[2], idesc, true);
                sm100::mma_bf16(d, ad[1], bd[1], idesc, true);
                sm100::mma_bf16(d, ad[1], bd[0], idesc, true);
                sm100::mma_bf16(d, ad[0], bd[1], idesc, true);
                sm100::mma_bf16(d, ad[0], bd[0], idesc, true);
            }
            mma_commit(&mbar_mma);
        }
        if (!__syncthreads_and(mbar_wait_bounded(&mbar_mma, it & 1))) {
            ok = false;
            break;
        }
        fence_after_sync();
        // add the K-step sums (each from a fresh accumulator, so the tensor
        // core's truncation never spans more than one step) pairwise in FP32,
        // then the epilogue of this thread's column
        const long long i = i0 + i_loc;
        const float dwi = (beta != 0.f && i < n) ? dw[i] : 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[8][16];
            const unsigned tc = tl + cw + 16 * h;
            tmem_ld16x4(tc, tc + 64, tc + 128, tc + 192, *reinterpret_cast<float(*)[4][16]>(&v[0][0]));
            if (nks > 4) tmem_ld16x4(tc + 256, tc + 320, tc + 384, tc + 448, *reinterpret_cast<float(*)[4][16]>(&v[4][0]));
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (u >= nks)
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[u][j] = 0.f;
            if (i < n) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = cw + 16 * h + j;
                    if (c < ncl) {
                        float r = ((v[0][j] + v[1][j]) + (v[2][j] + v[3][j])) + ((v[4][j] + v[5][j]) + (v[6][j] + v[7][j]));
                        if (beta != 0.f) r = fmaf(beta * dwi, Xc[(long long)(c0 + c) * ldx + i], r);
                        out[(long long)(c0 + c) * ldo + i] = r;
                    }
                }
            }
        }
        fence_before_sync();
    }
    if (!ok) {
        // flag it; give the copy and the MMAs still in flight a bounded wait
        if (tid == 0 && status) atomicExch(status, 1);
        if (inflight >= 0) mbar_wait_bounded(&mbar_raw, inflight & 1);
        mbar_wait_bounded(&mbar_mma, it & 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, 512);
}

// cuTensorMapEncodeTiled, from the driver through the runtime (no link
// against the driver library); null when unavailable
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        else
            cudaGetLastError();
    }
    return fn;
}

// map of rows [0, rows) of a block (pitch ld floats) over n elements, one
// box = 64 elements x all rows
bool encode_rows(CUtensorMap *m, const float *base, long long n, int rows, long long ld)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = tmap_encoder();
    if (!fn || rows < 1 || rows > 256) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)T5_K, (cuuint32_t)rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// tensor maps of a single-tile product (P: kp <= 128 rows from P1 / P2 split
// at kp1; Q likewise, at most 64 rows), or maps.use = 0
Tc05Maps tc05_maps(const float *P1, const float *P2, int kp1, int kp, const float *Q1, const float *Q2, int kq1,
                   int kq, long long ld, long long n)
{
    Tc05Maps mp;
    std::memset(&mp, 0, sizeof(mp));
    if (kp > T5_M || kq > T5_N || n < T5_K) return mp;
    const int h[4] = {std::min(kp1, kp), kp - std::min(kp1, kp), std::min(kq1, kq), kq - std::min(kq1, kq)};
    const float *b[4] = {P1, P2, Q1, Q2};
    const int off[4] = {0, h[0], T5_M, T5_M + h[2]};
    for (int i = 0; i < 4; ++i) {
        mp.h[i] = h[i];
        mp.off[i] = off[i];
        if (h[i] > 0 && (!b[i] || !encode_rows(&mp.m[i], b[i], n, h[i], ld))) {
            std::memset(&mp, 0, sizeof(mp));
            return mp;
        }
    }
    mp.use = 1;
    return mp;
}

// orientation of a product on the tcgen05 kernel: the operand with more
// rows (up to 128) takes the MMA's M
struct Tc05Shape {
    bool swap;           // P = B, Q = A
    int kp, kq;          // rows of P and Q
    int gx, gy;          // tiles along Q (64 rows) and P (128 rows)
};

Tc05Shape tc05_shape(int ka, int kb)
{
    Tc05Shape t;
    t.swap = kb > ka && kb <= T5_M && ka <= T5_N;
    t.kp = t.swap ? kb : ka;
    t.kq = t.swap ? ka : kb;
    t.gx = (t.kq + T5_N - 1) / T5_N;
    t.gy = (t.kp + T5_M - 1) / T5_M;
    return t;
}

int tc05_prepare(int *nsm_out)
{
    static bool attr[64] = {};
    static int nsm_of[64] = {};
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GBFWI_EINVAL;
    if (!attr[dev]) {
        GB_CUDA(cudaFuncSetAttribute(atb_tc05_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T5_SMEM));
        int nsm = 152;
        GB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        nsm_of[dev] = nsm;
        attr[dev] = true;
    }
    *nsm_out = nsm_of[dev];
    return GBFWI_OK;
}

// K range of one split: a multiple of the 64-deep stage
long long tc05_chunk(int ka, int kb, long long n, long long *nsplit_out)
{
    int nsm = 152;
    if (tc05_prepare(&nsm) != GBFWI_OK) return -1;
    const Tc05Shape t = tc05_shape(ka, kb);
    const long long tiles = (long long)t.gx * t.gy;
    // one wave of CTAs (one per SM), each split at least 8 stages long
    const long long nsplit = std::max<long long>(1, std::min<long long>(nsm / tiles, n / (8 * T5_K)));
    const long long chunk = ((n + nsplit - 1) / nsplit + T5_K - 1) / T5_K * T5_K;
    *nsplit_out = (n + chunk - 1) / chunk;
    return chunk;
}

}  // namespace

long long gb_tc_atb_splits(int ka, int kb, long long n)
{
    long long nsplit = 0;
    if (tc05_chunk(ka, kb, n, &nsplit) < 1) return -1;
    return nsplit;
}

int gb_tc_atb(const float *A1, const float *A2, int ka1, int ka, const float *B1, const float *B2, int kb1, int kb,
              long long ld, long long n, double *part, size_t part_doubles, double *out, long long ldo,
              int *status, cudaStream_t s)
{
    if (ka < 1 || kb < 1 || n < 1) return GBFWI_OK;
    if (ld % T5_K != 0 || ld < n || ((uintptr_t)A1 & 255) || ((uintptr_t)A2 & 255) || ((uintptr_t)B1 & 255) ||
        ((uintptr_t)B2 & 255))
        return GBFWI_EINVAL;
    long long nsplit = 0;
    const long long chunk = tc05_chunk(ka, kb, n, &nsplit);
    if (chunk < 1) return GBFWI_ECUDA;
    if ((size_t)nsplit * ka * kb > part_doubles) return GBFWI_EINVAL;
    const Tc05Shape t = tc05_shape(ka, kb);
    // part[sx][a][b]: (P, Q) = (A, B) writes row p at a, or (B, A) at b
    const long long sp = t.swap ? 1 : kb, sq = t.swap ? kb : 1;
    if (t.swap) {
        const Tc05Maps mp = tc05_maps(B1, B2, kb1, kb, A1, A2, ka1, ka, ld, n);
        atb_tc05_kernel<<<dim3(t.gx, t.gy, (unsigned)nsplit), T5_THREADS, T5_SMEM, s>>>(
            mp, B1, B2, kb1, kb, A1, A2, ka1, ka, ld, n, chunk, part, (long long)ka * kb, sp, sq, status);
    } else {
        const Tc05Maps mp = tc05_maps(A1, A2, ka1, ka, B1, B2, kb1, kb, ld, n);
        atb_tc05_kernel<<<dim3(t.gx, t.gy, (unsigned)nsplit), T5_THREADS, T5_SMEM, s>>>(
            mp, A1, A2, ka1, ka, B1, B2, kb1, kb, ld, n, chunk, part, (long long)ka * kb, sp, sq, status);
    }
    GB_LAUNCHED();
    const int nab = ka * kb;
    split_reduce_kernel<<<(nab + 255) / 256, 256, 0, s>>>(part, (int)nsplit, ka, kb, out, ldo);
    GB_LAUNCHED();
    return GBFWI_OK;
}

int gb_tc_combine(const float *R1, const float *R2, int k1, int ktot, long long ldr, const float *coef, int nc,
                  long long n, float *out, long long ldo, const float *dw, const float *Xc, long long ldx,
                  float beta, int *status, cudaStream_t s)
{
    if (nc < 1 || n < 1) return GBFWI_OK;
    if (ktot < 1 || ktot > 128 || ldr % C5_KB != 0 || ldr < n || ((uintptr_t)R1 & 255) || ((uintptr_t)R2 & 255))
        return GBFWI_EINVAL;
    static bool attr[64] = {};
    static int nsm_of[64] = {};
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GBFWI_EINVAL;
    if (!attr[dev]) {
        GB_CUDA(cudaFuncSetAttribute(combine_tc05_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C5_SMEM));
        int nsm = 152;
        GB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        nsm_of[dev] = nsm;
        attr[dev] = true;
    }
    // tensor maps of the two row blocks: box 128 columns x all rows of the block
    Cb5Maps mp;
    std::memset(&mp, 0, sizeof(mp));
    mp.h[0] = std::min(k1, ktot);
    mp.h[1] = ktot - mp.h[0];
    mp.use = n >= C5_M;
    const float *blk[2] = {R1, R2};
    PFN_cuTensorMapEncodeTiled_v12000 fn = tmap_encoder();
    for (int b = 0; b < 2 && mp.use; ++b) {
        if (mp.h[b] == 0) continue;
        const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)mp.h[b]};
        const cuuint64_t strides[1] = {(cuuint64_t)ldr * sizeof(float)};
        const cuuint32_t box[2] = {(cuuint32_t)C5_M, (cuuint32_t)mp.h[b]};
        const cuuint32_t es[2] = {1, 1};
        mp.use = fn && blk[b] &&
                 fn(&mp.m[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(blk[b]), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    const long long ntiles = (n + C5_M - 1) / C5_M;
    const int ny = (nc + C5_N - 1) / C5_N;
    const int gx = (int)std::max<long long>(1, std::min<long long>(ntiles, std::max(1, nsm_of[dev] / ny)));
    combine_tc05_kernel<<<dim3(gx, ny), C5_THREADS, C5_SMEM, s>>>(mp, R1, R2, k1, ktot, ldr, coef, nc, n, out, ldo, dw,
                                                                 Xc, ldx, beta, status);
    GB_LAUNCHED();
    return GBFWI_OK;
}
