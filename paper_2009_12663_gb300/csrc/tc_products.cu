// Tensor-core products of the compact BFGS apply and the randomized SVD
// (sm_103a): the tall-skinny [S B0Y]^T X-type products and the row
// combinations [S B0Y] (M W)-type of the compact form of the inverse
// Hessian (Section 2.3, Eq. 9, Algorithms 2-3; Byrd, Nocedal & Schnabel
// 1994), and the Gram / projection products of Algorithm 3.
//
// Precision.  Every operand is FP32.  Each value x is split exactly into
// three bfloat16 parts, x = x1 + x2 + x3 (x1 = bf16(x), x2 = bf16(x - x1),
// x3 = x - x1 - x2: 8 significant bits each, 24 in all), and a product is
// taken as the six terms x_i y_j with i + j <= 4 on the tensor cores
// (mma.sync m16n8k16 BF16, products exact in the FP32 accumulator), small
// terms first; the dropped x2 y3, x3 y2, x3 y3 are below 2^-23 of |x y|, so a
// product is as accurate as an FP32 product (the splitting of Ootomo &
// Yokota (2022) carried to three bfloat16 parts, which is exact where two
// TF32 parts are not).  The tensor core's FP32 accumulation is kept short:
// after every 16-deep K step its sum is folded into a compensated FP32 pair
// (TwoSum of Knuth), so the long sums over n of the split-K products are
// close to exact sums of the FP32 products, and the splits are reduced in
// FP64; the row combinations sum at most 128 terms the same way.  (A probe
// of mma.sync on sm_103a: a BF16 or TF32 MMA keeps about 24 bits below its
// largest term and truncates the rest.)
//
// Layout: rows are vectors of length n with a row stride ld (a multiple of
// 4 floats, rows 16-byte aligned); both kernels stage their operands in
// shared memory with 16-byte cp.async copies (zero-filled beyond n and
// beyond the last row).

#include <algorithm>

#include "gbfwi_internal.h"

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

__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// d += the six terms a_i b_j, i + j <= 4 (parts 0..2), smallest first
__device__ __forceinline__ void mma_split6(float (&d)[4], const unsigned (&a)[3][4], const unsigned (&b)[3][2])
{
    mma_bf16(d, a[2][0], a[2][1], a[2][2], a[2][3], b[0][0], b[0][1]);
    mma_bf16(d, a[0][0], a[0][1], a[0][2], a[0][3], b[2][0], b[2][1]);
    mma_bf16(d, a[1][0], a[1][1], a[1][2], a[1][3], b[1][0], b[1][1]);
    mma_bf16(d, a[1][0], a[1][1], a[1][2], a[1][3], b[0][0], b[0][1]);
    mma_bf16(d, a[0][0], a[0][1], a[0][2], a[0][3], b[1][0], b[1][1]);
    mma_bf16(d, a[0][0], a[0][1], a[0][2], a[0][3], b[0][0], b[0][1]);
}

__device__ __forceinline__ void cp16(void *smem, const void *gmem, int src_bytes)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

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
// split-K product: part[sx][a][b] = sum_{i in split sx} A_a[i] B_b[i]
// CTA: 64 x 64 output tile, 4 warps of 32 x 32 (2 m16 x 4 n8 MMA tiles);
// K staged 32 at a time (two 16-deep MMA steps) through a double-buffered
// cp.async pipeline; every staged element is split into its three bfloat16
// parts once, into shared planes the fragments are read from.
// grid (ceil(kb / 64), ceil(ka / 64), nsplit): the splits vary slowest, so
// the tiles that read the same K range run together and share it in L2.
// ---------------------------------------------------------------------------

// row pitches: raw FP32 tiles 32 floats (16-byte cp.async rows), split
// planes 20 words (the fragment loads of a warp hit 32 distinct banks)
constexpr int AT_M = 64, AT_N = 64, AT_K = 32, AT_P = AT_K, AT_PP = AT_K / 2 + 4, AT_THREADS = 128;
constexpr size_t AT_RAW = (size_t)(AT_M + AT_N) * AT_P;          // floats of one raw stage
constexpr size_t AT_PLANE = (size_t)(AT_M + AT_N) * AT_PP;       // words of one split plane
constexpr size_t AT_SMEM = (2 * AT_RAW + 3 * AT_PLANE) * sizeof(float);

__global__ void __launch_bounds__(AT_THREADS, 3) atb_tc_kernel(const float *__restrict__ A1, const float *__restrict__ A2,
                                                            int ka1, int ka, const float *__restrict__ B1,
                                                            const float *__restrict__ B2, int kb1, int kb,
                                                            long long ld, long long n, long long chunk,
                                                            double *__restrict__ part)
{
    extern __shared__ float4 at_smem4[];
    float *raw = reinterpret_cast<float *>(at_smem4);                  // [2][128 rows][32]
    unsigned *pl = reinterpret_cast<unsigned *>(raw + 2 * AT_RAW);     // [3][128 rows][20]
    const int sx = blockIdx.z;
    const int a0 = blockIdx.y * AT_M, b0 = blockIdx.x * AT_N;
    const long long ib = (long long)sx * chunk;
    const long long ie = min(n, ib + chunk);
    const int nk = (int)((ie - ib + AT_K - 1) / AT_K);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;

    // raw stage: rows 0..63 of A then 0..63 of B, 8 16-byte chunks each
    auto load = [&](int buf, int kt) {
        float *dst = raw + (size_t)buf * AT_RAW;
        const long long i0 = ib + (long long)kt * AT_K;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = tid + u * AT_THREADS;           // 0..1023
            const int r = q >> 3, c = q & 7;               // r: 0..127
            const bool isb = r >= 64;
            const int row = (isb ? b0 - 64 : a0) + r;
            const int lim = isb ? kb : ka;
            const long long i = i0 + 4 * c;
            int bytes = 0;
            const float *src = isb ? B1 : A1;
            if (row < lim && i < ie) {
                src = isb ? row_of(B1, B2, kb1, row, ld) + i : row_of(A1, A2, ka1, row, ld) + i;
                bytes = (int)min(16LL, (ie - i) * 4);
            }
            cp16(dst + r * AT_P + 4 * c, src, bytes);
        }
    };

    float S[2][4][4], E[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int v = 0; v < 4; ++v) S[mt][nt][v] = E[mt][nt][v] = 0.f;

    load(0, 0);
    cp_commit();
    if (nk > 1) load(1, 1);
    cp_commit();
    for (int kt = 0; kt < nk; ++kt) {
        cp_wait<1>();
        __syncthreads();                                   // raw stage kt landed; planes free
        {
            // split every element of the stage once: 128 rows x 16 pairs
            const float *src = raw + (size_t)(kt & 1) * AT_RAW;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int q = tid + u * AT_THREADS;        // 0..2047
                const int r = q >> 4, c = q & 15;
                const float2 v = *reinterpret_cast<const float2 *>(src + r * AT_P + 2 * c);
                unsigned s3[3];
                split3(v.x, v.y, s3);
#pragma unroll
                for (int part = 0; part < 3; ++part) pl[part * AT_PLANE + r * AT_PP + c] = s3[part];
            }
        }
        __syncthreads();                                   // planes ready; raw stage kt free
        if (kt + 2 < nk) load(kt & 1, kt + 2);
        cp_commit();
#pragma unroll
        for (int kk = 0; kk < AT_K; kk += 16) {
            unsigned a[2][3][4], b[4][3][2];
            const int kw = kk / 2 + t;                     // word of the pair (kk + 2t, kk + 2t + 1)
#pragma unroll
            for (int part = 0; part < 3; ++part) {
                const unsigned *P = pl + part * AT_PLANE;
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int r = wm + mt * 16 + g;
                    a[mt][part][0] = P[r * AT_PP + kw];
                    a[mt][part][1] = P[(r + 8) * AT_PP + kw];
                    a[mt][part][2] = P[r * AT_PP + kw + 4];
                    a[mt][part][3] = P[(r + 8) * AT_PP + kw + 4];
                }
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const int r = 64 + wn + nt * 8 + g;
                    b[nt][part][0] = P[r * AT_PP + kw];
                    b[nt][part][1] = P[r * AT_PP + kw + 4];
                }
            }
            // each 16-product sum goes into the compensated pair at once:
            // the tensor core truncates its FP32 sums, and a longer run in
            // its accumulator measurably biases the small directions of an
            // ill-conditioned block
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    float D[4] = {0.f, 0.f, 0.f, 0.f};
                    mma_split6(D, a[mt], b[nt]);
#pragma unroll
                    for (int v = 0; v < 4; ++v) two_sum_add(S[mt][nt][v], E[mt][nt][v], D[v]);
                }
        }
    }
    cp_wait<0>();
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int a = a0 + wm + mt * 16 + g + ((v & 2) ? 8 : 0);
                const int b = b0 + wn + nt * 8 + 2 * t + (v & 1);
                if (a < ka && b < kb)
                    part[((long long)sx * ka + a) * kb + b] = (double)S[mt][nt][v] + (double)E[mt][nt][v];
            }
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
// row combination: out[c][i] = sum_a coef[c][a] R_a[i] + beta dw[i] Xc[c][i]
// for c in [c0, c0 + 16 MT) (blockIdx.y selects c0 = 64 blockIdx.y).
// coef stays in shared memory, split once; persistent CTAs walk over
// 64-column tiles, streaming R in K steps of 32 rows (two 16-deep MMA steps)
// through a four-stage cp.async pipeline.  4 warps, each all MT m16 tiles x
// 2 n8 tiles (16 columns).  The sums over K (at most 128 terms) are folded
// into compensated FP32 pairs after every 16-deep step, as in the split-K
// product: the basis combinations of the randomized SVD have ill-conditioned
// coefficients, and a plain FP32 sum of their terms loses the small
// directions.
// ---------------------------------------------------------------------------

// R stages are raw FP32 [32 rows][64 columns]; each stage is split once into
// three planes of row pairs [16][72 words] (conflict-free fragment loads);
// coef is split once into three planes [16 MT][K/2 + 4 words].
constexpr int CB_N = 64, CB_K = 32, CB_RPP = CB_N + 8, CB_STAGES = 4, CB_THREADS = 128;
constexpr size_t CB_RAW = (size_t)CB_K * CB_N;            // floats of one raw stage
constexpr size_t CB_PLANE = (size_t)(CB_K / 2) * CB_RPP;  // words of one split plane of R

template <int MT>
__global__ void __launch_bounds__(CB_THREADS) combine_tc_kernel(const float *__restrict__ R1,
                                                                const float *__restrict__ R2, int k1, int ktot,
                                                                long long ldr, const float *__restrict__ coef,
                                                                int nc, long long n, float *__restrict__ out,
                                                                long long ldo, const float *__restrict__ dw,
                                                                const float *__restrict__ Xc, long long ldx,
                                                                float beta)
{
    extern __shared__ float4 cb_smem4[];
    const int kp = (ktot + CB_K - 1) / CB_K * CB_K;      // K padded to whole steps
    const int cpp = kp / 2 + 4;                          // coef plane pitch in words
    float *raw = reinterpret_cast<float *>(cb_smem4);                   // [stages][32][64]
    unsigned *rp = reinterpret_cast<unsigned *>(raw + CB_STAGES * CB_RAW);   // [3][16][72]
    unsigned *cp = rp + 3 * CB_PLANE;                                   // [3][16 MT][cpp]
    const int c0 = blockIdx.y * 64;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int wn = warp * 16;
    // coef planes: pairs along K of each output row
    for (int q = tid; q < 16 * MT * (kp / 2); q += CB_THREADS) {
        const int c = q / (kp / 2), w = q - c * (kp / 2);
        const int a = 2 * w;
        const bool ok = c0 + c < nc;
        const float u = (ok && a < ktot) ? coef[(long long)(c0 + c) * ktot + a] : 0.f;
        const float v = (ok && a + 1 < ktot) ? coef[(long long)(c0 + c) * ktot + a + 1] : 0.f;
        unsigned s3[3];
        split3(u, v, s3);
#pragma unroll
        for (int part = 0; part < 3; ++part) cp[(size_t)part * 16 * MT * cpp + c * cpp + w] = s3[part];
    }
    const long long ntiles = (n + CB_N - 1) / CB_N;
    const int nks = kp / CB_K;
    const long long my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long total = my_tiles * nks;
    auto load = [&](long long f) {
        const long long tile = blockIdx.x + (f / nks) * gridDim.x;
        const int ks = (int)(f % nks);
        float *dst = raw + (size_t)(f % CB_STAGES) * CB_RAW;
        const long long i0 = tile * CB_N;
#pragma unroll
        for (int u = 0; u < 4; ++u) {                     // 32 rows x 16 chunks = 512 chunks
            const int q = tid + u * CB_THREADS;
            const int r = q >> 4, c = q & 15;
            const int a = ks * CB_K + r;
            const long long i = i0 + 4 * c;
            int bytes = 0;
            const float *src = R1 ? R1 : R2;
            if (a < ktot && i < n) {
                src = row_of(R1, R2, k1, a, ldr) + i;
                bytes = (int)min(16LL, (n - i) * 4);
            }
            cp16(dst + r * CB_N + 4 * c, src, bytes);
        }
    };
    for (long long f = 0; f < CB_STAGES - 1; ++f) {
        if (f < total) load(f);
        cp_commit();
    }
    float S[MT][2][4], E[MT][2][4];
    for (long long f = 0; f < total; ++f) {
        const int ks = (int)(f % nks);
        if (ks == 0) {
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int v = 0; v < 4; ++v) S[mt][nt][v] = E[mt][nt][v] = 0.f;
        }
        cp_wait<CB_STAGES - 2>();
        __syncthreads();                                   // raw stage f landed; R planes free
        {
            const float *src = raw + (size_t)(f % CB_STAGES) * CB_RAW;
#pragma unroll
            for (int u = 0; u < 8; ++u) {                  // 16 row pairs x 64 columns
                const int q = tid + u * CB_THREADS;
                const int j = q >> 6, c = q & 63;
                unsigned s3[3];
                split3(src[(2 * j) * CB_N + c], src[(2 * j + 1) * CB_N + c], s3);
#pragma unroll
                for (int part = 0; part < 3; ++part) rp[part * CB_PLANE + j * CB_RPP + c] = s3[part];
            }
        }
        __syncthreads();                                   // R planes ready
        if (f + CB_STAGES - 1 < total) load(f + CB_STAGES - 1);
        cp_commit();
#pragma unroll
        for (int kk = 0; kk < CB_K; kk += 16) {
            unsigned b[2][3][2];
#pragma unroll
            for (int part = 0; part < 3; ++part)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const unsigned *P = rp + part * CB_PLANE + (kk / 2 + t) * CB_RPP + wn + nt * 8 + g;
                    b[nt][part][0] = P[0];
                    b[nt][part][1] = P[4 * CB_RPP];
                }
            const int kw = (ks * CB_K + kk) / 2 + t;
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                unsigned a[3][4];
#pragma unroll
                for (int part = 0; part < 3; ++part) {
                    const unsigned *P = cp + (size_t)part * 16 * MT * cpp + (mt * 16 + g) * cpp + kw;
                    a[part][0] = P[0];
                    a[part][1] = P[8 * cpp];
                    a[part][2] = P[4];
                    a[part][3] = P[8 * cpp + 4];
                }
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    float D[4] = {0.f, 0.f, 0.f, 0.f};
                    mma_split6(D, a, b[nt]);
#pragma unroll
                    for (int v = 0; v < 4; ++v) two_sum_add(S[mt][nt][v], E[mt][nt][v], D[v]);
                }
            }
        }
        if (ks == nks - 1) {
            const long long i0 = (blockIdx.x + (f / nks) * gridDim.x) * CB_N;
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int c = c0 + mt * 16 + g + ((v & 2) ? 8 : 0);
                        const long long i = i0 + wn + nt * 8 + 2 * t + (v & 1);
                        if (c < nc && i < n) {
                            float r = S[mt][nt][v] + E[mt][nt][v];
                            if (beta != 0.f) r = fmaf(beta * dw[i], Xc[(long long)c * ldx + i], r);
                            out[(long long)c * ldo + i] = r;
                        }
                    }
        }
    }
    cp_wait<0>();
}

template <int MT>
int launch_combine(const float *R1, const float *R2, int k1, int ktot, long long ldr, const float *coef, int nc,
                   long long n, float *out, long long ldo, const float *dw, const float *Xc, long long ldx,
                   float beta, cudaStream_t s)
{
    auto bytes_for = [](int kp) {
        return (CB_STAGES * CB_RAW + 3 * CB_PLANE + (size_t)3 * 16 * MT * (kp / 2 + 4)) * sizeof(float);
    };
    const int kp = (ktot + CB_K - 1) / CB_K * CB_K;
    const size_t smem = bytes_for(kp);
    static bool attr[64] = {};
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GBFWI_EINVAL;
    if (!attr[dev]) {
        GB_CUDA(cudaFuncSetAttribute(combine_tc_kernel<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bytes_for(128)));
        attr[dev] = true;
    }
    int nsm = 152, occ = 1;
    GB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, combine_tc_kernel<MT>, CB_THREADS, smem));
    const long long ntiles = (n + CB_N - 1) / CB_N;
    const int ny = (nc + 63) / 64;
    const int gx = (int)std::max<long long>(1, std::min<long long>(ntiles, (long long)nsm * std::max(occ, 1) / ny));
    combine_tc_kernel<MT><<<dim3(gx, ny), CB_THREADS, smem, s>>>(R1, R2, k1, ktot, ldr, coef, nc, n, out, ldo, dw,
                                                                 Xc, ldx, beta);
    GB_LAUNCHED();
    return GBFWI_OK;
}

// CTAs of atb_tc_kernel resident per SM on the current device (one wave of
// splits fills the GPU)
int atb_occupancy(int *nsm_out, int *occ_out)
{
    static int occ_of[64] = {}, nsm_of[64] = {};
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GBFWI_EINVAL;
    if (!occ_of[dev]) {
        GB_CUDA(cudaFuncSetAttribute(atb_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AT_SMEM));
        int nsm = 152, occ = 1;
        GB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, atb_tc_kernel, AT_THREADS, AT_SMEM));
        nsm_of[dev] = nsm;
        occ_of[dev] = std::max(occ, 1);
    }
    *nsm_out = nsm_of[dev];
    *occ_out = occ_of[dev];
    return GBFWI_OK;
}

}  // namespace

long long gb_tc_atb_splits(int ka, int kb, long long n)
{
    int nsm = 152, occ = 1;
    if (atb_occupancy(&nsm, &occ) != GBFWI_OK) return -1;
    const long long tiles = (long long)((kb + AT_N - 1) / AT_N) * ((ka + AT_M - 1) / AT_M);
    // one wave of CTAs, each split at least 8 K steps long
    long long nsplit = std::max<long long>(1, std::min<long long>((long long)nsm * occ / tiles, n / (8 * AT_K)));
    const long long chunk = ((n + nsplit - 1) / nsplit + AT_K - 1) / AT_K * AT_K;
    return (n + chunk - 1) / chunk;
}

int gb_tc_atb(const float *A1, const float *A2, int ka1, int ka, const float *B1, const float *B2, int kb1, int kb,
              long long ld, long long n, double *part, size_t part_doubles, double *out, long long ldo,
              cudaStream_t s)
{
    if (ka < 1 || kb < 1 || n < 1) return GBFWI_OK;
    if (ld % 4 != 0 || ((uintptr_t)A1 & 15) || ((uintptr_t)A2 & 15) || ((uintptr_t)B1 & 15) || ((uintptr_t)B2 & 15))
        return GBFWI_EINVAL;
    const long long nsplit0 = gb_tc_atb_splits(ka, kb, n);
    if (nsplit0 < 1) return GBFWI_ECUDA;
    const long long chunk = ((n + nsplit0 - 1) / nsplit0 + AT_K - 1) / AT_K * AT_K;
    const long long nsplit = (n + chunk - 1) / chunk;
    if ((size_t)nsplit * ka * kb > part_doubles) return GBFWI_EINVAL;
    const int gx = (kb + AT_N - 1) / AT_N, gy = (ka + AT_M - 1) / AT_M;
    atb_tc_kernel<<<dim3(gx, gy, (unsigned)nsplit), AT_THREADS, AT_SMEM, s>>>(A1, A2, ka1, ka, B1, B2, kb1, kb, ld, n,
                                                                            chunk, part);
    GB_LAUNCHED();
    const int nab = ka * kb;
    split_reduce_kernel<<<(nab + 255) / 256, 256, 0, s>>>(part, (int)nsplit, ka, kb, out, ldo);
    GB_LAUNCHED();
    return GBFWI_OK;
}

int gb_tc_combine(const float *R1, const float *R2, int k1, int ktot, long long ldr, const float *coef, int nc,
                  long long n, float *out, long long ldo, const float *dw, const float *Xc, long long ldx,
                  float beta, cudaStream_t s)
{
    if (nc < 1 || n < 1) return GBFWI_OK;
    if (ktot < 1 || ktot > 128 || ldr % 4 != 0 || ((uintptr_t)R1 & 15) || ((uintptr_t)R2 & 15))
        return GBFWI_EINVAL;
    const int m = std::min(nc, 64);
    if (m <= 16) return launch_combine<1>(R1, R2, k1, ktot, ldr, coef, nc, n, out, ldo, dw, Xc, ldx, beta, s);
    if (m <= 32) return launch_combine<2>(R1, R2, k1, ktot, ldr, coef, nc, n, out, ldo, dw, Xc, ldx, beta, s);
    return launch_combine<4>(R1, R2, k1, ktot, ldr, coef, nc, n, out, ldo, dw, Xc, ldx, beta, s);
}
