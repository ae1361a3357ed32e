// Tensor-core products of the compact BFGS apply and the randomized SVD
// (sm_103a): the tall-skinny [S B0Y]^T X-type products and the row
// combinations [S B0Y] (M W)-type of the compact form of the inverse
// Hessian (Section 2.3, Eq. 9, Algorithms 2-3; Byrd, Nocedal & Schnabel
// 1994), and the Gram / projection products of Algorithm 3.
//
// Precision.  Every operand is FP32.  Each value x is split into two TF32
// parts, hi = tf32(x) and lo = tf32(x - hi), and a product is taken as
// hi*hi + hi*lo + lo*hi on the tensor cores (mma.sync m16n8k8 TF32, FP32
// accumulation): the 3xTF32 scheme of Ootomo & Yokota (2022), whose error
// is that of an FP32 product (the dropped lo*lo term and the residual of lo
// are ~2^-22 relative).  The long sums over n of the split-K products are
// accumulated per split in a compensated FP32 pair (TwoSum of Knuth, taken
// after every 32 products of a K step), so they are close to an exact sum
// of the FP32 products, and the splits are reduced in FP64.  The row
// combinations sum at most 128 terms and keep a plain FP32 accumulator.
//
// Layout: rows are vectors of length n with a row stride ld (a multiple of
// 4 floats, rows 16-byte aligned); both kernels stage their operands in
// shared memory with 16-byte cp.async copies (zero-filled beyond n and
// beyond the last row).

#include <algorithm>

#include "gbfwi_internal.h"

namespace {

__device__ __forceinline__ unsigned tf32_of(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split_tf32(float x, unsigned &hi, unsigned &lo)
{
    hi = tf32_of(x);
    lo = tf32_of(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
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
// K staged 32 at a time, three-stage cp.async pipeline.
// grid (ceil(kb / 64), ceil(ka / 64), nsplit): the splits vary slowest, so
// the tiles that read the same K range run together and share it in L2.
// ---------------------------------------------------------------------------

constexpr int AT_M = 64, AT_N = 64, AT_K = 32, AT_P = AT_K + 4, AT_STAGES = 3, AT_THREADS = 128;
constexpr size_t AT_SMEM = (size_t)AT_STAGES * (AT_M + AT_N) * AT_P * sizeof(float);

__global__ void __launch_bounds__(AT_THREADS) atb_tc_kernel(const float *__restrict__ A1, const float *__restrict__ A2,
                                                            int ka1, int ka, const float *__restrict__ B1,
                                                            const float *__restrict__ B2, int kb1, int kb,
                                                            long long ld, long long n, long long chunk,
                                                            double *__restrict__ part)
{
    extern __shared__ float4 at_smem4[];
    float *sm = reinterpret_cast<float *>(at_smem4);
    const int sx = blockIdx.z;
    const int a0 = blockIdx.y * AT_M, b0 = blockIdx.x * AT_N;
    const long long ib = (long long)sx * chunk;
    const long long ie = min(n, ib + chunk);
    const int nk = (int)((ie - ib + AT_K - 1) / AT_K);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;

    // stage loader: 64 rows of A and 64 rows of B, 32 floats each = 8
    // 16-byte chunks per row; 1024 chunks, 8 per thread
    auto load = [&](int stage, int kt) {
        float *As = sm + (size_t)stage * (AT_M + AT_N) * AT_P;
        float *Bs = As + AT_M * AT_P;
        const long long i0 = ib + (long long)kt * AT_K;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = tid + u * AT_THREADS;           // 0..1023
            const int r = (q >> 3) & 63, c = q & 7;
            const bool isb = q >= 512;
            const int row = (isb ? b0 : a0) + r;
            const int lim = isb ? kb : ka;
            const long long i = i0 + 4 * c;
            int bytes = 0;
            const float *src = isb ? B1 : A1;
            if (row < lim && i < ie) {
                src = isb ? row_of(B1, B2, kb1, row, ld) + i : row_of(A1, A2, ka1, row, ld) + i;
                bytes = (int)min(16LL, (ie - i) * 4);
            }
            cp16((isb ? Bs : As) + r * AT_P + 4 * c, src, bytes);
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
        __syncthreads();
        if (kt + 2 < nk) load((kt + 2) % AT_STAGES, kt + 2);
        cp_commit();
        const float *As = sm + (size_t)(kt % AT_STAGES) * (AT_M + AT_N) * AT_P;
        const float *Bs = As + AT_M * AT_P;
        float D[2][4][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int v = 0; v < 4; ++v) D[mt][nt][v] = 0.f;
#pragma unroll
        for (int kk = 0; kk < AT_K; kk += 8) {
            unsigned ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const float *p = As + (wm + mt * 16 + g) * AT_P + kk + t;
                split_tf32(p[0], ah[mt][0], al[mt][0]);
                split_tf32(p[8 * AT_P], ah[mt][1], al[mt][1]);
                split_tf32(p[4], ah[mt][2], al[mt][2]);
                split_tf32(p[8 * AT_P + 4], ah[mt][3], al[mt][3]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const float *p = Bs + (wn + nt * 8 + g) * AT_P + kk + t;
                split_tf32(p[0], bh[nt][0], bl[nt][0]);
                split_tf32(p[4], bh[nt][1], bl[nt][1]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    mma_tf32(D[mt][nt], al[mt][0], al[mt][1], al[mt][2], al[mt][3], bh[nt][0], bh[nt][1]);
                    mma_tf32(D[mt][nt], ah[mt][0], ah[mt][1], ah[mt][2], ah[mt][3], bl[nt][0], bl[nt][1]);
                    mma_tf32(D[mt][nt], ah[mt][0], ah[mt][1], ah[mt][2], ah[mt][3], bh[nt][0], bh[nt][1]);
                }
        }
        // fold this K step's 32-product sums into the compensated pairs
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int v = 0; v < 4; ++v) two_sum_add(S[mt][nt][v], E[mt][nt][v], D[mt][nt][v]);
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
// coef (FP32, [nc][ktot]) stays in shared memory; persistent CTAs walk over
// 64-column tiles, streaming R in K steps of 32 rows through a four-stage
// cp.async pipeline.  4 warps, each all MT m16 tiles x 2 n8 tiles (16
// columns).
// ---------------------------------------------------------------------------

constexpr int CB_N = 64, CB_K = 32, CB_RP = CB_N + 8, CB_STAGES = 4, CB_THREADS = 128;

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
    float *sm = reinterpret_cast<float *>(cb_smem4);
    const int kp = (ktot + CB_K - 1) / CB_K * CB_K;      // K padded to whole steps
    const int cpitch = kp + 4;
    float *Cs = sm;                                      // [16 MT][cpitch]
    float *Rs = sm + 16 * MT * cpitch;                   // [stages][CB_K][CB_RP]
    const int c0 = blockIdx.y * 64;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int wn = warp * 16;
    for (int q = tid; q < 16 * MT * cpitch; q += CB_THREADS) {
        const int c = q / cpitch, a = q - c * cpitch;
        Cs[q] = (c0 + c < nc && a < ktot) ? coef[(long long)(c0 + c) * ktot + a] : 0.f;
    }
    const long long ntiles = (n + CB_N - 1) / CB_N;
    const int nks = kp / CB_K;
    // flat sequence of (tile, K step) pairs of this CTA
    const long long my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long total = my_tiles * nks;
    auto load = [&](long long f) {
        const long long tile = blockIdx.x + (f / nks) * gridDim.x;
        const int ks = (int)(f % nks);
        float *dst = Rs + (size_t)(f % CB_STAGES) * CB_K * CB_RP;
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
            cp16(dst + r * CB_RP + 4 * c, src, bytes);
        }
    };
    for (long long f = 0; f < CB_STAGES - 1; ++f) {
        if (f < total) load(f);
        cp_commit();
    }
    float D[MT][2][4];
    for (long long f = 0; f < total; ++f) {
        const int ks = (int)(f % nks);
        if (ks == 0) {
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int v = 0; v < 4; ++v) D[mt][nt][v] = 0.f;
        }
        cp_wait<CB_STAGES - 2>();
        __syncthreads();
        if (f + CB_STAGES - 1 < total) load(f + CB_STAGES - 1);
        cp_commit();
        const float *Rb = Rs + (size_t)(f % CB_STAGES) * CB_K * CB_RP;
#pragma unroll
        for (int kk = 0; kk < CB_K; kk += 8) {
            unsigned bh[2][2], bl[2][2];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const float *p = Rb + (kk + t) * CB_RP + wn + nt * 8 + g;
                split_tf32(p[0], bh[nt][0], bl[nt][0]);
                split_tf32(p[4 * CB_RP], bh[nt][1], bl[nt][1]);
            }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const float *p = Cs + (mt * 16 + g) * cpitch + ks * CB_K + kk + t;
                unsigned ah0, al0, ah1, al1, ah2, al2, ah3, al3;
                split_tf32(p[0], ah0, al0);
                split_tf32(p[8 * cpitch], ah1, al1);
                split_tf32(p[4], ah2, al2);
                split_tf32(p[8 * cpitch + 4], ah3, al3);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    mma_tf32(D[mt][nt], al0, al1, al2, al3, bh[nt][0], bh[nt][1]);
                    mma_tf32(D[mt][nt], ah0, ah1, ah2, ah3, bl[nt][0], bl[nt][1]);
                    mma_tf32(D[mt][nt], ah0, ah1, ah2, ah3, bh[nt][0], bh[nt][1]);
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
                            float r = D[mt][nt][v];
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
    const int kp = (ktot + CB_K - 1) / CB_K * CB_K;
    const size_t smem = ((size_t)16 * MT * (kp + 4) + (size_t)CB_STAGES * CB_K * CB_RP) * sizeof(float);
    const size_t smem_max = ((size_t)16 * MT * (128 + 4) + (size_t)CB_STAGES * CB_K * CB_RP) * sizeof(float);
    static bool attr[64] = {};
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GBFWI_EINVAL;
    if (!attr[dev]) {
        GB_CUDA(cudaFuncSetAttribute(combine_tc_kernel<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_max));
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
