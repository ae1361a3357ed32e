// Learned diagonal preconditioner: a U-Net in bfloat16 that predicts the
// logarithm of the diagonal pseudo-Hessian (the P-maps of Eqs. 5-8) from
// the model and the acquisition, with its training (backward pass, mean
// squared loss, Adam) and inference on sm_103a.  The paper has no learned
// component; the network is the standard U-Net of Ronneberger, Fischer &
// Brox (2015): per level two 3x3 convolutions with ReLU, 2x2 average
// pooling down, nearest 2x upsampling up, skip connections concatenated
// after the upsampled features, a 1x1 output convolution.
//
// Every convolution is a dense contraction and runs on the tensor cores as
// one BF16 GEMM with FP32 accumulation (mma.sync m16n8k16, operands staged
// by cp.async and fed by ldmatrix):
//   forward        Y[co][p]     = W[co][kk] Xcol[kk][p]          (+ bias, ReLU, -> bf16)
//   input grad     dXcol[kk][p] = W^T[kk][co] G[co][p]           (then a gathering col2im)
//   weight grad    dW[co][kk]  += G[co][p] Xcol^T[p][kk]         (split over p, splits summed in order)
// with kk = c*9 + ky*3 + kx and Xcol[kk][y*W + x] = X[c][y+ky-1][x+kx-1]
// (zero outside).  The four operand layouts of these products are the
// template arguments of one kernel.  Everything around the GEMMs (im2col
// with fused upsampling and concatenation, col2im, pooling, the ReLU masks
// of the gradients, bias sums, loss, Adam, resampling) is memory-bound and
// written as plain coalesced kernels.
//
// Storage points (where values are rounded to bfloat16, round to nearest
// even): input image, weights, every ReLU activation, the average-pooled
// maps, and the masked gradients fed to the GEMMs.  The output map, the
// input-gradient sums and all parameter gradients are FP32.

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "gbfwi_internal.h"

typedef __nv_bfloat16 bf16;

namespace {

// ---------------------------------------------------------------------------
// BF16 GEMM on the tensor cores
// ---------------------------------------------------------------------------

constexpr int GBK = 32;        // k extent of a staged tile
constexpr int GPAD = 8;        // bf16 padding per shared row (ldmatrix rows on distinct banks)
constexpr int GTHREADS = 256;  // 8 warps, each owning a 32 x 32 block of C
constexpr int GSTAGES = 3;     // cp.async pipeline depth (tiles in flight + 1)

struct GemmArgs {
    const bf16 *A;
    long long lda;
    const bf16 *B;
    long long ldb;
    int M, N, K;
    int kchunk;                // k range of one split
    float *Cf;                 // FP32 output (or split partials), may be null
    bf16 *Cb;                  // bf16 output, may be null
    const float *bias;         // per row of C, may be null
    int relu;
    int accumulate;            // Cf += result
    long long ldc;
    long long split_stride;    // elements between split partials (splits > 1)
    int splits;
};

__device__ __forceinline__ void cp16(void *smem, const void *gmem, bool valid)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0));
}

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void *p)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}

__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void *p)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared tiles of one stage.  A_KM: A stored [K][M] (m contiguous), else
// [M][K]; B_NK: B stored [N][K] (k contiguous), else [K][N].
template <int BM, int BN, bool A_KM, bool B_NK>
struct GemmTile {
    static constexpr int AP = A_KM ? BM + GPAD : GBK + GPAD;     // shared row pitch (bf16)
    static constexpr int BP = B_NK ? GBK + GPAD : BN + GPAD;
    static constexpr int AE = A_KM ? GBK * AP : BM * AP;          // elements per stage
    static constexpr int BE = B_NK ? BN * BP : GBK * BP;
    static constexpr int ACH = BM * GBK / 8;                      // 16-byte chunks per stage
    static constexpr int BCH = BN * GBK / 8;
};

template <int BM, int BN, bool A_KM, bool B_NK>
__device__ __forceinline__ void gemm_stage(const GemmArgs &g, bf16 *As, bf16 *Bs, int m0, int n0, int k0, int kend)
{
    using T = GemmTile<BM, BN, A_KM, B_NK>;
    for (int q = threadIdx.x; q < T::ACH; q += GTHREADS) {
        int r, c;
        const bf16 *src;
        bool ok;
        if (A_KM) {                       // rows k, 8 m per chunk
            r = q / (BM / 8);
            c = (q % (BM / 8)) * 8;
            ok = (k0 + r < kend) && (m0 + c < g.M);
            src = g.A + (long long)(k0 + r) * g.lda + m0 + c;
        } else {                          // rows m, 8 k per chunk
            r = q / (GBK / 8);
            c = (q % (GBK / 8)) * 8;
            ok = (m0 + r < g.M) && (k0 + c < kend);
            src = g.A + (long long)(m0 + r) * g.lda + k0 + c;
        }
        cp16(As + r * T::AP + c, ok ? src : g.A, ok);
    }
    for (int q = threadIdx.x; q < T::BCH; q += GTHREADS) {
        int r, c;
        const bf16 *src;
        bool ok;
        if (B_NK) {                       // rows n, 8 k per chunk
            r = q / (GBK / 8);
            c = (q % (GBK / 8)) * 8;
            ok = (n0 + r < g.N) && (k0 + c < kend);
            src = g.B + (long long)(n0 + r) * g.ldb + k0 + c;
        } else {                          // rows k, 8 n per chunk
            r = q / (BN / 8);
            c = (q % (BN / 8)) * 8;
            ok = (k0 + r < kend) && (n0 + c < g.N);
            src = g.B + (long long)(k0 + r) * g.ldb + n0 + c;
        }
        cp16(Bs + r * T::BP + c, ok ? src : g.B, ok);
    }
    asm volatile("cp.async.commit_group;\n" ::);
}

// C tile BM x BN per CTA, warps arranged (BM/32) x (BN/32), each warp
// 2 x 4 mma tiles of 16 x 8.  Requirements (checked on the host): K % 8 == 0,
// lda, ldb multiples of 8, 16-byte aligned bases, M % 8 == 0 when A_KM,
// N % 8 == 0 when !B_NK, N even.
template <int BM, int BN, bool A_KM, bool B_NK>
__global__ void __launch_bounds__(GTHREADS) gemm_bf16_kernel(const GemmArgs g)
{
    using T = GemmTile<BM, BN, A_KM, B_NK>;
    static_assert((BM / 32) * (BN / 32) == GTHREADS / 32, "warp layout");
    extern __shared__ __align__(16) unsigned char gsm[];   // GSTAGES x (A tile, B tile)
    bf16 *As0 = reinterpret_cast<bf16 *>(gsm);
    bf16 *Bs0 = As0 + GSTAGES * T::AE;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp % (BM / 32), wn = warp / (BM / 32);
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * g.kchunk;
    const int kend = min(g.K, kbeg + g.kchunk);

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[i][j][v] = 0.f;

    // GSTAGES-deep cp.async pipeline: tiles it+1 .. it+GSTAGES-1 are in flight
    // while tile it is consumed; every iteration commits one group (empty
    // past the end) so that wait_group GSTAGES-2 always means "tile it landed"
#pragma unroll
    for (int sidx = 0; sidx < GSTAGES - 1; ++sidx) {
        const int kk0 = kbeg + sidx * GBK;
        if (kk0 < kend)
            gemm_stage<BM, BN, A_KM, B_NK>(g, As0 + sidx * T::AE, Bs0 + sidx * T::BE, m0, n0, kk0, kend);
        else
            asm volatile("cp.async.commit_group;\n" ::);
    }
    int it = 0;
    for (int k0 = kbeg; k0 < kend; k0 += GBK, ++it) {
        asm volatile("cp.async.wait_group %0;\n" ::"n"(GSTAGES - 2));
        __syncthreads();
        {
            // refill the slot consumed in the previous iteration (all threads
            // are past it: the barrier above)
            const int kn = k0 + (GSTAGES - 1) * GBK;
            const int slot = (it + GSTAGES - 1) % GSTAGES;
            if (kn < kend)
                gemm_stage<BM, BN, A_KM, B_NK>(g, As0 + slot * T::AE, Bs0 + slot * T::BE, m0, n0, kn, kend);
            else
                asm volatile("cp.async.commit_group;\n" ::);
        }
        const int cur = it % GSTAGES;
        const bf16 *as = As0 + cur * T::AE, *bs = Bs0 + cur * T::BE;
#pragma unroll
        for (int kk = 0; kk < GBK; kk += 16) {
            unsigned a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int mb = wm * 32 + i * 16;
                if (A_KM) {
                    int k = kk + (lane & 7) + ((lane >> 4) << 3);
                    int m = mb + (((lane >> 3) & 1) << 3);
                    ldsm_x4_t(a[i], as + k * T::AP + m);
                } else {
                    int m = mb + (lane & 15);
                    int k = kk + ((lane >> 4) << 3);
                    ldsm_x4(a[i], as + m * T::AP + k);
                }
            }
#pragma unroll
            for (int jb = 0; jb < 2; ++jb) {
                const int nb = wn * 32 + jb * 16;
                unsigned r[4];
                if (B_NK) {
                    int n = nb + (lane & 7) + ((lane >> 4) << 3);
                    int k = kk + (((lane >> 3) & 1) << 3);
                    ldsm_x4(r, bs + n * T::BP + k);
                } else {
                    int k = kk + (lane & 15);
                    int n = nb + ((lane >> 4) << 3);
                    ldsm_x4_t(r, bs + k * T::BP + n);
                }
                b[2 * jb][0] = r[0];
                b[2 * jb][1] = r[1];
                b[2 * jb + 1][0] = r[2];
                b[2 * jb + 1][1] = r[3];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j][0], b[j][1]);
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);

    // epilogue: thread holds rows g, g+8 and columns 2t, 2t+1 of each 16 x 8 tile
    const int gr = lane >> 2, tc = (lane & 3) * 2;
    const bool partial = g.splits > 1;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = m0 + wm * 32 + i * 16 + gr + 8 * h;
            if (m >= g.M) continue;
            const float bm = (!partial && g.bias) ? g.bias[m] : 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = n0 + wn * 32 + j * 8 + tc;
                if (n >= g.N) continue;
                float v0 = acc[i][j][2 * h] + bm, v1 = acc[i][j][2 * h + 1] + bm;
                if (partial) {
                    float2 *p = reinterpret_cast<float2 *>(g.Cf + blockIdx.z * g.split_stride + (long long)m * g.ldc + n);
                    *p = make_float2(v0, v1);
                    continue;
                }
                if (g.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                if (g.Cf) {
                    float2 *p = reinterpret_cast<float2 *>(g.Cf + (long long)m * g.ldc + n);
                    if (g.accumulate) {
                        float2 o = *p;
                        v0 += o.x;
                        v1 += o.y;
                    }
                    *p = make_float2(v0, v1);
                }
                if (g.Cb) {
                    __nv_bfloat162 o = __floats2bfloat162_rn(v0, v1);
                    *reinterpret_cast<__nv_bfloat162 *>(g.Cb + (long long)m * g.ldc + n) = o;
                }
            }
        }
}

// sum of the split partials in split order, then the epilogue of the GEMM
__global__ void gemm_reduce_kernel(const float *__restrict__ part, int splits, long long split_stride, int M, int N,
                                   long long ldc, const float *__restrict__ bias, int relu, int accumulate,
                                   float *__restrict__ Cf, bf16 *__restrict__ Cb)
{
    const long long total = (long long)M * N;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(q / N), n = (int)(q - (long long)m * N);
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[z * split_stride + (long long)m * N + n];
        if (bias) s += bias[m];
        if (relu) s = fmaxf(s, 0.f);
        if (Cf) Cf[(long long)m * ldc + n] = accumulate ? Cf[(long long)m * ldc + n] + s : s;
        if (Cb) Cb[(long long)m * ldc + n] = __float2bfloat16_rn(s);
    }
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// layout kernels
// ---------------------------------------------------------------------------

// Xcol[kk][p] = X[c][y+ky-1][x+kx-1] with kk = c*9 + ky*3 + kx, zero outside
// the image and for kk >= 9 (C1 + C2).  Channels c < C1 come from s1,
// nearest-upsampled from (H/2, W/2) when up1; the rest from s2 (the skip
// connection, concatenated after s1).  Each thread writes 8 consecutive p.
__global__ void im2col_kernel(const bf16 *__restrict__ s1, int C1, int up1, const bf16 *__restrict__ s2, int C2,
                              int H, int W, int Kp, bf16 *__restrict__ out)
{
    const long long P = (long long)H * W;
    const long long groups = (long long)Kp * (P / 8);
    const int C = C1 + C2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < groups;
         q += (long long)gridDim.x * blockDim.x) {
        const int kk = (int)(q / (P / 8));
        const long long p0 = (q - (long long)kk * (P / 8)) * 8;
        const int y = (int)(p0 / W), x0 = (int)(p0 - (long long)y * W);
        __align__(16) bf16 v[8];
        const int c = kk / 9, r = kk - 9 * c, ky = r / 3, kx = r - 3 * ky;
        const int ys = y + ky - 1;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int xs = x0 + i + kx - 1;
            bf16 val = __float2bfloat16_rn(0.f);
            if (c < C && ys >= 0 && ys < H && xs >= 0 && xs < W) {
                if (c < C1) {
                    val = up1 ? s1[((long long)c * (H / 2) + ys / 2) * (W / 2) + xs / 2]
                              : s1[((long long)c * H + ys) * W + xs];
                } else {
                    val = s2[((long long)(c - C1) * H + ys) * W + xs];
                }
            }
            v[i] = val;
        }
        *reinterpret_cast<uint4 *>(out + (long long)kk * P + p0) = *reinterpret_cast<const uint4 *>(v);
    }
}

// dX[c][y][x] = sum_{ky,kx} dXcol[c*9+ky*3+kx][(y-ky+1)*W + (x-kx+1)]
// over the taps whose output pixel lies in the image (fixed order)
__global__ void col2im_kernel(const float *__restrict__ dcol, int C, int H, int W, float *__restrict__ dX)
{
    const long long P = (long long)H * W;
    const long long total = (long long)C * P;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(q / P);
        const long long p = q - (long long)c * P;
        const int y = (int)(p / W), x = (int)(p - (long long)y * W);
        float s = 0.f;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const int yo = y - ky + 1;
            if (yo < 0 || yo >= H) continue;
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int xo = x - kx + 1;
                if (xo < 0 || xo >= W) continue;
                s += dcol[(long long)(c * 9 + ky * 3 + kx) * P + (long long)yo * W + xo];
            }
        }
        dX[q] = s;
    }
}

// out[c][y][x] = mean of in[c][2y..2y+1][2x..2x+1] (H, W of the output)
__global__ void avgpool_kernel(const bf16 *__restrict__ in, int C, int H, int W, bf16 *__restrict__ out)
{
    const long long total = (long long)C * H * W;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(q % W);
        const long long cy = q / W;
        const int y = (int)(cy % H), c = (int)(cy / H);
        const bf16 *r0 = in + ((long long)c * 2 * H + 2 * y) * (2 * W) + 2 * x;
        const bf16 *r1 = r0 + 2 * W;
        float s = (__bfloat162float(r0[0]) + __bfloat162float(r0[1])) +
                  (__bfloat162float(r1[0]) + __bfloat162float(r1[1]));
        out[q] = __float2bfloat16_rn(0.25f * s);
    }
}

// Gradient reaching a ReLU activation y [C][H][W], masked by y > 0 and
// rounded for the next GEMM:
//   g = fine (2x2 sum of a [C][2H][2W] map: upsampling adjoint)   when fine
//     + 0.25 * coarse[c][y/2][x/2]   (average-pooling adjoint)      when coarse
//     + direct[c][y][x]                                             when direct
__global__ void grad_mask_kernel(const float *__restrict__ fine, const float *__restrict__ coarse,
                                 const float *__restrict__ direct, const bf16 *__restrict__ y, int C, int H, int W,
                                 bf16 *__restrict__ out)
{
    const long long total = (long long)C * H * W;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(q % W);
        const long long cy = q / W;
        const int yy = (int)(cy % H), c = (int)(cy / H);
        float g = 0.f;
        if (fine) {
            const float *r0 = fine + ((long long)c * 2 * H + 2 * yy) * (2 * W) + 2 * x;
            const float *r1 = r0 + 2 * W;
            g += (r0[0] + r0[1]) + (r1[0] + r1[1]);
        }
        if (coarse) g += 0.25f * coarse[((long long)c * (H / 2) + yy / 2) * (W / 2) + x / 2];
        if (direct) g += direct[q];
        out[q] = __float2bfloat16_rn(__bfloat162float(y[q]) > 0.f ? g : 0.f);
    }
}

// db[m] += sum_p G[m][p]: one CTA per row, fixed-order tree
__global__ void rowsum_kernel(const bf16 *__restrict__ G, long long P, float *__restrict__ db)
{
    __shared__ float red[256];
    const int m = blockIdx.x;
    float s = 0.f;
    for (long long p = threadIdx.x; p < P; p += blockDim.x) s += __bfloat162float(G[(long long)m * P + p]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[m] += red[0];
}

__global__ void to_bf16_kernel(const float *__restrict__ in, long long n, bf16 *__restrict__ out)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        out[q] = __float2bfloat16_rn(in[q]);
}

// Mean squared error over `cout` channels of pred [cpad][P] against
// target [cout][P]: per-block partial sums (FP32 products, FP64 block sums),
// and dy [cpad][P] = gscale 2 (pred - target) / (cout P) (zero rows beyond
// cout; gscale = 1 / batch gives the gradient of the batch mean).
__global__ void mse_kernel(const float *__restrict__ pred, const float *__restrict__ target, int cout, int cpad,
                           long long P, float gscale, double *__restrict__ partial, bf16 *__restrict__ dy)
{
    __shared__ double red[256];
    const long long n = (long long)cout * P;
    const float scale = (float)(2.0 / (double)n) * gscale;
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)cpad * P;
         q += (long long)gridDim.x * blockDim.x) {
        float d = 0.f;
        if (q < n) {
            d = pred[q] - target[q];
            s += (double)d * (double)d;
        }
        dy[q] = __float2bfloat16_rn(q < n ? scale * d : 0.f);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void mse_finish_kernel(const double *__restrict__ partial, int nb, long long n, double *__restrict__ out,
                                  int *__restrict__ flag)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[b];
    s /= (double)n;
    *out = s;
    if (!isfinite(s)) *flag = 1;
}

// Adam (Kingma & Ba 2015) with bias correction; refreshes the bf16 copy
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2, bf16 *__restrict__ pb)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.f - b1) * gq;
        const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        const float pq = p[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
        p[q] = pq;
        pb[q] = __float2bfloat16_rn(pq);
    }
}

// Bilinear resampling [C][sh][sw] -> [C][dh][dw] with aligned corner
// samples; op 1 takes log(max(src, 1e-30)) before interpolating, op 2
// exponentiates the interpolated value.
__global__ void resample_kernel(const float *__restrict__ src, int C, int sh, int sw, float *__restrict__ dst, int dh,
                                int dw, int op)
{
    const long long total = (long long)C * dh * dw;
    const float ry = dh > 1 ? (float)(sh - 1) / (float)(dh - 1) : 0.f;
    const float rx = dw > 1 ? (float)(sw - 1) / (float)(dw - 1) : 0.f;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(q % dw);
        const long long ci = q / dw;
        const int i = (int)(ci % dh), c = (int)(ci / dh);
        const float y = i * ry, x = j * rx;
        const int y0 = min((int)floorf(y), sh - 1), x0 = min((int)floorf(x), sw - 1);
        const int y1 = min(y0 + 1, sh - 1), x1 = min(x0 + 1, sw - 1);
        const float fy = y - y0, fx = x - x0;
        const float *s = src + (long long)c * sh * sw;
        float a = s[(long long)y0 * sw + x0], b = s[(long long)y0 * sw + x1];
        float cc = s[(long long)y1 * sw + x0], d = s[(long long)y1 * sw + x1];
        if (op == 1) {
            a = logf(fmaxf(a, 1e-30f));
            b = logf(fmaxf(b, 1e-30f));
            cc = logf(fmaxf(cc, 1e-30f));
            d = logf(fmaxf(d, 1e-30f));
        }
        float v = (1.f - fy) * ((1.f - fx) * a + fx * b) + fy * ((1.f - fx) * cc + fx * d);
        if (op == 2) v = expf(v);
        dst[q] = v;
    }
}

// Node-grid features: vp / 4700, vs / 2700, rho / 2500 and the unnormalised
// source / receiver masks sum exp(-|x - x_s|^2 / 2 sigma^2).
__global__ void features_kernel(const float *__restrict__ rho, const float *__restrict__ vp,
                                const float *__restrict__ vs, const double *__restrict__ xs,
                                const double *__restrict__ zs, int nsrc, const double *__restrict__ rxz, int nrec,
                                const double *__restrict__ cx, const double *__restrict__ cz, int nx, int nz,
                                double inv2s2, float *__restrict__ out)
{
    const long long N = (long long)nx * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(q % nx), iz = (int)(q / nx);
        const double x = cx[ix], z = cz[iz];
        out[q] = vp[q] / 4700.f;
        out[N + q] = vs[q] / 2700.f;
        out[2 * N + q] = rho[q] / 2500.f;
        double ms = 0.0, mr = 0.0;
        for (int s = 0; s < nsrc; ++s) {
            const double dx = x - xs[s], dz = z - zs[s];
            ms += exp(-(dx * dx + dz * dz) * inv2s2);
        }
        for (int r = 0; r < nrec; ++r) {
            const double dx = x - rxz[2 * r], dz = z - rxz[2 * r + 1];
            mr += exp(-(dx * dx + dz * dz) * inv2s2);
        }
        out[3 * N + q] = (float)ms;
        out[4 * N + q] = (float)mr;
    }
}

// divide channel c of x [C][N] by its maximum (one CTA per channel)
__global__ void normalise_max_kernel(float *__restrict__ x, long long N, int c0)
{
    __shared__ float red[256];
    float *v = x + (long long)(c0 + blockIdx.x) * N;
    float mx = 0.f;
    for (long long q = threadIdx.x; q < N; q += blockDim.x) mx = fmaxf(mx, v[q]);
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    const float inv = red[0] > 0.f ? 1.f / red[0] : 0.f;
    for (long long q = threadIdx.x; q < N; q += blockDim.x) v[q] *= inv;
}

__global__ void finite_flag_kernel(const float *__restrict__ x, long long n, int *__restrict__ flag)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        if (!isfinite(x[q])) *flag = 1;
}

int grid_for(long long n, int per = 1)
{
    long long b = (n / per + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(b, 152LL * 16));
}

}  // namespace

// ---------------------------------------------------------------------------
// network handle
// ---------------------------------------------------------------------------

namespace {

constexpr int kMaxLevels = 6;

struct UnetLayer {
    int cin, cout, k;       // logical shape
    int kcp, coutp;         // padded: kcp = round8(cin k k), coutp = round8(cout)
    long long w_off, b_off; // into the flat parameter buffers
};

long long round8(long long v) { return (v + 7) / 8 * 8; }

}  // namespace

struct gbfwi_unet {
    gbfwi_unet_desc d{};
    int ch[kMaxLevels] = {};
    std::vector<UnetLayer> layers;
    long long nparam = 0;
    long long step = 0;                 // Adam steps taken
    DevBuf p32, g32, m32, v32, pb;      // master params, grads, Adam moments, bf16 copy
    DevBuf xin32, xb, tgt32;            // input (FP32 staging, bf16), target staging
    DevBuf ea[kMaxLevels], e[kMaxLevels], pl[kMaxLevels], da[kMaxLevels], dd[kMaxLevels];
    DevBuf yout, gyb;                   // output [coutp][P0] FP32, its gradient (bf16)
    DevBuf col, dcol;                   // im2col (bf16), its gradient (FP32)
    DevBuf dcat[kMaxLevels];            // gradient of the concatenated decoder input (FP32)
    DevBuf fA, fP, gb;                  // FP32 input gradients, masked bf16 gradient
    DevBuf part;                        // split-K partials
    DevBuf red, flag;                   // loss partials / result, non-finite flag
    long long part_cap = 0;
};

namespace {

long long npix(const gbfwi_unet *n, int l) { return (long long)(n->d.height >> l) * (n->d.width >> l); }

template <int BM, bool AK, bool BK>
int launch_gemm(const GemmArgs &g, cudaStream_t s)
{
    constexpr int BN = 256 * 32 / BM;
    dim3 grid((unsigned)((g.N + BN - 1) / BN), (unsigned)((g.M + BM - 1) / BM), (unsigned)g.splits);
    using T = GemmTile<BM, BN, AK, BK>;
    constexpr size_t smem = (size_t)GSTAGES * (T::AE + T::BE) * sizeof(bf16);
    static bool attr_done[64] = {};      // per device ordinal
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        GB_CUDA(cudaFuncSetAttribute(gemm_bf16_kernel<BM, BN, AK, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        attr_done[dev] = true;
    }
    gemm_bf16_kernel<BM, BN, AK, BK><<<grid, GTHREADS, smem, s>>>(g);
    GB_LAUNCHED();
    return GBFWI_OK;
}

template <int BM>
int launch_gemm_bm(const GemmArgs &g, bool a_km, bool b_nk, cudaStream_t s)
{
    if (a_km) return b_nk ? launch_gemm<BM, true, true>(g, s) : launch_gemm<BM, true, false>(g, s);
    return b_nk ? launch_gemm<BM, false, true>(g, s) : launch_gemm<BM, false, false>(g, s);
}

// C[M][N] (+)= A B (+ bias, ReLU) with A = [M][K] or [K][M] (a_km), B = [K][N]
// or [N][K] (b_nk); FP32 output Cf and/or bf16 output Cb, row pitch ldc.
int gemm(gbfwi_unet *net, const bf16 *A, long long lda, bool a_km, const bf16 *B, long long ldb, bool b_nk, int M,
         int N, int K, float *Cf, bf16 *Cb, const float *bias, int relu, int accumulate, long long ldc, cudaStream_t s)
{
    if (M < 1 || N < 1 || K < 8 || K % 8 || lda % 8 || ldb % 8 || N % 2 || ldc % 2 || ((uintptr_t)A & 15) ||
        ((uintptr_t)B & 15) || (a_km && M % 8) || (!b_nk && N % 8))
        return GBFWI_EINVAL;
    const int BM = M <= 32 ? 32 : (M <= 64 ? 64 : 128);
    const int BN = 256 * 32 / BM;
    const long long tiles = (long long)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    int splits = 1;
    if (tiles < 2 * 152 && K >= 8 * GBK) {
        long long want = (2 * 152 + tiles - 1) / tiles;
        want = std::min<long long>(want, K / (4 * GBK));
        want = std::min<long long>(want, std::max<long long>(1, net->part_cap / ((long long)M * N)));
        splits = (int)std::max<long long>(1, want);
    }
    int kchunk = (int)(((K + splits - 1) / splits + GBK - 1) / GBK * GBK);
    splits = (K + kchunk - 1) / kchunk;
    GemmArgs g{A, lda, B, ldb, M, N, K, kchunk, Cf, Cb, bias, relu, accumulate, ldc, 0, splits};
    if (splits > 1) {
        g.Cf = net->part.as<float>();
        g.Cb = nullptr;
        g.bias = nullptr;
        g.relu = 0;
        g.accumulate = 0;
        g.ldc = N;
        g.split_stride = (long long)M * N;
    }
    int rc = BM == 32 ? launch_gemm_bm<32>(g, a_km, b_nk, s)
                      : (BM == 64 ? launch_gemm_bm<64>(g, a_km, b_nk, s) : launch_gemm_bm<128>(g, a_km, b_nk, s));
    GB_TRY(rc);
    if (splits > 1) {
        gemm_reduce_kernel<<<grid_for((long long)M * N), 256, 0, s>>>(net->part.as<float>(), splits, (long long)M * N,
                                                                      M, N, ldc, bias, relu, accumulate, Cf, Cb);
        GB_LAUNCHED();
    }
    return GBFWI_OK;
}

int im2col(const bf16 *s1, int C1, int up1, const bf16 *s2, int C2, int H, int W, int Kp, bf16 *out, cudaStream_t s)
{
    im2col_kernel<<<grid_for((long long)Kp * H * W, 8), 256, 0, s>>>(s1, C1, up1, s2, C2, H, W, Kp, out);
    GB_LAUNCHED();
    return GBFWI_OK;
}

// 3x3 convolution + bias + ReLU -> bf16 output [cout][H][W]
int conv_fwd(gbfwi_unet *n, const UnetLayer &L, const bf16 *s1, int C1, int up1, const bf16 *s2, int C2, int H, int W,
             bf16 *out, cudaStream_t s)
{
    const long long P = (long long)H * W;
    GB_TRY(im2col(s1, C1, up1, s2, C2, H, W, L.kcp, n->col.as<bf16>(), s));
    return gemm(n, n->pb.as<bf16>() + L.w_off, L.kcp, false, n->col.as<bf16>(), P, false, L.cout, (int)P, L.kcp,
                nullptr, out, n->p32.as<float>() + L.b_off, 1, 0, P, s);
}

// Backward of a 3x3 convolution given its masked output gradient G
// (bf16 [cout][P]): dW, db accumulate into the gradient buffer; when dX is
// not null, the input gradient (FP32 [cin][P]) is written there.
int conv_bwd(gbfwi_unet *n, const UnetLayer &L, const bf16 *s1, int C1, int up1, const bf16 *s2, int C2, int H, int W,
             const bf16 *G, float *dX, cudaStream_t s)
{
    const long long P = (long long)H * W;
    GB_TRY(im2col(s1, C1, up1, s2, C2, H, W, L.kcp, n->col.as<bf16>(), s));
    GB_TRY(gemm(n, G, P, false, n->col.as<bf16>(), P, true, L.cout, L.kcp, (int)P, n->g32.as<float>() + L.w_off,
                nullptr, nullptr, 0, 1, L.kcp, s));
    rowsum_kernel<<<L.cout, 256, 0, s>>>(G, P, n->g32.as<float>() + L.b_off);
    GB_LAUNCHED();
    if (!dX) return GBFWI_OK;
    GB_TRY(gemm(n, n->pb.as<bf16>() + L.w_off, L.kcp, true, G, P, false, L.kcp, (int)P, L.coutp,
                n->dcol.as<float>(), nullptr, nullptr, 0, 0, P, s));
    col2im_kernel<<<grid_for((long long)L.cin * P), 256, 0, s>>>(n->dcol.as<float>(), L.cin, H, W, dX);
    GB_LAUNCHED();
    return GBFWI_OK;
}

int grad_mask(const float *fine, const float *coarse, const float *direct, const bf16 *y, int C, int H, int W,
              bf16 *out, cudaStream_t s)
{
    grad_mask_kernel<<<grid_for((long long)C * H * W), 256, 0, s>>>(fine, coarse, direct, y, C, H, W, out);
    GB_LAUNCHED();
    return GBFWI_OK;
}

// forward pass on n->xb (bf16 input already staged) -> n->yout
int net_forward(gbfwi_unet *n, cudaStream_t s)
{
    const int Lv = n->d.levels;
    int li = 0;
    for (int l = 0; l < Lv; ++l) {
        const int H = n->d.height >> l, W = n->d.width >> l;
        const bf16 *in;
        int cin;
        if (l == 0) {
            in = n->xb.as<bf16>();
            cin = n->d.cin;
        } else {
            cin = n->ch[l - 1];
            avgpool_kernel<<<grid_for((long long)cin * H * W), 256, 0, s>>>(n->e[l - 1].as<bf16>(), cin, H, W,
                                                                           n->pl[l].as<bf16>());
            GB_LAUNCHED();
            in = n->pl[l].as<bf16>();
        }
        GB_TRY(conv_fwd(n, n->layers[li++], in, cin, 0, nullptr, 0, H, W, n->ea[l].as<bf16>(), s));
        GB_TRY(conv_fwd(n, n->layers[li++], n->ea[l].as<bf16>(), n->ch[l], 0, nullptr, 0, H, W, n->e[l].as<bf16>(), s));
    }
    const bf16 *h = n->e[Lv - 1].as<bf16>();
    for (int l = Lv - 2; l >= 0; --l) {
        const int H = n->d.height >> l, W = n->d.width >> l;
        GB_TRY(conv_fwd(n, n->layers[li++], h, n->ch[l + 1], 1, n->e[l].as<bf16>(), n->ch[l], H, W,
                        n->da[l].as<bf16>(), s));
        GB_TRY(conv_fwd(n, n->layers[li++], n->da[l].as<bf16>(), n->ch[l], 0, nullptr, 0, H, W, n->dd[l].as<bf16>(), s));
        h = n->dd[l].as<bf16>();
    }
    const UnetLayer &O = n->layers[li];
    const long long P0 = npix(n, 0);
    return gemm(n, n->pb.as<bf16>() + O.w_off, O.kcp, false, h, P0, false, O.coutp, (int)P0, O.kcp,
                n->yout.as<float>(), nullptr, n->p32.as<float>() + O.b_off, 0, 0, P0, s);
}

// backward pass from the output gradient n->gyb (bf16 [coutp][P0]);
// parameter gradients accumulate into n->g32
int net_backward(gbfwi_unet *n, cudaStream_t s)
{
    const int Lv = n->d.levels;
    const long long P0 = npix(n, 0);
    int li = (int)n->layers.size() - 1;
    const UnetLayer &O = n->layers[li];
    const bf16 *top = Lv > 1 ? n->dd[0].as<bf16>() : n->e[0].as<bf16>();
    // output 1x1 convolution
    GB_TRY(gemm(n, n->gyb.as<bf16>(), P0, false, top, P0, true, O.coutp, O.kcp, (int)P0, n->g32.as<float>() + O.w_off,
                nullptr, nullptr, 0, 1, O.kcp, s));
    rowsum_kernel<<<O.coutp, 256, 0, s>>>(n->gyb.as<bf16>(), P0, n->g32.as<float>() + O.b_off);
    GB_LAUNCHED();
    GB_TRY(gemm(n, n->pb.as<bf16>() + O.w_off, O.kcp, true, n->gyb.as<bf16>(), P0, false, O.kcp, (int)P0, O.coutp,
                n->fA.as<float>(), nullptr, nullptr, 0, 0, P0, s));
    --li;
    // decoder, fine to coarse; the gradient of level l's output arrives as
    // fA (level 0) or as the upsampling adjoint of dcat[l-1]
    for (int l = 0; l <= Lv - 2; ++l) {
        const int H = n->d.height >> l, W = n->d.width >> l;
        const float *fine = l > 0 ? n->dcat[l - 1].as<float>() : nullptr;
        const float *direct = l == 0 ? n->fA.as<float>() : nullptr;
        GB_TRY(grad_mask(fine, nullptr, direct, n->dd[l].as<bf16>(), n->ch[l], H, W, n->gb.as<bf16>(), s));
        GB_TRY(conv_bwd(n, n->layers[li], n->da[l].as<bf16>(), n->ch[l], 0, nullptr, 0, H, W, n->gb.as<bf16>(),
                        n->fA.as<float>(), s));
        --li;
        GB_TRY(grad_mask(nullptr, nullptr, n->fA.as<float>(), n->da[l].as<bf16>(), n->ch[l], H, W, n->gb.as<bf16>(), s));
        const bf16 *coarse = (l + 1 <= Lv - 2) ? n->dd[l + 1].as<bf16>() : n->e[Lv - 1].as<bf16>();
        GB_TRY(conv_bwd(n, n->layers[li], coarse, n->ch[l + 1], 1, n->e[l].as<bf16>(), n->ch[l], H, W,
                        n->gb.as<bf16>(), n->dcat[l].as<float>(), s));
        --li;
    }
    // encoder, bottleneck first; the gradient of e[l] sums the decoder's
    // upsampling adjoint (bottleneck), the pooling adjoint of the level
    // below and the skip connection
    for (int l = Lv - 1; l >= 0; --l) {
        const int H = n->d.height >> l, W = n->d.width >> l;
        const long long P = (long long)H * W;
        const float *fine = nullptr, *coarse = nullptr, *direct = nullptr;
        if (l == Lv - 1) {
            if (Lv > 1)
                fine = n->dcat[Lv - 2].as<float>();
            else
                direct = n->fA.as<float>();
        } else {
            coarse = n->fP.as<float>();
            direct = n->dcat[l].as<float>() + (long long)n->ch[l + 1] * P;
        }
        GB_TRY(grad_mask(fine, coarse, direct, n->e[l].as<bf16>(), n->ch[l], H, W, n->gb.as<bf16>(), s));
        GB_TRY(conv_bwd(n, n->layers[li], n->ea[l].as<bf16>(), n->ch[l], 0, nullptr, 0, H, W, n->gb.as<bf16>(),
                        n->fA.as<float>(), s));
        --li;
        GB_TRY(grad_mask(nullptr, nullptr, n->fA.as<float>(), n->ea[l].as<bf16>(), n->ch[l], H, W, n->gb.as<bf16>(), s));
        const bf16 *in = l == 0 ? n->xb.as<bf16>() : n->pl[l].as<bf16>();
        const int cin = l == 0 ? n->d.cin : n->ch[l - 1];
        GB_TRY(conv_bwd(n, n->layers[li], in, cin, 0, nullptr, 0, H, W, n->gb.as<bf16>(),
                        l > 0 ? n->fP.as<float>() : nullptr, s));
        --li;
    }
    return GBFWI_OK;
}

int stage_input(gbfwi_unet *n, const float *x, cudaStream_t s)
{
    const long long cnt = (long long)n->d.cin * npix(n, 0);
    const float *src = x;
    if (!gb_is_device_ptr(x)) {
        GB_CUDA(cudaMemcpyAsync(n->xin32.p, x, cnt * sizeof(float), cudaMemcpyHostToDevice, s));
        src = n->xin32.as<float>();
    }
    to_bf16_kernel<<<grid_for(cnt), 256, 0, s>>>(src, cnt, n->xb.as<bf16>());
    GB_LAUNCHED();
    return GBFWI_OK;
}

int read_flag(gbfwi_unet *n, cudaStream_t s, int *out)
{
    GB_CUDA(cudaMemcpyAsync(out, n->flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    return GBFWI_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------

extern "C" int gbfwi_unet_create(const gbfwi_unet_desc *d, gbfwi_unet **out)
{
    if (!d || !out || d->levels < 1 || d->levels > kMaxLevels || d->base < 8 || d->base % 8 || d->cin < 1 ||
        d->cout < 1 || d->height < 1 || d->width < 1)
        return GBFWI_EINVAL;
    const int f = 1 << (d->levels - 1);
    if (d->height % f || d->width % (8 * f)) return GBFWI_EINVAL;
    gbfwi_unet *n = new (std::nothrow) gbfwi_unet();
    if (!n) return GBFWI_ENOMEM;
    n->d = *d;
    const int Lv = d->levels;
    for (int l = 0; l < Lv; ++l) n->ch[l] = d->base << l;
    auto add = [&](int cin, int cout, int k) {
        UnetLayer L{cin, cout, k, (int)round8((long long)cin * k * k), (int)round8(cout), 0, 0};
        L.w_off = n->nparam;
        L.b_off = L.w_off + (long long)L.coutp * L.kcp;
        n->nparam = round8(L.b_off + L.coutp);
        n->layers.push_back(L);
    };
    for (int l = 0; l < Lv; ++l) {
        add(l == 0 ? d->cin : n->ch[l - 1], n->ch[l], 3);
        add(n->ch[l], n->ch[l], 3);
    }
    for (int l = Lv - 2; l >= 0; --l) {
        add(n->ch[l + 1] + n->ch[l], n->ch[l], 3);
        add(n->ch[l], n->ch[l], 3);
    }
    add(n->ch[0], d->cout, 1);
    const long long P0 = npix(n, 0);
    long long colmax = 0, cmax = 0;
    for (int l = 0; l < Lv; ++l) cmax = std::max(cmax, (long long)n->ch[l] * npix(n, l));
    {
        int li = 0;
        for (int l = 0; l < Lv; ++l) {
            colmax = std::max(colmax, (long long)n->layers[li++].kcp * npix(n, l));
            colmax = std::max(colmax, (long long)n->layers[li++].kcp * npix(n, l));
        }
        for (int l = Lv - 2; l >= 0; --l) {
            colmax = std::max(colmax, (long long)n->layers[li++].kcp * npix(n, l));
            colmax = std::max(colmax, (long long)n->layers[li++].kcp * npix(n, l));
        }
    }
    const UnetLayer &O = n->layers.back();
    cmax = std::max(cmax, (long long)O.coutp * P0);
    n->part_cap = 32LL << 20;   // floats of split-K partials
    int rc = GBFWI_OK;
    auto need = [&](DevBuf &b, long long bytes) {
        if (!rc) rc = b.ensure((size_t)std::max<long long>(bytes, 16));
    };
    const size_t F = sizeof(float), B2 = sizeof(bf16);
    need(n->p32, n->nparam * F);
    need(n->g32, n->nparam * F);
    need(n->m32, n->nparam * F);
    need(n->v32, n->nparam * F);
    need(n->pb, n->nparam * B2);
    need(n->xin32, (long long)d->cin * P0 * F);
    need(n->xb, (long long)d->cin * P0 * B2);
    need(n->tgt32, (long long)d->cout * P0 * F);
    for (int l = 0; l < Lv; ++l) {
        const long long P = npix(n, l);
        need(n->ea[l], n->ch[l] * P * B2);
        need(n->e[l], n->ch[l] * P * B2);
        if (l > 0) need(n->pl[l], n->ch[l - 1] * P * B2);
        if (l <= Lv - 2) {
            need(n->da[l], n->ch[l] * P * B2);
            need(n->dd[l], n->ch[l] * P * B2);
            need(n->dcat[l], (long long)(n->ch[l + 1] + n->ch[l]) * P * F);
        }
    }
    need(n->yout, (long long)O.coutp * P0 * F);
    need(n->gyb, (long long)O.coutp * P0 * B2);
    need(n->col, colmax * B2);
    need(n->dcol, colmax * F);
    need(n->fA, cmax * F);
    need(n->fP, cmax * F);
    need(n->gb, cmax * B2);
    need(n->part, n->part_cap * F);
    need(n->red, 4096 * sizeof(double));
    need(n->flag, 16);
    if (rc) {
        delete n;
        return rc;
    }
    cudaMemset(n->p32.p, 0, n->nparam * F);
    cudaMemset(n->pb.p, 0, n->nparam * B2);
    cudaMemset(n->m32.p, 0, n->nparam * F);
    cudaMemset(n->v32.p, 0, n->nparam * F);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        gb_set_last_cuda_error(cudaGetLastError(), "unet init", __FILE__, __LINE__);
        delete n;
        return GBFWI_ECUDA;
    }
    *out = n;
    return GBFWI_OK;
}

extern "C" int gbfwi_unet_destroy(gbfwi_unet *n)
{
    delete n;
    return GBFWI_OK;
}

extern "C" long long gbfwi_unet_num_params(const gbfwi_unet *n) { return n ? n->nparam : GBFWI_EINVAL; }

extern "C" int gbfwi_unet_layer_info(const gbfwi_unet *n, int layer, int *info)
{
    if (!n) return GBFWI_EINVAL;
    if (layer < 0) return (int)n->layers.size();
    if (layer >= (int)n->layers.size() || !info) return GBFWI_EINVAL;
    const UnetLayer &L = n->layers[layer];
    info[0] = L.cout;
    info[1] = L.cin;
    info[2] = L.k;
    info[3] = L.coutp;
    info[4] = L.kcp;
    info[5] = (int)L.w_off;
    info[6] = (int)L.b_off;
    return GBFWI_OK;
}

extern "C" int gbfwi_unet_set_params(gbfwi_unet *n, const float *params, void *stream)
{
    if (!n || !params) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(params));
    cudaStream_t s = (cudaStream_t)stream;
    GB_CUDA(cudaMemcpyAsync(n->p32.p, params, n->nparam * sizeof(float),
                            gb_is_device_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    to_bf16_kernel<<<grid_for(n->nparam), 256, 0, s>>>(n->p32.as<float>(), n->nparam, n->pb.as<bf16>());
    GB_LAUNCHED();
    GB_CUDA(cudaMemsetAsync(n->m32.p, 0, n->nparam * sizeof(float), s));
    GB_CUDA(cudaMemsetAsync(n->v32.p, 0, n->nparam * sizeof(float), s));
    n->step = 0;
    GB_CUDA(cudaStreamSynchronize(s));
    return GBFWI_OK;
}

extern "C" int gbfwi_unet_get_params(const gbfwi_unet *n, float *params, void *stream)
{
    if (!n || !params) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(params));
    cudaStream_t s = (cudaStream_t)stream;
    GB_CUDA(cudaMemcpyAsync(params, n->p32.p, n->nparam * sizeof(float),
                            gb_is_device_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    return GBFWI_OK;
}

extern "C" int gbfwi_unet_forward(gbfwi_unet *n, const float *x, float *y, void *stream)
{
    if (!n || !x || !y) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(x, y));
    cudaStream_t s = (cudaStream_t)stream;
    const long long P0 = npix(n, 0);
    GB_TRY(stage_input(n, x, s));
    GB_TRY(net_forward(n, s));
    const long long cnt = (long long)n->d.cout * P0;
    GB_CUDA(cudaMemsetAsync(n->flag.p, 0, sizeof(int), s));
    finite_flag_kernel<<<grid_for(cnt), 256, 0, s>>>(n->yout.as<float>(), cnt, n->flag.as<int>());
    GB_LAUNCHED();
    GB_CUDA(cudaMemcpyAsync(y, n->yout.p, cnt * sizeof(float),
                            gb_is_device_ptr(y) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    int f = 0;
    GB_TRY(read_flag(n, s, &f));
    return f ? gb_nonfinite("U-Net output") : GBFWI_OK;
}

extern "C" int gbfwi_unet_gradient(gbfwi_unet *n, const float *x, const float *dy, float *grad, void *stream)
{
    if (!n || !x || !dy || !grad) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(x, dy, grad));
    cudaStream_t s = (cudaStream_t)stream;
    const long long P0 = npix(n, 0);
    const UnetLayer &O = n->layers.back();
    GB_TRY(stage_input(n, x, s));
    GB_TRY(net_forward(n, s));
    // dy [cout][P0] -> bf16 rows of the padded output gradient
    const long long cnt = (long long)n->d.cout * P0;
    const float *dys = dy;
    if (!gb_is_device_ptr(dy)) {
        GB_CUDA(cudaMemcpyAsync(n->tgt32.p, dy, cnt * sizeof(float), cudaMemcpyHostToDevice, s));
        dys = n->tgt32.as<float>();
    }
    GB_CUDA(cudaMemsetAsync(n->gyb.p, 0, (size_t)O.coutp * P0 * sizeof(bf16), s));
    to_bf16_kernel<<<grid_for(cnt), 256, 0, s>>>(dys, cnt, n->gyb.as<bf16>());
    GB_LAUNCHED();
    GB_CUDA(cudaMemsetAsync(n->g32.p, 0, n->nparam * sizeof(float), s));
    GB_TRY(net_backward(n, s));
    GB_CUDA(cudaMemcpyAsync(grad, n->g32.p, n->nparam * sizeof(float),
                            gb_is_device_ptr(grad) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    return GBFWI_OK;
}

extern "C" int gbfwi_unet_train_step(gbfwi_unet *n, const float *x, const float *target, int batch, double lr,
                                     double *loss, void *stream)
{
    if (!n || !x || !target || batch < 1 || !(lr > 0)) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(x, target));
    cudaStream_t s = (cudaStream_t)stream;
    const long long P0 = npix(n, 0);
    const UnetLayer &O = n->layers.back();
    const long long xin = (long long)n->d.cin * P0, tin = (long long)n->d.cout * P0;
    const bool dx = gb_is_device_ptr(x), dt = gb_is_device_ptr(target);
    GB_CUDA(cudaMemsetAsync(n->g32.p, 0, n->nparam * sizeof(float), s));
    GB_CUDA(cudaMemsetAsync(n->flag.p, 0, sizeof(int), s));
    const int nb = 512;
    double *partial = n->red.as<double>();
    double *lsum = partial + nb;          // per-sample losses [batch] (<= 1024)
    if (batch > 1024) return GBFWI_EINVAL;
    for (int b = 0; b < batch; ++b) {
        const float *xb = x + b * xin;
        GB_TRY(stage_input(n, xb, s));
        GB_TRY(net_forward(n, s));
        const float *tb = target + b * tin;
        if (!dt) {
            GB_CUDA(cudaMemcpyAsync(n->tgt32.p, tb, tin * sizeof(float), cudaMemcpyHostToDevice, s));
            tb = n->tgt32.as<float>();
        }
        mse_kernel<<<nb, 256, 0, s>>>(n->yout.as<float>(), tb, n->d.cout, O.coutp, P0, 1.f / (float)batch, partial,
                                      n->gyb.as<bf16>());
        GB_LAUNCHED();
        mse_finish_kernel<<<1, 32, 0, s>>>(partial, nb, tin, lsum + b, n->flag.as<int>());
        GB_LAUNCHED();
        GB_TRY(net_backward(n, s));
    }
    (void)dx;
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
    adam_kernel<<<grid_for(n->nparam), 256, 0, s>>>(n->p32.as<float>(), n->g32.as<float>(), n->m32.as<float>(),
                                                     n->v32.as<float>(), n->nparam, (float)lr, b1, b2, eps, c1, c2,
                                                     n->pb.as<bf16>());
    GB_LAUNCHED();
    std::vector<double> lh(batch);
    GB_CUDA(cudaMemcpyAsync(lh.data(), lsum, batch * sizeof(double), cudaMemcpyDeviceToHost, s));
    int f = 0;
    GB_TRY(read_flag(n, s, &f));
    if (f) return gb_nonfinite("U-Net training loss");
    double tot = 0.0;
    for (double v : lh) tot += v;
    if (loss) *loss = tot / batch;
    return GBFWI_OK;
}

extern "C" int gbfwi_resample(const float *src, int channels, int sh, int sw, float *dst, int dh, int dw, int op,
                              void *stream)
{
    if (!src || !dst || channels < 1 || sh < 1 || sw < 1 || dh < 1 || dw < 1 || op < 0 || op > 2 ||
        !gb_is_device_ptr(src) || !gb_is_device_ptr(dst))
        return GBFWI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    resample_kernel<<<grid_for((long long)channels * dh * dw), 256, 0, s>>>(src, channels, sh, sw, dst, dh, dw, op);
    GB_LAUNCHED();
    return GBFWI_OK;
}

extern "C" int gbfwi_unet_features(gbfwi_mesh *m, const float *rho, const float *vp, const float *vs, double sigma_m,
                                   int height, int width, float *x, void *stream)
{
    if (!m || !rho || !vp || !vs || !x || !(sigma_m > 0) || height < 1 || width < 1) return GBFWI_EINVAL;
    GB_TRY(gb_check_local(rho, vp, vs, x));
    cudaStream_t s = (cudaStream_t)stream;
    const int nx = m->nx, nz = m->nz;
    const long long N = (long long)nx * nz;
    const int ns = (int)m->src.size(), nr = m->nrec;
    std::vector<double> X((size_t)N), Z((size_t)N);
    GB_TRY(gbfwi_node_coords(m, X.data(), Z.data()));
    std::vector<double> tab;
    tab.reserve(nx + nz + 2 * ns + 2 * nr + 4);
    for (int i = 0; i < nx; ++i) tab.push_back(X[i]);
    for (int i = 0; i < nz; ++i) tab.push_back(Z[(size_t)i * nx]);
    for (int i = 0; i < ns; ++i) tab.push_back(m->src[i].x);
    for (int i = 0; i < ns; ++i) tab.push_back(m->src[i].z);
    for (int i = 0; i < 2 * nr; ++i) tab.push_back(m->rec_xz[i]);
    DevBuf dtab, dmod, dfeat, dout;
    GB_TRY(dtab.ensure(tab.size() * sizeof(double)));
    GB_TRY(dfeat.ensure((size_t)5 * N * sizeof(float)));
    GB_CUDA(cudaMemcpyAsync(dtab.p, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    const float *r = rho, *p = vp, *v = vs;
    if (!gb_is_device_ptr(rho) || !gb_is_device_ptr(vp) || !gb_is_device_ptr(vs)) {
        GB_TRY(dmod.ensure((size_t)3 * N * sizeof(float)));
        float *dm = dmod.as<float>();
        GB_CUDA(cudaMemcpyAsync(dm, rho, N * sizeof(float), cudaMemcpyDefault, s));
        GB_CUDA(cudaMemcpyAsync(dm + N, vp, N * sizeof(float), cudaMemcpyDefault, s));
        GB_CUDA(cudaMemcpyAsync(dm + 2 * N, vs, N * sizeof(float), cudaMemcpyDefault, s));
        r = dm;
        p = dm + N;
        v = dm + 2 * N;
    }
    const double *t = dtab.as<double>();
    features_kernel<<<grid_for(N), 256, 0, s>>>(r, p, v, t + nx + nz, t + nx + nz + ns, ns, t + nx + nz + 2 * ns, nr,
                                                t, t + nx, nx, nz, 1.0 / (2.0 * sigma_m * sigma_m), dfeat.as<float>());
    GB_LAUNCHED();
    normalise_max_kernel<<<2, 256, 0, s>>>(dfeat.as<float>(), N, 3);
    GB_LAUNCHED();
    const bool devx = gb_is_device_ptr(x);
    const long long cnt = 5LL * height * width;
    float *dst = x;
    if (!devx) {
        GB_TRY(dout.ensure(cnt * sizeof(float)));
        dst = dout.as<float>();
    }
    resample_kernel<<<grid_for(cnt), 256, 0, s>>>(dfeat.as<float>(), 5, nz, nx, dst, height, width, 0);
    GB_LAUNCHED();
    if (!devx) GB_CUDA(cudaMemcpyAsync(x, dst, cnt * sizeof(float), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    return GBFWI_OK;
}
