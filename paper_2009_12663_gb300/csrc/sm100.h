// Blackwell (sm_100 family) building blocks in inline PTX: mbarriers, bulk
// asynchronous copies (TMA unit), and the 5th-generation tensor cores
// (tcgen05: MMA with operands in shared memory and the accumulator in tensor
// memory, TMEM).  Internal to the gbfwi library.
//
// Operand layout used with tcgen05.mma here: K-major tiles of bfloat16 with
// the 128-byte swizzle.  A tile holds R rows (M or N index) of 64 elements
// (128 bytes) of K; rows are 128 bytes apart, the 16-byte chunk c of row r is
// stored at chunk c ^ (r % 8), and the tile base is 1024-byte aligned (8-row
// swizzle atoms 1024 bytes apart).  The K = 16 slice kk of the tile starts
// 32 kk bytes after the base.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sm100 {

// bound of a device-side wait: about one second at the SM clock
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// ---------------------------------------------------------------------------
// mbarrier
// ---------------------------------------------------------------------------

__device__ __forceinline__ void mbar_init(unsigned long long *mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// the calling thread's arrival, announcing `bytes` of copies
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *mbar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *mbar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// wait for the phase with the given parity to complete; false when the bound ran out
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *mbar, unsigned parity)
{
    if (mbar_try_wait(mbar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

// ---------------------------------------------------------------------------
// bulk copies
// ---------------------------------------------------------------------------

// global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned), completing on mbar
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(mbar))
                 : "memory");
}

// 2-D tensor-map load of the box at (x, y) (x: innermost element index, a
// multiple of 16 bytes' worth) into dst, completing on mbar; the map lives in
// kernel-parameter or constant memory (a __grid_constant__ parameter)
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y, unsigned long long *mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_addr(mbar))
        : "memory");
}

// ---------------------------------------------------------------------------
// tcgen05
// ---------------------------------------------------------------------------

// instruction descriptor of kind::f16 with bfloat16 A and B, FP32
// accumulator, both operands K-major, shape M x N
__host__ __device__ constexpr unsigned idesc_bf16_f32(int M, int N)
{
    return (1u << 4)                           // accumulator format F32
           | (1u << 7)                         // A format BF16
           | (1u << 10)                        // B format BF16
           | ((unsigned)(N >> 3) << 17)        // N / 8
           | ((unsigned)(M >> 4) << 24);       // M / 16
}

// shared-memory descriptor of a K-major, 128-byte-swizzled bfloat16 tile
// (see the header comment); tile_base 1024-byte aligned
__device__ __forceinline__ unsigned long long sdesc_k128(const void *tile_base)
{
    const unsigned long long start = (smem_addr(tile_base) >> 4) & 0x3FFFu;
    return start                               // start address / 16
           | (1ull << 16)                      // leading-dimension byte offset (unused with this swizzle)
           | (64ull << 32)                     // stride between 8-row atoms: 1024 B / 16
           | (1ull << 46)                      // descriptor version of sm_100
           | (2ull << 61);                     // layout: 128-byte swizzle
}

// byte offset of element (r, k) in a K-major 128-byte-swizzled bfloat16 tile
__device__ __forceinline__ unsigned k128_offset(int r, int k)
{
    return (unsigned)r * 128u + ((((unsigned)k >> 3) ^ ((unsigned)r & 7u)) << 4) + ((unsigned)k & 7u) * 2u;
}

// TMEM allocation of ncols columns (power of two, 32..512) by one whole warp;
// the address is written to *slot (shared memory)
__device__ __forceinline__ void tmem_alloc(unsigned *slot, unsigned ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] B[smem]^T, issued by one thread
__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long adesc, unsigned long long bdesc,
                                         unsigned idesc, bool accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((unsigned)accumulate)
        : "memory");
}

// arrive on mbar once every tcgen05.mma issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(unsigned long long *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes of shared memory made visible to the tensor core
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of the warp's 32 TMEM lanes, waited for: thread
// t gets lane (taddr lane + t), columns taddr col .. + 15 (the wait sits in
// the same asm block, so no use of the registers can move above it)
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16])
{
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// four loads of 16 columns (at taddr + col[i]) behind one wait
__device__ __forceinline__ void tmem_ld16x4(unsigned t0, unsigned t1, unsigned t2, unsigned t3, float (&v)[4][16])
{
    unsigned r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%64];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
        "%29, %30, %31}, [%65];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, "
        "%45, %46, %47}, [%66];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, "
        "%61, %62, %63}, [%67];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
          "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
          "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(t0), "r"(t1), "r"(t2), "r"(t3)
        : "memory");
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int i = 0; i < 16; ++i) v[k][i] = __uint_as_float(r[16 * k + i]);
}

}  // namespace sm100
