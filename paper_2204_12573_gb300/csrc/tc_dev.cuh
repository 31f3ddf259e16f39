// Device helpers of the tensor-core kernels (tcgen05 + TMA + mbarrier, sm_103a):
// shared-memory addresses, bounded mbarrier waits, 2-D tensor loads,
// shared-memory matrix descriptors, MMA issue and commit, and tensor-memory
// loads and stores of 16 columns of a warp's lane quarter.
//
// Every wait here is bounded by a deadline on %globaltimer (kDeadlineNs) or
// by an abort flag another role sets, so a kernel that loses a signal
// returns instead of hanging.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace flr {
namespace tc {

constexpr unsigned long long kDeadlineNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false on timeout or when another role already aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > kDeadlineNs) return false;
    }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
// 2-D tensor store from shared memory (bulk group of the issuing thread)
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(src), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void tma_store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of this thread's committed stores have been read
__device__ __forceinline__ void tma_store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// ... and their global writes have completed
__device__ __forceinline__ void tma_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused with swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)2 << 61;                           // 128-byte swizzle
    return d;
}
template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    if (BF16)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// store 16 columns of this warp's TMEM lane quarter (one row per thread);
// tmem_wait_st makes them visible to later tcgen05.ld of the same thread
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float v[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
          "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
          "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
          "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
          "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
          "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}


// shared-memory matrix descriptor: K-major, 32-byte swizzle (8-row atoms of
// 32 bytes, 256 bytes apart), for operands whose K block is 16 BF16 values
__device__ __forceinline__ uint64_t sw32_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused with swizzle)
    d |= (uint64_t)(256 >> 4) << 32;                  // stride byte offset: 8-row groups
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)6 << 61;                           // 32-byte swizzle
    return d;
}
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16 columns without the wait: several loads can be in flight before one
// tmem_wait_ld()
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t r[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 8-column forms of the tensor-memory load and store (fewer live registers)
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float v[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                   "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                   "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

// The K-major A operand tile of 128 one-species rows, BF16, K = N(N+1)/2 * 4
// columns without padding: columns below 64 NA lie in 64-column atoms with
// 128-byte swizzle (8 rows x 128 bytes per swizzle block, the 16-byte chunk
// index XORed with the row within the block), the rest in 16-column blocks
// with 32-byte swizzle (8 rows x 32 bytes per block, the 16-byte half XORed
// with bit 2 of the row) -- the layouts TMA loads of 64 x 128 and 16 x 128
// boxes with those swizzles produce.  One MMA K step (16 columns) addresses
// one block.
template <int N>
struct ATile {
    static constexpr int M = 128;
    static constexpr int K = N * (N + 1) / 2 * 4;
    static constexpr int NA = K / 64;
    static constexpr int NT = (K - 64 * NA) / 16;
    static constexpr int PART = NA * M * 128 + NT * M * 32;   // bytes of the hi (or lo) part
    static constexpr int KSTEPS = K / 16;
    static_assert(PART % 1024 == 0, "A parts keep 1024-byte alignment");

    __device__ __forceinline__ static uint32_t off(int r, int c)
    {
        if (c < 64 * NA)
            return (uint32_t)((c >> 6) * (M * 128) + (r >> 3) * 1024 + (r & 7) * 128 +
                              ((((c & 63) >> 3) ^ (r & 7)) << 4) + ((c & 7) << 1));
        const int ct = c - 64 * NA;
        return (uint32_t)(NA * (M * 128) + (ct >> 4) * (M * 32) + (r >> 3) * 256 + (r & 7) * 32 +
                          ((((ct & 15) >> 3) ^ ((r >> 2) & 1)) << 4) + ((ct & 7) << 1));
    }
    // shared-memory descriptor of K step ks of a part at byte address base
    __device__ __forceinline__ static uint64_t desc(uint32_t base, int ks)
    {
        if (ks < 4 * NA) return sw128_desc(base + (uint32_t)((ks >> 2) * (M * 128) + (ks & 3) * 32));
        return sw32_desc(base + (uint32_t)(NA * (M * 128) + (ks - 4 * NA) * (M * 32)));
    }
    // 8 columns c .. c+7 of row r (c a multiple of 8), rebuilt as hi + lo
    __device__ __forceinline__ static void read_d8(const uint8_t *hi_part, const uint8_t *lo_part, int r, int c,
                                                   float v[8])
    {
        const uint32_t o = off(r, c);
        const uint4 hi = *reinterpret_cast<const uint4 *>(hi_part + o);
        const uint4 lo = *reinterpret_cast<const uint4 *>(lo_part + o);
        const uint32_t hw[4] = {hi.x, hi.y, hi.z, hi.w}, lw[4] = {lo.x, lo.y, lo.z, lo.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 fh = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&hw[k]));
            const float2 fl = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&lw[k]));
            v[2 * k] = fh.x + fl.x;
            v[2 * k + 1] = fh.y + fl.y;
        }
    }
};

}  // namespace tc
}  // namespace flr
