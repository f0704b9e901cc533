// Blackwell (sm_100 family) tensor-core helpers written as inline PTX: tensor
// memory (TMEM) allocation, shared-memory matrix descriptors, tcgen05.mma of
// kind::f16 (BF16 x BF16 -> FP32 in TMEM), tcgen05.commit to an mbarrier,
// tcgen05.ld of accumulator rows, the proxy fences, thread-block cluster
// barriers and distributed shared memory, and 4-byte cp.async staging.
//
// Operand layout (both A and B "K-major", no swizzle): an R x K tile of BF16 is
// stored as 8 x 8 core matrices of 128 contiguous bytes (8 rows of 16 bytes);
// core matrix (r/8, k/8) starts at (r/8) * (K/8) * 128 + (k/8) * 128 bytes, so the
// leading-dimension byte offset (between core matrices along K) is 128 and the
// stride-dimension byte offset (between 8-row groups) is (K/8) * 128.
//
// An "MN-major" operand (instruction-descriptor bit 15 for A, 16 for B) has the
// M (or N) index contiguous instead: a core matrix is 8 consecutive K rows of 8
// consecutive M/N elements (16 bytes each); the leading-dimension byte offset is
// then the stride between core matrices along K and the stride-dimension byte
// offset the stride between core matrices along M/N. A buffer of per-row records
// (row r holding elements c) in K-major core matrices can therefore feed a
// contraction over r directly, read as MN-major, without being transposed.
#pragma once
#include <stdint.h>

namespace cva {
namespace umma {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (r, k) in an R x K canonical tile
__host__ __device__ __forceinline__ uint32_t kmajor_offset(uint32_t r, uint32_t k, uint32_t K)
{
    return (r >> 3) * (K >> 3) * 128u + (k >> 3) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

// shared-memory matrix descriptor, no swizzle, version bits 46-48 = 0b001
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    return d;
}

// instruction descriptor: kind::f16, A = B = BF16, D = FP32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16_f32(uint32_t M, uint32_t N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

constexpr uint32_t kMnMajorA = 1u << 15, kMnMajorB = 1u << 16;

// instruction descriptor: kind::tf32, A = B = TF32, D = FP32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32_f32(uint32_t M, uint32_t N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// byte offset of 4-byte element (r, k) in an R x K canonical tile (core matrices of
// 8 rows x 16 bytes = 4 elements along K)
__host__ __device__ __forceinline__ uint32_t kmajor_offset32(uint32_t r, uint32_t k, uint32_t K)
{
    return (r >> 3) * (K >> 2) * 128u + (k >> 2) * 128u + (r & 7u) * 16u + (k & 3u) * 4u;
}

// x rounded to TF32 (10 explicit mantissa bits, nearest, ties away), in a 32-bit container
__device__ __forceinline__ float tf32_round(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void tmem_alloc(uint32_t *smem_result, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_result)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem desc] * B[smem desc]^T, issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// D[tmem] (+)= A[smem desc] * B[smem desc]^T with TF32 operands, issued by one thread
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive on the mbarrier once every previously issued tcgen05.mma of this thread completes
__device__ __forceinline__ void commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make generic-proxy shared-memory writes visible to the tensor-core (async) proxy
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Wait until the mbarrier phase with parity `phase` completes; gives up after
// `max_iter` polls and returns false (the caller records the timeout).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase, uint32_t max_iter)
{
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < max_iter; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 lanes x 32 bits, 16 consecutive columns: thread t of the warp receives TMEM
// lane (warp's quarter base + t), columns [col, col + 16).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 64 consecutive columns (four x16 loads in flight, one wait). The empty asm
// statements after the wait tie every value to it, so that no use of a loaded
// register can be scheduled before the load has completed.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64])
{
    float a[16], b[16], c[16], d[16];
    tmem_ld16(taddr, a);
    tmem_ld16(taddr + 16u, b);
    tmem_ld16(taddr + 32u, c);
    tmem_ld16(taddr + 48u, d);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        v[i] = a[i];
        v[16 + i] = b[i];
        v[32 + i] = c[i];
        v[48 + i] = d[i];
    }
#pragma unroll
    for (int i = 0; i < 64; ++i) asm volatile("" : "+f"(v[i]));
}

// ---- bulk asynchronous copies global -> shared, completing on an mbarrier ----
// the mbarrier's current phase expects `bytes` more transaction bytes (one arrival)
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// `bytes` (a multiple of 16) from 16-byte aligned global `src` to 16-byte aligned
// shared address `dst` of this CTA; completes `bytes` transactions on `bar`
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// `bytes` (a multiple of 16) from this CTA's 16-byte aligned shared address `src` to
// the 16-byte aligned shared::cluster address `dst` (another CTA's shared memory, from
// map_rank); completes `bytes` transactions on the mbarrier at shared::cluster address
// `bar` (in the CTA that owns `dst`)
__device__ __forceinline__ void bulk_s2c(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst),
                 "r"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// 2-D tiled TMA load: the box of the tensor map at coordinates (x, y) (x innermost;
// x * element size a multiple of 16 bytes) into 128-byte aligned shared address
// `dst`; completes the box's bytes on `bar`. `tmap` is the generic address of a
// CUtensorMap in kernel-parameter (grid-constant) memory.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int32_t x, int32_t y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// ---- thread-block clusters: rank, size, barrier, distributed shared memory ----
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_size()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// all threads of all CTAs of the cluster; shared-memory writes before it (local or
// remote) are visible to every CTA after it
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// address in CTA `rank`'s shared memory of the same offset as the local address `saddr`
__device__ __forceinline__ uint32_t map_rank(uint32_t saddr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

// no memory clobber: consecutive remote loads stay in flight together; the
// cluster barriers (which clobber memory) order them against the writes
__device__ __forceinline__ float ld_cluster_f32(uint32_t addr)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// 16-byte forms (addr 16-byte aligned)
__device__ __forceinline__ float4 ld_cluster_f32x4(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}

__device__ __forceinline__ void st_cluster_f32x4(uint32_t addr, float4 v)
{
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

// ---- asynchronous global -> shared copies of 4 bytes (per-thread staging) ----
__device__ __forceinline__ void cp_async4(uint32_t saddr, const void *g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace umma
}  // namespace cva
