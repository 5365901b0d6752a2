// tma_common.cuh -- mbarrier / bulk-copy helpers and row-unit geometry shared
// by the bulk-copy forward sweep and the bulk-copy adjoint sweep.
#pragma once
#include "lbmbt_internal.cuh"
#include "sweep_common.cuh"

namespace lbmbt {
namespace {

constexpr unsigned long long WAIT_NS = 2000000000ull;  // bound of every wait: 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// try_wait with a suspend-time hint (ns): the waiting warp sleeps until the
// phase completes or the hint elapses instead of spinning on issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for one phase of an mbarrier; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns = WAIT_NS)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() - t0 > limit_ns) return false;
    return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}


__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}

// Where unit u lies: member, z-plane, first row, rows, first site, sites.
struct UnitGeo {
    int m, z, y0, rows, L;
    unsigned s0;
};

__device__ __forceinline__ UnitGeo unit_geo(const MemberDesc* __restrict__ members, const long long* __restrict__ unit_start,
                                        int n_members, long long u, bool adj = false)
{
    UnitGeo G;
    G.m = n_members == 1 ? 0 : find_member(unit_start, n_members, u);
    const MemberDesc* __restrict__ d = members + G.m;
    const int ny = d->ny, nx = d->nx, rpu = adj ? d->rpu_adj : d->rpu;
    const int lu = (int)(u - (adj ? d->unit0_adj : d->unit0));
    const int upz = (ny + rpu - 1) / rpu;
    G.z = lu / upz;
    G.y0 = (lu - G.z * upz) * rpu;
    G.rows = min(rpu, ny - G.y0);
    G.L = G.rows * nx;
    G.s0 = (unsigned)G.z * ((unsigned)nx * ny) + (unsigned)G.y0 * nx;
    return G;
}

// Boundary transform of a value pulled across a face (see pull()).
__device__ __forceinline__ float2 face_fix(float2 v, int bc, float2 f)
{
    if (bc == BC_MIR || bc == BC_HALO) return v;
    if (bc == BC_MIR_CONJ) v.y = -v.y;
    return cmul(v, f);
}

}  // namespace
}  // namespace lbmbt
