// sweep_common.cuh -- device helpers shared by the forward sweep and the
// adjoint sweep: complex multiply, work-list lookup, the outer-boundary
// factors of one step and the pull of one D3Q7 direction.
#pragma once
#include "lbmbt_internal.cuh"

namespace lbmbt {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int find_member(const long long* __restrict__ ts, int n, long long b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(ts + mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Outer-boundary factors of one member at one step, from F_k (FP64):
//   periodic (Sec. 2.4.3, Eq. collision_BC): a population pulled across the low
//     face (from node N-1 into node 0) is multiplied by exp(+i phi), across the
//     high face by exp(-i phi), phi = gamma G_a L_a F_k, L_a = N_a dx;
//   mirror with G normal to the face (Sec. 2.4.4): the buffer value is
//     conj(hat g_ibar(x_n) exp(i psi)) with psi = gamma G_a (x_n + x_m) F_k
//     (origin x_o = 0), i.e. conj(hat g_ibar) * exp(-i psi): psi = -dx at the
//     low face, (2N-1) dx at the high face.
// For z, N is the whole grid's nzg and each face has its own mode (a slab
// face towards another slab takes the periodic factor only across the
// global face, BC_HALO_PER).
// fac[a][0] is the low-face factor, fac[a][1] the high-face factor.
__device__ __forceinline__ void boundary_factors(const MemberDesc& sd, double F, float2 fac[3][2])
{
    const int dims[3] = {sd.nx, sd.ny, sd.nzg};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        float2 lo = make_float2(1.f, 0.f), hi = lo;
        const double g = sd.gG[ax] * sd.dx * F;
        if (g != 0.0) {
            const int bl = ax == 2 ? sd.zbc[0] : sd.bc[ax];
            const int bh = ax == 2 ? sd.zbc[1] : sd.bc[ax];
            double sn, cs;
            if (bl == BC_PER || bl == BC_HALO_PER) {
                sincos(g * dims[ax], &sn, &cs);
                lo = make_float2((float)cs, (float)sn);
            } else if (bl == BC_MIR_CONJ) {
                sincos(g, &sn, &cs);
                lo = make_float2((float)cs, (float)sn);
            }
            if (bh == BC_PER || bh == BC_HALO_PER) {
                sincos(g * dims[ax], &sn, &cs);
                hi = make_float2((float)cs, (float)-sn);
            } else if (bh == BC_MIR_CONJ) {
                sincos(g * (2.0 * dims[ax] - 1.0), &sn, &cs);
                hi = make_float2((float)cs, (float)-sn);
            }
        }
        fac[ax][0] = lo;
        fac[ax][1] = hi;
    }
}

// Pull of direction I = 1 + 2*AX + (SIGN > 0 ? 0 : 1) into site s.
// SIGN = +1: direction +e_AX, the population comes from coord - 1;
// SIGN = -1: direction -e_AX, it comes from coord + 1.
// Crossing the low face (+ direction at coord 0) uses fac[2*AX], the high
// face fac[2*AX + 1] (loaded only by threads that cross):
//   periodic : value from the wrapped node times exp(+-i gamma L G F_k)
//   mirror   : hat g_ibar of the node itself (G parallel to the face), or its
//              conjugate times exp(-i psi) (G normal to the face)
//   slab face: the halo plane's value at (x, y) (times the wrap factor
//              across the periodic global face)
template <int AX, int SIGN>
__device__ __forceinline__ float2 pull(const float2* __restrict__ src, unsigned P, unsigned s, int coord,
                                       int dim, unsigned stride, int bc, const float2* __restrict__ fac,
                                       const float2* const* halo = nullptr)
{
    constexpr int I = 1 + 2 * AX + (SIGN > 0 ? 0 : 1);
    constexpr int IB = (SIGN > 0) ? I + 1 : I - 1;
    const bool cr = (SIGN > 0) ? (coord == 0) : (coord == dim - 1);
    unsigned nb = (SIGN > 0) ? s - stride : s + stride;
    int pl = I;
    float2 v;
    if (cr && (bc == BC_HALO || bc == BC_HALO_PER)) {
        v = __ldg(*halo + ((SIGN > 0) ? s : s - (unsigned)(dim - 1) * stride));   // pointer read only here
    } else {
        if (cr) {
            if (bc == BC_PER) nb = (SIGN > 0) ? s + (unsigned)(dim - 1) * stride : s - (unsigned)(dim - 1) * stride;
            else { nb = s; pl = IB; }
        }
        v = __ldg(src + (size_t)pl * P + nb);
    }
    if (cr && bc != BC_MIR && bc != BC_HALO) {
        if (bc == BC_MIR_CONJ) v.y = -v.y;
        v = cmul(v, __ldg(fac + 2 * AX + (SIGN > 0 ? 0 : 1)));
    }
    return v;
}

// Exact n / d for n < 2^28 with host-computed (m, s) (Granlund-Montgomery,
// 28-bit dividends: m = floor(2^(28+l)/d) + 1, s = 28 + l, l = ceil(log2 d)).
__device__ __forceinline__ unsigned fdiv(unsigned n, unsigned m, int s)
{
    return (unsigned)(((unsigned long long)n * m) >> s);
}

// Site coordinates of linear index s.
__device__ __forceinline__ void coords(const MemberDesc* __restrict__ d, unsigned s, int nx, int ny, int& x, int& y,
                                       int& z)
{
    const unsigned row = fdiv(s, d->div_m[0], d->div_s[0]);
    x = (int)(s - row * (unsigned)nx);
    const unsigned zz = fdiv(row, d->div_m[1], d->div_s[1]);
    z = (int)zz;
    y = (int)(row - zz * (unsigned)ny);
}

// exp(i theta) - 1 for theta = fk * sum_a ctheta_a n_a, returned as
// (cos theta - 1, sin theta).  For fk in {-1, +1} from the per-axis tables,
// combining axes by (1+u)(1+v) - 1 = u + v + u v; otherwise sincosf.  The
// arithmetic order is fixed with explicit roundings so every kernel that
// calls this gets the same bits.
__device__ __forceinline__ float2 cadd_prod(float2 u, float2 v)
{
    // u + v + u v
    const float pr = __fmaf_rn(u.x, v.x, __fmul_rn(-u.y, v.y));
    const float pi = __fmaf_rn(u.x, v.y, __fmul_rn(u.y, v.x));
    return make_float2(__fadd_rn(__fadd_rn(u.x, v.x), pr), __fadd_rn(__fadd_rn(u.y, v.y), pi));
}

__device__ __forceinline__ float2 rotation_m1(const MemberDesc* __restrict__ d, float fk, int x, int y, int z)
{
    const float2* __restrict__ et = d->etab;
    const int ax = d->axes;
    if (et != nullptr && (fk == 1.f || fk == -1.f)) {
        float2 q = make_float2(0.f, 0.f);
        bool any = false;
        if (ax & 1) { q = __ldg(et + x); any = true; }
        if (ax & 2) { const float2 v = __ldg(et + d->nx + y); q = any ? cadd_prod(q, v) : v; any = true; }
        if (ax & 4) { const float2 v = __ldg(et + d->nx + d->ny + z); q = any ? cadd_prod(q, v) : v; }
        if (fk < 0.f) q.y = -q.y;
        return q;
    }
    const float th = __fmul_rn(fk, __fmaf_rn(d->ctheta[2], (float)(z + d->z0),
                                              __fmaf_rn(d->ctheta[1], (float)y, __fmul_rn(d->ctheta[0], (float)x))));
    float sh2, ch2;
    sincosf(0.5f * th, &sh2, &ch2);
    return make_float2(__fmul_rn(-2.f, __fmul_rn(sh2, sh2)), __fmul_rn(2.f, __fmul_rn(sh2, ch2)));
}

// Reaction factor minus one, q = exp(i theta)(1 - eps) - 1, from rot = exp(i theta) - 1.
__device__ __forceinline__ float2 reaction_q(float2 rot, float ep)
{
    return make_float2(__fmaf_rn(-ep, __fadd_rn(1.f, rot.x), rot.x), __fmul_rn(rot.y, __fsub_rn(1.f, ep)));
}

// Membrane link: o + s (v - o) (Eq. B5 with r = 1 - s).
__device__ __forceinline__ float2 mix(float2 o, float2 v, float sh)
{
    return make_float2(__fmaf_rn(sh, __fsub_rn(v.x, o.x), o.x), __fmaf_rn(sh, __fsub_rn(v.y, o.y), o.y));
}

// Reaction g <- g + g q in place, with M = sum_i g_i (fixed order).
__device__ __forceinline__ void react(float2 (&g)[Q], float2 q, float& mr, float& mi)
{
    mr = 0.f;
    mi = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float gr = g[i].x, gi = g[i].y;
        g[i].x = __fmaf_rn(gr, q.x, __fmaf_rn(-gi, q.y, gr));
        g[i].y = __fmaf_rn(gi, q.x, __fmaf_rn(gr, q.y, gi));
        mr = __fadd_rn(mr, g[i].x);
        mi = __fadd_rn(mi, g[i].y);
    }
}

// BGK collision hat g = g + omega (w M - g) in place.
__device__ __forceinline__ void collide(float2 (&g)[Q], float om, float mr, float mi)
{
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float w = i == 0 ? W0 : WI;
        g[i].x = __fmaf_rn(om, __fmaf_rn(w, mr, -g[i].x), g[i].x);
        g[i].y = __fmaf_rn(om, __fmaf_rn(w, mi, -g[i].y), g[i].y);
    }
}

// collide() with the weights given at run time (w0 rest, wxy the four
// in-plane velocities, wz the two z velocities); the same operations, so
// with the D3Q7 weights it gives collide()'s bits.
__device__ __forceinline__ void collide_w(float2 (&g)[Q], float om, float mr, float mi, float w0, float wxy, float wz)
{
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float w = i == 0 ? w0 : i < 5 ? wxy : wz;
        g[i].x = __fmaf_rn(om, __fmaf_rn(w, mr, -g[i].x), g[i].x);
        g[i].y = __fmaf_rn(om, __fmaf_rn(w, mi, -g[i].y), g[i].y);
    }
}

// Classical scheme (Appendix A, Eq. A12): collision with the reaction as a
// source, hat g_i = g_i + omega (w_i M - g_i) + w_i (sr + i si), where
// (sr, si) = dt R M, R = -i gamma x.G0 f - 1/T2 (Eq. A2), M = sum_i g_i.
__device__ __forceinline__ void collide_source_w(float2 (&g)[Q], float om, float mr, float mi, float sr, float si,
                                                 float w0, float wxy, float wz)
{
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float w = i == 0 ? w0 : i < 5 ? wxy : wz;
        g[i].x = __fmaf_rn(w, sr, __fmaf_rn(om, __fmaf_rn(w, mr, -g[i].x), g[i].x));
        g[i].y = __fmaf_rn(w, si, __fmaf_rn(om, __fmaf_rn(w, mi, -g[i].y), g[i].y));
    }
}

// The reaction angle itself, theta = f * sum_a ctheta_a n_a = -gamma x.G0 f dt
// (the classical scheme's source is linear in it).
__device__ __forceinline__ float theta_lin(const MemberDesc* __restrict__ d, float fk, int x, int y, int z)
{
    return __fmul_rn(fk, __fmaf_rn(d->ctheta[2], (float)(z + d->z0),
                                   __fmaf_rn(d->ctheta[1], (float)y, __fmul_rn(d->ctheta[0], (float)x))));
}

// dt R M for R = -eps + i theta (eps = dt/T2): (-eps mr - theta mi, -eps mi + theta mr).
__device__ __forceinline__ float2 source_dtRM(float ep, float th, float mr, float mi)
{
    return make_float2(__fmaf_rn(-ep, mr, __fmul_rn(-th, mi)), __fmaf_rn(-ep, mi, __fmul_rn(th, mr)));
}

// A CTA of a persistent sweep is done with the step word: take a ticket;
// the last of the launch's `nblocks` advances the word and clears the
// counters for the next sweep (which sees both at its launch: kernel
// boundary).  Every CTA has read k before it takes its ticket, so none can
// see the new value.  One thread per CTA calls, right after a CTA barrier
// that follows every thread's read of the step control; with `fence` those
// reads are ordered before the ticket at device scope.
// The ticket has two levels, since atomics on one address serialise (about
// 7 ns each, measured: a register sweep has ~10^5 blocks a step): block b
// counts on shard b % CTL_SHARDS, and the last block of each shard counts on
// `done`.
__device__ __forceinline__ void step_done(StepCtl* ctl, int k, unsigned nblocks, bool fence)
{
    if (fence) __threadfence();
    const unsigned s = blockIdx.x % CTL_SHARDS;
    const unsigned in_shard = (nblocks - s + CTL_SHARDS - 1u) / CTL_SHARDS;   // blocks b < nblocks, b % S == s
    if (atomicAdd(&ctl->shard[s], 1u) != in_shard - 1u) return;
    ctl->shard[s] = 0u;
    const unsigned shards = nblocks < CTL_SHARDS ? nblocks : CTL_SHARDS;
    if (atomicAdd(&ctl->done, 1u) == shards - 1u) {
        ctl->done = 0u;
        ctl->k = k + 1;
    }
}

// boundary_factors() into a flat [6] array: index 2*axis + (0 low, 1 high).
__device__ __forceinline__ void boundary_factors6(const MemberDesc& sd, double F, float2* out6)
{
    float2 f[3][2];
    boundary_factors(sd, F, f);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        out6[2 * a] = f[a][0];
        out6[2 * a + 1] = f[a][1];
    }
}

}  // namespace
}  // namespace lbmbt
