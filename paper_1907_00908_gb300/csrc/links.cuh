// links.cuh -- membranes at given positions on the links (theta = 0,
// Eqs. B4a-B4c with the coefficients of Eqs. c_n and c_d): second-neighbour
// reads with the outer-face transforms, the six-term combination, and the
// arriving population of one listed link.  Used by the register sweep only.
#pragma once
#include "sweep_common.cuh"

namespace lbmbt {
namespace {

// Value of population p (lying along axis a) at the node d steps along axis
// a from site s (coordinate c of dim nodes, stride between nodes), with the
// outer-boundary transforms of a node beyond a face: periodic -> the wrapped
// node times the face's wrap factor; mirror -> the node mirrored in the face
// (node -1-m mirrors m, node dim+m mirrors dim-1-m), opposite population,
// conjugated and rewound when G is normal to the face.  |d| <= 2.
__device__ __forceinline__ float2 read_along(const float2* __restrict__ src, unsigned P, unsigned s, int p, int a,
                                             int d, int c, int dim, unsigned stride, int bc_lo, int bc_hi,
                                             const float2* __restrict__ fac)
{
    const int cp = c + d;
    if (cp >= 0 && cp < dim) return __ldg(src + (size_t)p * P + (unsigned)((int)s + d * (int)stride));
    const bool lo = cp < 0;
    const int bc = lo ? bc_lo : bc_hi;
    const float2 f = __ldg(fac + 2 * a + (lo ? 0 : 1));
    if (bc == BC_PER) {
        const int dw = lo ? d + dim : d - dim;
        return cmul(__ldg(src + (size_t)p * P + (unsigned)((int)s + dw * (int)stride)), f);
    }
    const int m = lo ? -1 - cp : 2 * dim - 1 - cp;      // mirrored node
    const int pr = (p & 1) ? p + 1 : p - 1;             // opposite population
    float2 v = __ldg(src + (size_t)pr * P + (unsigned)((int)s + (m - c) * (int)stride));
    if (bc == BC_MIR) return v;
    v.y = -v.y;
    return cmul(v, f);
}

// Membrane on the link from site s towards its upstream neighbour y = s - e_i
// with the membrane at dl*dx from s (theta = 0, Eqs. B4a-B4c): the arriving
// population i is
//   A1 g_ib(s) + A2 g_ib(s + e_i) + A3 g_i(s) + B1 g_i(y) + B2 g_i(y - e_i) + B3 g_ib(y)
// (ib = opposite of i, post-collision values, each read with the outer-face
// transforms), with the coefficients from the Neumann (Eq. c_n) and Dirichlet
// (Eq. c_d) coefficients of dl and 1 - dl and rho = kappa dt / (eps_D dx).
// Used only when s + e_i lies in s's compartment and y - e_i in y's, and
// kappa is finite.
__device__ __forceinline__ float2 link_combine(float dl, float rho, float2 own_ib, float2 v_behind, float2 own_i,
                                               float2 v1, float2 v_far, float2 w_y)
{
    float cn[4], cd[4], cns[4], cds[4];
    const float ds = 1.f - dl;
    const float q = __frcp_rn(2.f * dl + 1.f), qs = __frcp_rn(2.f * ds + 1.f);
    const float u = 2.f * dl - 1.f, us = 2.f * ds - 1.f;
    cn[0] = 1.f; cn[1] = -u * q; cn[2] = u * q; cn[3] = 2.f * q;
    cd[0] = 2.f * (dl - 1.f); cd[1] = -u * u * q; cd[2] = 2.f * u * q; cd[3] = (3.f - 2.f * dl) * q;
    cns[0] = 1.f; cns[1] = -us * qs; cns[2] = us * qs; cns[3] = 2.f * qs;
    cds[0] = 2.f * (ds - 1.f); cds[1] = -us * us * qs; cds[2] = 2.f * us * qs; cds[3] = (3.f - 2.f * ds) * qs;
    const float invF = __frcp_rn(cd[3] * cds[3] + (cd[3] * cns[3] + cn[3] * cds[3]) * rho);
    float A[3], B[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        A[j] = (cd[3] * cds[3] * cn[j] + (cds[3] * cn[3] * cd[j] + cns[3] * cd[3] * cn[j]) * rho) * invF;
        B[j] = cd[3] * cn[3] * (cns[j] - cds[j]) * rho * invF;
    }
    float2 r;
    r.x = A[0] * own_ib.x + A[1] * v_behind.x + A[2] * own_i.x + B[0] * v1.x + B[1] * v_far.x + B[2] * w_y.x;
    r.y = A[0] * own_ib.y + A[1] * v_behind.y + A[2] * own_i.y + B[0] * v1.y + B[1] * v_far.y + B[2] * w_y.y;
    return r;
}

// Arriving population i at site so (coordinates xo, yo, zo) across the
// membrane on its link to y = so - e_i, at the position dl (from so): the
// position rule when so + e_i lies in so's compartment and y - e_i in y's
// (the caller checked the first, the mask byte of y decides the second),
// else the half-link rule (Eq. B5).
__device__ __forceinline__ float2 link_population(const MemberDesc* __restrict__ sd,
                                                  const float2* __restrict__ src, const float2* __restrict__ fac,
                                                  unsigned so, int xo, int yo, int zo, int i)
{
    const unsigned P = (unsigned)sd->plane;
    const int ax = (i - 1) >> 1, e = (i & 1) ? 1 : -1, ib = (i & 1) ? i + 1 : i - 1;
    const int c = ax == 0 ? xo : ax == 1 ? yo : zo;
    const int dim = ax == 0 ? sd->nx : ax == 1 ? sd->ny : sd->nz;
    const unsigned st = ax == 0 ? 1u : ax == 1 ? (unsigned)sd->nx : (unsigned)sd->nx * sd->ny;
    const int bl = ax == 2 ? sd->zbc[0] : sd->bc[ax], bh = ax == 2 ? sd->zbc[1] : sd->bc[ax];
    const int cy = c - e;   // y = so - e_i, wrapped when periodic (a membrane never crosses a mirror face)
    const unsigned sy = (unsigned)((int)so + (cy < 0 ? dim - 1 : cy >= dim ? 1 - dim : -e) * (int)st);
    const unsigned mky = __ldg(sd->mask + sy);
    const float dl = __ldg(sd->dlt + (size_t)(ib - 1) * P + so);
    const float2 own_ib = __ldg(src + (size_t)ib * P + so);
    const float2 own_i = __ldg(src + (size_t)i * P + so);
    const float2 v1 = read_along(src, P, so, i, ax, -e, c, dim, st, bl, bh, fac);        // the plain pull
    const float2 vb = read_along(src, P, so, ib, ax, e, c, dim, st, bl, bh, fac);        // g_ib(so + e_i)
    const float2 vf = read_along(src, P, so, i, ax, -2 * e, c, dim, st, bl, bh, fac);    // g_i(y - e_i)
    const float2 wy = read_along(src, P, so, ib, ax, -e, c, dim, st, bl, bh, fac);       // g_ib(y)
    if (mky & (1u << (ib - 1))) return mix(own_ib, v1, sd->s_share);
    return link_combine(dl, sd->lrho, own_ib, vb, own_i, v1, vf, wy);
}

}  // namespace
}  // namespace lbmbt
