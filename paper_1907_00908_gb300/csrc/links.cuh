// links.cuh -- membranes at given positions on the links (theta = 0,
// Eqs. B4a-B4c with the coefficients of Eqs. c_n and c_d) and, on one-plane
// D2Q5 grids, at given angles (the general-angle rule of Appendix B):
// second-neighbour reads with the outer-face transforms, the combinations,
// and the arriving population of one listed link.  Used by the register
// sweep only.
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
// Population p at the node (xo + ox, yo + oy) of a one-plane grid, the node
// possibly beyond periodic faces of both axes (at most one period away):
// the wrapped node times the wrap factor of each face crossed.
__device__ __forceinline__ float2 read_2d(const float2* __restrict__ src, unsigned P, int nx, int ny, int p, int x,
                                          int y, const float2* __restrict__ fac)
{
    float2 f = make_float2(1.f, 0.f);
    bool wr = false;
    if (x < 0) { x += nx; f = __ldg(fac + 0); wr = true; }
    else if (x >= nx) { x -= nx; f = __ldg(fac + 1); wr = true; }
    if (y < 0) { y += ny; f = wr ? cmul(f, __ldg(fac + 2)) : __ldg(fac + 2); }
    else if (y >= ny) { y -= ny; f = wr ? cmul(f, __ldg(fac + 3)) : __ldg(fac + 3); }
    const float2 v = __ldg(src + (size_t)p * P + (unsigned)(y * nx + x));
    return cmul(v, f);
}

__device__ __forceinline__ unsigned mask_2d(const uint8_t* __restrict__ mask, int nx, int ny, int x, int y)
{
    x = x < 0 ? x + nx : x >= nx ? x - nx : x;
    y = y < 0 ? y + ny : y >= ny ? y - ny : y;
    return __ldg(mask + (unsigned)(y * nx + x));
}

// General-angle rule (2-D, Appendix B) for population i arriving at (xo, yo)
// across the membrane on its link to y = x - e_i, Delta_m = dl, angle th
// (normal from x's compartment to y's = cos th e_ib + sin th e_perp, e_perp =
// +y for x links, +x for y links; beta = sign(th) e_perp).  a, b are the
// theta = 0 rule's values (hat g_ib(x), hat g_ib(x + e_i), hat g_i(x)) and
// (hat g_i(y), hat g_i(y - e_i), hat g_ib(y)).  The values at the membrane
// point x_m and at x_m -+ e_beta come from quadratic extrapolation along the
// link over the three nearest nodes of each side.  With Sn, Sd (S*n, S*d) the
// Neumann and Dirichlet sums of Eqs. neumann_1, dirichlet_1 (their far-side
// forms), Tp, Tq the Neumann-minus-Dirichlet sums at Delta_m = 0 along beta
// (Eqs. phi_1, phi_2), r' = c'_n4 / c'_d4 and Ki, Ke the brackets of Eqs.
// phi_1, phi_2, the relations give
//   X = (R0 + r' V) c_n4 / Ki,    R0 = Tp st / c'_d4 - (Sn - Sd) st / c_d4 + Ki Sn / c_n4
//   V (1 + rho r' (c_n4 / (c_d4 Ki) + c*_n4 / (c*_d4 Ke)))
//     = rho (Sd / c_d4 - S*d / c*_d4) - rho c_n4 R0 / (c_d4 Ki) + rho c*_n4 R1 / (c*_d4 Ke)
// with R1 the far side's R0 and V = (dt/dx) Phi_n (Eqs. B1, B1.5).  Returns
// false (theta = 0 rule) when a stencil node lies in another compartment or
// beyond a mirror face, or when an axis is shorter than 4 nodes.
__device__ __noinline__ bool angled_population(const MemberDesc* __restrict__ sd, const float2* __restrict__ src,
                                               const float2* __restrict__ fac, int xo, int yo, int i, float dl,
                                               float th, float2 a0, float2 a1, float2 a2, float2 b0, float2 b1,
                                               float2 b2, float2* out)
{
    const int nx = sd->nx, ny = sd->ny;
    if (nx < 4 || ny < 4) return false;
    const unsigned P = (unsigned)sd->plane;
    const uint8_t* __restrict__ mask = sd->mask;
    const int ax = (i - 1) >> 1, e = (i & 1) ? 1 : -1, ib = (i & 1) ? i + 1 : i - 1;
    const int sb = th > 0.f ? 1 : -1;
    // beta along the other axis: directions 1/2 (+-x) or 3/4 (+-y)
    const int bet = ax == 0 ? (sb > 0 ? 3 : 4) : (sb > 0 ? 1 : 2);
    const int bbar = (bet & 1) ? bet + 1 : bet - 1;
    // node at (link offset k, beta offset h) from x: coordinates
    const int lx = ax == 0 ? e : 0, ly = ax == 0 ? 0 : e;         // e_i
    const int px = ax == 0 ? 0 : sb, py = ax == 0 ? sb : 0;       // e_beta
    // stencil: link offsets -3 .. 2, beta offsets -1 .. 1; no mirror face
    {
        const int cl = ax == 0 ? xo : yo, dl_ = ax == 0 ? nx : ny, cp = ax == 0 ? yo : xo, dp = ax == 0 ? ny : nx;
        const int bl = sd->bc[ax], bp = sd->bc[1 - ax];
        const int lo = min(cl + 2 * e, cl - 3 * e), hi = max(cl + 2 * e, cl - 3 * e);
        if (bl != BC_PER && (lo < 0 || hi >= dl_)) return false;
        if (bp != BC_PER && (cp - 1 < 0 || cp + 1 >= dp)) return false;
    }
    // compartments, by chains of links without membrane bits:
    // x + e_i -> x + 2 e_i; x -> x - e_beta -> + e_i -> + 2 e_i;
    // y - e_i -> y - 2 e_i; y -> y + e_beta -> - e_i -> - 2 e_i  (y = x - e_i)
    const unsigned bi = 1u << (i - 1), bib = 1u << (ib - 1);
    const unsigned mx = mask_2d(mask, nx, ny, xo, yo);
    const unsigned my = mask_2d(mask, nx, ny, xo - lx, yo - ly);
    if (mask_2d(mask, nx, ny, xo + lx, yo + ly) & bi) return false;
    if (mx & (1u << (bbar - 1))) return false;
    if (mask_2d(mask, nx, ny, xo - px, yo - py) & bi) return false;
    if (mask_2d(mask, nx, ny, xo - px + lx, yo - py + ly) & bi) return false;
    if (mask_2d(mask, nx, ny, xo - 2 * lx, yo - 2 * ly) & bib) return false;
    if (my & (1u << (bet - 1))) return false;
    if (mask_2d(mask, nx, ny, xo + px - lx, yo + py - ly) & bib) return false;
    if (mask_2d(mask, nx, ny, xo + px - 2 * lx, yo + py - 2 * ly) & bib) return false;

    // quadratic extrapolation weights (nodes 0, 1, 2 steps in, point t out)
    const float ti = dl, te = 1.f - dl;
    const float wi0 = 0.5f * (1.f + ti) * (2.f + ti), wi1 = -ti * (2.f + ti), wi2 = 0.5f * ti * (1.f + ti);
    const float we0 = 0.5f * (1.f + te) * (2.f + te), we1 = -te * (2.f + te), we2 = 0.5f * te * (1.f + te);
    auto ext_x = [&](int p, int h) {   // x side, shifted by h e_beta
        const float2 u0 = read_2d(src, P, nx, ny, p, xo + h * px, yo + h * py, fac);
        const float2 u1 = read_2d(src, P, nx, ny, p, xo + h * px + lx, yo + h * py + ly, fac);
        const float2 u2 = read_2d(src, P, nx, ny, p, xo + h * px + 2 * lx, yo + h * py + 2 * ly, fac);
        return make_float2(wi0 * u0.x + wi1 * u1.x + wi2 * u2.x, wi0 * u0.y + wi1 * u1.y + wi2 * u2.y);
    };
    auto ext_y = [&](int p, int h) {   // y side, shifted by h e_beta
        const float2 u0 = read_2d(src, P, nx, ny, p, xo + h * px - lx, yo + h * py - ly, fac);
        const float2 u1 = read_2d(src, P, nx, ny, p, xo + h * px - 2 * lx, yo + h * py - 2 * ly, fac);
        const float2 u2 = read_2d(src, P, nx, ny, p, xo + h * px - 3 * lx, yo + h * py - 3 * ly, fac);
        return make_float2(we0 * u0.x + we1 * u1.x + we2 * u2.x, we0 * u0.y + we1 * u1.y + we2 * u2.y);
    };
    // Delta_m = 0: c'_n - c'_d = (3, 2, 1), c'_n4 = 2, c'_d4 = 3
    const float2 p0 = ext_x(bet, 0), p1 = ext_x(bet, -1), p2 = ext_x(bbar, 0);
    const float2 q0 = ext_y(bbar, 0), q1 = ext_y(bbar, 1), q2 = ext_y(bet, 0);
    const float2 Tp = make_float2(3.f * p0.x + 2.f * p1.x + p2.x, 3.f * p0.y + 2.f * p1.y + p2.y);
    const float2 Tq = make_float2(3.f * q0.x + 2.f * q1.x + q2.x, 3.f * q0.y + 2.f * q1.y + q2.y);

    const float ds = 1.f - dl;
    const float q = 1.f / (2.f * dl + 1.f), qs = 1.f / (2.f * ds + 1.f);
    const float u = 2.f * dl - 1.f, us = 2.f * ds - 1.f;
    const float cn1 = -u * q, cn2 = u * q, cn3 = 2.f * q;
    const float cd0 = 2.f * (dl - 1.f), cd1 = -u * u * q, cd2 = 2.f * u * q, cd3 = (3.f - 2.f * dl) * q;
    const float sn1 = -us * qs, sn2 = us * qs, sn3 = 2.f * qs;
    const float sd0 = 2.f * (ds - 1.f), sd1 = -us * us * qs, sd2 = 2.f * us * qs, sd3 = (3.f - 2.f * ds) * qs;
    const float2 Sn = make_float2(a0.x + cn1 * a1.x + cn2 * a2.x, a0.y + cn1 * a1.y + cn2 * a2.y);
    const float2 Sd = make_float2(cd0 * a0.x + cd1 * a1.x + cd2 * a2.x, cd0 * a0.y + cd1 * a1.y + cd2 * a2.y);
    const float2 Sns = make_float2(b0.x + sn1 * b1.x + sn2 * b2.x, b0.y + sn1 * b1.y + sn2 * b2.y);
    const float2 Sds = make_float2(sd0 * b0.x + sd1 * b1.x + sd2 * b2.x, sd0 * b0.y + sd1 * b1.y + sd2 * b2.y);
    float st, ct;
    sincosf(th, &st, &ct);
    st = fabsf(st);
    const float rp = 2.f / 3.f, rho = sd->lrho;
    const float Ki = cn3 / cd3 * st + rp * ct, Ke = sn3 / sd3 * st + rp * ct;
    // R0, R1 (complex), then V and X
    const float k1 = st / 3.f, k2 = st / cd3, k3 = Ki / cn3, k4 = st / sd3, k5 = Ke / sn3;
    const float2 R0 = make_float2(k1 * Tp.x - k2 * (Sn.x - Sd.x) + k3 * Sn.x, k1 * Tp.y - k2 * (Sn.y - Sd.y) + k3 * Sn.y);
    const float2 R1 = make_float2(k1 * Tq.x - k4 * (Sns.x - Sds.x) + k5 * Sns.x,
                                  k1 * Tq.y - k4 * (Sns.y - Sds.y) + k5 * Sns.y);
    const float hi_ = cn3 / (cd3 * Ki), he = sn3 / (sd3 * Ke);
    const float den = 1.f / (1.f + rho * rp * (hi_ + he));
    const float2 V = make_float2(rho * (Sd.x / cd3 - Sds.x / sd3 - hi_ * R0.x + he * R1.x) * den,
                                 rho * (Sd.y / cd3 - Sds.y / sd3 - hi_ * R0.y + he * R1.y) * den);
    const float g = cn3 / Ki;
    *out = make_float2((R0.x + rp * V.x) * g, (R0.y + rp * V.y) * g);
    return true;
}

template <bool ANG>
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
    if (ANG && sd->dth != nullptr) {   // a batch member may have positions without angles
        const float th = __ldg(sd->dth + (size_t)(ib - 1) * P + so);
        float2 r;
        if (th != 0.f && angled_population(sd, src, fac, xo, yo, i, dl, th, own_ib, vb, own_i, v1, vf, wy, &r))
            return r;
    }
    return link_combine(dl, sd->lrho, own_ib, vb, own_i, v1, vf, wy);
}

}  // namespace
}  // namespace lbmbt
