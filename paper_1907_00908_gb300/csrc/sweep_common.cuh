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
// fac[a][0] is the low-face factor, fac[a][1] the high-face factor.
__device__ __forceinline__ void boundary_factors(const MemberDesc& sd, double F, float2 fac[3][2])
{
    const int dims[3] = {sd.nx, sd.ny, sd.nz};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        float2 lo = make_float2(1.f, 0.f), hi = lo;
        const double g = sd.gG[ax] * sd.dx * F;
        if (g != 0.0) {
            double sn, cs;
            if (sd.bc[ax] == BC_PER) {
                sincos(g * dims[ax], &sn, &cs);
                lo = make_float2((float)cs, (float)sn);
                hi = make_float2((float)cs, (float)-sn);
            } else if (sd.bc[ax] == BC_MIR_CONJ) {
                sincos(g, &sn, &cs);
                lo = make_float2((float)cs, (float)sn);
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
// Crossing the low face (+ direction at coord 0) uses fac = sfac[AX][0],
// the high face uses sfac[AX][1]:
//   periodic : value from the wrapped node times exp(+-i gamma L G F_k)
//   mirror   : hat g_ibar of the node itself (G parallel to the face), or its
//              conjugate times exp(-i psi) (G normal to the face)
template <int AX, int SIGN>
__device__ __forceinline__ float2 pull(const float2* __restrict__ src, unsigned P, unsigned s, int coord,
                                       int dim, unsigned stride, int bc, float2 fac)
{
    constexpr int I = 1 + 2 * AX + (SIGN > 0 ? 0 : 1);
    constexpr int IB = (SIGN > 0) ? I + 1 : I - 1;
    const bool cr = (SIGN > 0) ? (coord == 0) : (coord == dim - 1);
    unsigned nb = (SIGN > 0) ? s - stride : s + stride;
    int pl = I;
    if (cr) {
        if (bc == BC_PER) nb = (SIGN > 0) ? s + (unsigned)(dim - 1) * stride : s - (unsigned)(dim - 1) * stride;
        else { nb = s; pl = IB; }
    }
    float2 v = __ldg(src + (size_t)pl * P + nb);
    if (cr && bc != BC_MIR) {
        if (bc == BC_MIR_CONJ) v.y = -v.y;
        v = cmul(v, fac);
    }
    return v;
}

}  // namespace
}  // namespace lbmbt
