// adjoint_tma.cu -- the adjoint sweep nu^k -> nu^(k-1) with bulk-copy staging.
//
// Same arithmetic as adjoint_kernel (adjoint.cu; derivation there), same data
// movement as sweep_tma_kernel: per work unit (rows of one z-plane of one
// member) a producer warp copies into a shared-memory stage
//   * the 7 source row-blocks of u^(k-1) in the forward pull pattern
//     (population i from the node upstream of i), and
//   * the 7 row-blocks of nu^k in the transposed pattern (population J from
//     its consumer, the node downstream of J; at a face the wrapped row, or
//     for a mirror the own row of the opposite plane),
//   * the mask bytes,
// completing on a "full" mbarrier; consumer warps compute and release the
// stage on an "empty" mbarrier.  Own-site values of planes 3..6 (membrane
// links in y and z) are read from global memory at the start of the unit.
// Every wait is bounded; a timed-out wait sets the step control's error word.
#include "lbmbt_internal.cuh"
#include "sweep_common.cuh"
#include "tma_common.cuh"

namespace lbmbt {
namespace {

constexpr int ADJ_MAX_STAGES = 4;
constexpr int ADJ_SLOTS = 16;                  // gradient slots per unit (>= consumer warps)

__host__ __device__ __forceinline__ size_t adj_stage_bytes(int cap)
{
    return ((size_t)14 * (cap + 2) * sizeof(float2) + cap + 127) / 128 * 128;
}

// Stage one time level into 7 slots (slot i at slot0 + i (cap + 2)).
// transposed = false: forward pull pattern; true: transposed pattern.
__device__ void stage_level(const MemberDesc& d, const UnitGeo& G, const float2* lvl, bool transposed, float2* slot0,
                            int cap, uint64_t* bar)
{
    const long long nx = d.nx, ny = d.ny, nz = d.nz, sxy = nx * ny;
    const long long L = (long long)G.rows * nx, s0 = G.s0;
    const int z = G.z, y0 = G.y0, rows = G.rows;
    const size_t P = (size_t)d.plane;
    const uint32_t rowb = (uint32_t)(nx * sizeof(float2)), Lb = (uint32_t)(L * sizeof(float2));
    auto pl = [&](int i) { return lvl + (size_t)i * P; };
    auto slot = [&](int i) { return slot0 + (size_t)i * (cap + 2); };
    bulk_g2s(slot(0), pl(0) + s0, Lb, bar);
    // x: upstream pattern [s0-2, s0+L), downstream pattern [s0, s0+L+2)
    bulk_g2s(slot(1), pl(1) + (transposed ? s0 : s0 - 2), Lb + 16, bar);
    bulk_g2s(slot(2), pl(2) + (transposed ? s0 - 2 : s0), Lb + 16, bar);
    auto stage_y = [&](float2* dst, bool up, int pm, int pmir) {
        if (up) {   // rows y0-1 .. y0+rows-2
            if (y0 >= 1) {
                bulk_g2s(dst, pl(pm) + s0 - nx, Lb, bar);
            } else {
                const float2* face = d.bc[1] == BC_PER ? pl(pm) + z * sxy + (ny - 1) * nx : pl(pmir) + s0;
                bulk_g2s(dst, face, rowb, bar);
                if (rows > 1) bulk_g2s(dst + nx, pl(pm) + s0, Lb - rowb, bar);
            }
        } else {    // rows y0+1 .. y0+rows
            if (y0 + rows <= ny - 1) {
                bulk_g2s(dst, pl(pm) + s0 + nx, Lb, bar);
            } else {
                if (rows > 1) bulk_g2s(dst, pl(pm) + s0 + nx, Lb - rowb, bar);
                const long long last = s0 + (long long)(rows - 1) * nx;
                const float2* face = d.bc[1] == BC_PER ? pl(pm) + z * sxy : pl(pmir) + last;
                bulk_g2s(dst + (rows - 1) * nx, face, rowb, bar);
            }
        }
    };
    auto stage_z = [&](float2* dst, bool up, int pm, int pmir) {
        const float2* src;
        if (up) src = z >= 1 ? pl(pm) + s0 - sxy : (d.bc[2] == BC_PER ? pl(pm) + s0 + (nz - 1) * sxy : pl(pmir) + s0);
        else src = z <= nz - 2 ? pl(pm) + s0 + sxy : (d.bc[2] == BC_PER ? pl(pm) + (long long)y0 * nx : pl(pmir) + s0);
        bulk_g2s(dst, src, Lb, bar);
    };
    stage_y(slot(3), !transposed, 3, 4);
    stage_y(slot(4), transposed, 4, 3);
    stage_z(slot(5), !transposed, 5, 6);
    stage_z(slot(6), transposed, 6, 5);
}

__device__ __forceinline__ uint32_t level_bytes(long long L) { return (uint32_t)(7 * L * 8 + 32); }

// Boundary treatment of a transposed pull across a face: periodic -> times
// conj(fac of the wrapped consumer); mirror -> as the forward mirror rule.
__device__ __forceinline__ float2 adj_fix(float2 v, int bc, float2 f_per, float2 f_mir)
{
    if (bc == BC_PER) return cmul(v, make_float2(f_per.x, -f_per.y));
    return face_fix(v, bc, f_mir);
}

// ADJ_CONSUMERS consumer threads x ADJ_SPT sites cover a unit of <= 512 sites.
template <int ADJ_CONSUMERS, int ADJ_SPT>
__global__ void __launch_bounds__(ADJ_CONSUMERS + 32, 1)
    adjoint_tma_kernel(const AdjointArgs a, long long n_units, int cap, int nst)
{
    constexpr int ADJ_WARPS = ADJ_CONSUMERS / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t full[ADJ_MAX_STAGES];
    __shared__ uint64_t empty[ADJ_MAX_STAGES];
    __shared__ UnitGeo infos[ADJ_MAX_STAGES];
    __shared__ int s_abort;

    const size_t stb = adj_stage_bytes(cap);
    const int tid = threadIdx.x;
    auto unit_of = [&](long long j) { return blockIdx.x + j * (long long)gridDim.x; };

    if (tid == 0) {
        for (int st = 0; st < nst; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], ADJ_WARPS);
        }
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    if (tid >= ADJ_CONSUMERS) {
        // ---------------- producer warp (lane 0 issues)
        if (tid != ADJ_CONSUMERS) return;
        long long j = 0;
        int st = 0;          // j % nst and (j / nst) & 1, kept by increments (no division per unit)
        uint32_t ph = 0;
        for (;; ++j, st = st + 1 == nst ? 0 : st + 1, ph = st == 0 ? ph ^ 1u : ph) {
            const long long u = unit_of(j);
            if (u >= n_units || s_abort) break;
            if (j >= nst && !mbar_wait(&empty[st], ph ^ 1u)) {
                s_abort = 1;
                break;
            }
            fence_proxy_async_smem();
            const UnitGeo G = unit_geo(a.members, a.unit_start, a.n_members, u, true);
            infos[st] = G;
            const MemberDesc& d = a.members[G.m];
            const long long L = (long long)G.rows * d.nx;
            unsigned char* sb = smem + st * stb;
            float2* slots = reinterpret_cast<float2*>(sb);
            mbar_arrive_expect_tx(&full[st], level_bytes(L) * (a.first ? 1u : 2u) + (uint32_t)L);
            const size_t lv = (size_t)7 * d.plane;
            stage_level(d, G, d.state + (size_t)a.fwd_slot * lv, false, slots, cap, &full[st]);
            if (!a.first)
                stage_level(d, G, d.adj + (size_t)a.lam_parity * lv, true, slots + (size_t)7 * (cap + 2), cap,
                            &full[st]);
            bulk_g2s(sb + (size_t)14 * (cap + 2) * sizeof(float2), d.mask + G.s0, (uint32_t)L, &full[st]);
        }
        for (long long q = j - 1; q >= 0 && q >= j - nst; --q)
            mbar_wait(&full[q % nst], (uint32_t)((q / nst) & 1));
        if (s_abort) atomicOr(&a.ctl_err[0], 1);
        return;
    }

    // ---------------- consumer warps
    const int warp = tid >> 5, lane = tid & 31;
    const float fk = a.fprev;
    // Gradient partials stay in registers over the CTA's consecutive units of
    // one member (a run) and go, warp-reduced, to the slot of (the run's first
    // unit, warp): the unit-to-CTA map is fixed, so every step adds the same
    // groups in the same order.
    float acc[NGACC];
#pragma unroll
    for (int q = 0; q < NGACC; ++q) acc[q] = 0.f;
    long long u_run = -1;
    int m_run = -1;
    // constants of the current member, reloaded only when the member changes
    const MemberDesc* __restrict__ sd = a.members;
    int nx = 1, ny = 1, nz = 1, bcx = 0, bcy = 0, bcz = 0, ax = 0, rmode = 0, ds0 = 0;
    unsigned P = 0, dm0 = 0;
    float sh = 0.f;
    float2 sL = make_float2(0.f, 0.f);
    auto flush = [&]() {
#pragma unroll
        for (int q = 0; q < NGACC; ++q)
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
        if (lane == 0) {
            double* g = a.gacc + ((size_t)u_run * ADJ_SLOTS + warp) * NGACC;
#pragma unroll
            for (int q = 0; q < NGACC; ++q) g[q] += (double)acc[q];
        }
#pragma unroll
        for (int q = 0; q < NGACC; ++q) acc[q] = 0.f;
    };
    int st = 0;              // i % nst and (i / nst) & 1, kept by increments
    uint32_t ph = 0;
    for (long long i = 0;; ++i, st = st + 1 == nst ? 0 : st + 1, ph = st == 0 ? ph ^ 1u : ph) {
        const long long u = unit_of(i);
        if (u >= n_units) break;
        // warp-uniform, so the warp's lanes leave the loop together
        if (!__all_sync(0xffffffffu, mbar_wait(&full[st], ph))) {
            s_abort = 1;
            break;
        }
        const UnitGeo G = infos[st];
        if (G.m != m_run) {
            if (m_run >= 0) flush();
            m_run = G.m;
            u_run = u;
            sd = a.members + G.m;
            nx = sd->nx; ny = sd->ny; nz = sd->nz;
            bcx = sd->bc[0]; bcy = sd->bc[1]; bcz = sd->bc[2];
            P = (unsigned)sd->plane;
            dm0 = sd->div_m[0]; ds0 = sd->div_s[0];
            sh = sd->s_share;
            ax = sd->axes;
            const bool tab = sd->etab != nullptr && (fk == 1.f || fk == -1.f);
            rmode = fk == 0.f ? 0 : !tab ? 3 : (ax == 1 || ax == 2 || ax == 4) ? 1 : 2;
            if (a.first) {
                const double2 Ld = a.lam_init[G.m];
                sL = make_float2((float)Ld.x, (float)Ld.y);
            }
        }
        unsigned char* sb = smem + st * stb;
        const float2* __restrict__ U = reinterpret_cast<const float2*>(sb);
        const float2* __restrict__ V = U + (size_t)7 * (cap + 2);
        const uint8_t* __restrict__ rm = sb + (size_t)14 * (cap + 2) * sizeof(float2);
        auto Us = [&](int i2) { return U + (size_t)i2 * (cap + 2); };
        auto Vs = [&](int i2) { return V + (size_t)i2 * (cap + 2); };
        const float2* __restrict__ ug = sd->state + (size_t)a.fwd_slot * 7 * P;
        const float2* __restrict__ vg = sd->adj + (size_t)a.lam_parity * 7 * P;
        float2* __restrict__ out = sd->adj + (size_t)(a.lam_parity ^ 1) * 7 * P;
        const float2* __restrict__ facP = a.ftab + ((size_t)(a.k - 1) * a.n_members + G.m) * 6;
        const float2* __restrict__ facK = a.ftab + ((size_t)a.k * a.n_members + G.m) * 6;
        const float2* __restrict__ et = sd->etab;
        // reaction rotation form of the member (values as rotation_m1): 0
        // none (f = 0), 1 one table entry (G on one axis), 2 x and y entries
        // per site and the z entry per unit, 3 general
        const float2* __restrict__ rbase = et + (ax == 1 ? 0 : ax == 2 ? nx : nx + ny + G.z);
        const int rcx = ax == 1, rcy = ax == 2;
        const float2 ez = rmode == 2 ? __ldg(et + nx + ny + G.z) : make_float2(0.f, 0.f);

        // own-site values of planes 3..6 for membrane links in y and z
        float2 ou[ADJ_SPT][4], ov[ADJ_SPT][4];
#pragma unroll
        for (int j = 0; j < ADJ_SPT; ++j) {
            const int l = tid + j * ADJ_CONSUMERS;
            if (l < G.rows * nx) {
                const unsigned mk = rm[l];
                const unsigned s = G.s0 + (unsigned)l;
                if (mk & 0x3cu) {
                    if (mk & 4u) { ou[j][0] = __ldg(ug + (size_t)3 * P + s); if (!a.first) ov[j][1] = __ldg(vg + (size_t)4 * P + s); }
                    if (mk & 8u) { ou[j][1] = __ldg(ug + (size_t)4 * P + s); if (!a.first) ov[j][0] = __ldg(vg + (size_t)3 * P + s); }
                    if (mk & 16u) { ou[j][2] = __ldg(ug + (size_t)5 * P + s); if (!a.first) ov[j][3] = __ldg(vg + (size_t)6 * P + s); }
                    if (mk & 32u) { ou[j][3] = __ldg(ug + (size_t)6 * P + s); if (!a.first) ov[j][2] = __ldg(vg + (size_t)5 * P + s); }
                }
            }
        }

#pragma unroll
        for (int j = 0; j < ADJ_SPT; ++j) {
            const int l = tid + j * ADJ_CONSUMERS;
            if (l >= G.rows * nx) break;
            const int r = G.rows == 1 ? 0 : (int)fdiv((unsigned)l, dm0, ds0);
            const int x = l - r * nx, y = G.y0 + r, z = G.z;
            const unsigned s = G.s0 + (unsigned)l;
            const unsigned mk = rm[l];
            const int ph = mk >> 6;

            // forward recompute of g'^(k-1) from u^(k-1) (forward pull pattern)
            float2 gp[Q];
            gp[0] = Us(0)[l];
            if (x == 0) gp[1] = bcx == BC_PER ? cmul(Us(1)[l + nx + 1], __ldg(facP + 0)) : face_fix(Us(2)[l], bcx, __ldg(facP + 0));
            else gp[1] = Us(1)[l + 1];
            if (x == nx - 1) gp[2] = bcx == BC_PER ? cmul(Us(2)[l - nx + 1], __ldg(facP + 1)) : face_fix(Us(1)[l + 2], bcx, __ldg(facP + 1));
            else gp[2] = Us(2)[l + 1];
            gp[3] = Us(3)[l];
            if (y == 0) gp[3] = face_fix(gp[3], bcy, __ldg(facP + 2));
            gp[4] = Us(4)[l];
            if (y == ny - 1) gp[4] = face_fix(gp[4], bcy, __ldg(facP + 3));
            gp[5] = Us(5)[l];
            if (z == 0) gp[5] = face_fix(gp[5], bcz, __ldg(facP + 4));
            gp[6] = Us(6)[l];
            if (z == nz - 1) gp[6] = face_fix(gp[6], bcz, __ldg(facP + 5));
            // pre-mix values and own values on membrane links (kept for d/d s)
            float2 vpre[Q], own[Q];
            if (mk & 0x3fu) {
#pragma unroll
                for (int i2 = 1; i2 < Q; ++i2) vpre[i2] = gp[i2];
                own[1] = Us(2)[l];
                own[2] = Us(1)[l + 2];
                own[3] = ou[j][1];
                own[4] = ou[j][0];
                own[5] = ou[j][3];
                own[6] = ou[j][2];
                if (mk & 2u) gp[1] = mix(own[1], gp[1], sh);
                if (mk & 1u) gp[2] = mix(own[2], gp[2], sh);
                if (mk & 8u) gp[3] = mix(own[3], gp[3], sh);
                if (mk & 4u) gp[4] = mix(own[4], gp[4], sh);
                if (mk & 32u) gp[5] = mix(own[5], gp[5], sh);
                if (mk & 16u) gp[6] = mix(own[6], gp[6], sh);
            }
            const float ep = __ldg(sd->eps + ph);   // the member's values, L1-resident
            float2 rot;
            if (rmode == 0) {
                rot = make_float2(0.f, 0.f);
            } else if (rmode == 1) {
                rot = __ldg(rbase + x * rcx + y * rcy);
                if (fk < 0.f) rot.y = -rot.y;
            } else if (rmode == 2) {
                rot = cadd_prod(cadd_prod(__ldg(et + x), __ldg(et + nx + y)), ez);
                if (fk < 0.f) rot.y = -rot.y;
            } else {
                rot = rotation_m1(sd, fk, x, y, z);
            }
            const float2 q = reaction_q(rot, ep);

            // lambda^k (transposed pattern from nu^k)
            float2 lam[Q];
            if (a.first) {
#pragma unroll
                for (int i2 = 0; i2 < Q; ++i2) lam[i2] = sL;
            } else {
                lam[0] = Vs(0)[l];
                if (x == nx - 1) lam[1] = bcx == BC_PER ? cmul(Vs(1)[l - nx + 1], make_float2(__ldg(facK + 0).x, -__ldg(facK + 0).y))
                                                        : face_fix(Vs(2)[l + 2], bcx, __ldg(facK + 1));
                else lam[1] = Vs(1)[l + 1];
                if (x == 0) lam[2] = bcx == BC_PER ? cmul(Vs(2)[l + nx + 1], make_float2(__ldg(facK + 1).x, -__ldg(facK + 1).y))
                                                   : face_fix(Vs(1)[l], bcx, __ldg(facK + 0));
                else lam[2] = Vs(2)[l + 1];
                lam[3] = Vs(3)[l];
                if (y == ny - 1) lam[3] = adj_fix(lam[3], bcy, __ldg(facK + 2), __ldg(facK + 3));
                lam[4] = Vs(4)[l];
                if (y == 0) lam[4] = adj_fix(lam[4], bcy, __ldg(facK + 3), __ldg(facK + 2));
                lam[5] = Vs(5)[l];
                if (z == nz - 1) lam[5] = adj_fix(lam[5], bcz, __ldg(facK + 4), __ldg(facK + 5));
                lam[6] = Vs(6)[l];
                if (z == 0) lam[6] = adj_fix(lam[6], bcz, __ldg(facK + 5), __ldg(facK + 4));
                if (mk & 0x3fu) {   // membrane link (y, y + e_J): bit J-1, own nu_Jbar
                    if (mk & 1u) lam[1] = mix(Vs(2)[l + 2], lam[1], sh);
                    if (mk & 2u) lam[2] = mix(Vs(1)[l], lam[2], sh);
                    if (mk & 4u) lam[3] = mix(ov[j][1], lam[3], sh);
                    if (mk & 8u) lam[4] = mix(ov[j][0], lam[4], sh);
                    if (mk & 16u) lam[5] = mix(ov[j][3], lam[5], sh);
                    if (mk & 32u) lam[6] = mix(ov[j][2], lam[6], sh);
                }
            }

            // The step's reacted populations g_i = (1 + q) g'_i and mu = C^T lambda
            // enter only through sums over i: Sg = sum g'_i (M = (1 + q) Sg),
            // D = sum conj(lambda_i) g'_i (sum <lambda_i, g_i> = Re((1 + q) D)) and
            // lw = sum w_i lambda_i (mu_i = (1 - omega) lambda_i + omega lw).
            float sgr = 0.f, sgi = 0.f, dr = 0.f, di = 0.f, lwr = 0.f, lwi = 0.f;
#pragma unroll
            for (int i2 = 0; i2 < Q; ++i2) {
                const float w = i2 == 0 ? W0 : WI;
                sgr += gp[i2].x;
                sgi += gp[i2].y;
                dr += lam[i2].x * gp[i2].x + lam[i2].y * gp[i2].y;
                di += lam[i2].x * gp[i2].y - lam[i2].y * gp[i2].x;
                lwr += w * lam[i2].x;
                lwi += w * lam[i2].y;
            }
            const float q1r = 1.f + q.x, q1i = q.y;
            const float Mr = q1r * sgr - q1i * sgi, Mi = q1r * sgi + q1i * sgr;
            // d/d omega: sum_i <lambda_i, w_i M - g_i> = Re(conj(lw) M) - Re((1 + q) D)
            const float dOm = (lwr * Mr + lwi * Mi) - (q1r * dr - q1i * di);
            const float om = __ldg(sd->omega + ph), om1 = 1.f - om;
            const float er = 1.f + rot.x, ei = rot.y;
            // d/d eps: -Re(exp(i theta) c), c = sum_i conj(mu_i) g'_i = (1 - omega) D + omega conj(lw) Sg
            const float cr = om1 * dr + om * (lwr * sgr + lwi * sgi);
            const float ci = om1 * di + om * (lwr * sgi - lwi * sgr);
            const float dEp = -(er * cr - ei * ci);
            // nu_i = conj(1 + q) mu_i = a lambda_i + b, a = conj(1 + q)(1 - omega),
            // b = conj(1 + q) omega lw
            const float ar = q1r * om1, ai = -q1i * om1;
            const float br = om * (q1r * lwr + q1i * lwi), bi = om * (q1r * lwi - q1i * lwr);
#pragma unroll
            for (int i2 = 0; i2 < Q; ++i2) {
                const float2 l = lam[i2];
                lam[i2] = make_float2(ar * l.x - ai * l.y + br, ar * l.y + ai * l.x + bi);
                __stcs(out + (size_t)i2 * P + s, lam[i2]);
            }
            // d/d s on membrane links of step k-1: <nu_i, v_i - o_i>
            float dS = 0.f;
            if (mk & 0x3fu) {
                const unsigned bitof[Q] = {0u, 2u, 1u, 8u, 4u, 32u, 16u};
#pragma unroll
                for (int i2 = 1; i2 < Q; ++i2)
                    if (mk & bitof[i2])
                        dS += lam[i2].x * (vpre[i2].x - own[i2].x) + lam[i2].y * (vpre[i2].y - own[i2].y);
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                acc[p] += (ph == p) ? dOm : 0.f;
                acc[4 + p] += (ph == p) ? dEp : 0.f;
            }
            acc[8] += dS;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
    }
    if (m_run >= 0) flush();
    if (s_abort && tid == 0) atomicOr(&a.ctl_err[0], 1);
}

}  // namespace

int adj_tma_slots_per_unit() { return ADJ_SLOTS; }
// units of <= 512 sites (shapes 0, 1) or <= 480 (shape 2)
int adj_tma_max_sites(int shape) { return shape == 2 ? 480 : 512; }

// shape 0: 8 consumer warps x 2 sites (168 registers); 1: 16 x 1 (96
// registers: with the producer, 17 warps put 5 on one of the SM's four
// register-file partitions); 2: 15 x 1 (16 warps, 4 a partition: 127
// registers, no spills)
static void* adj_kernel(int shape)
{
    return shape == 1   ? (void*)adjoint_tma_kernel<512, 1>
           : shape == 2 ? (void*)adjoint_tma_kernel<480, 1>
                        : (void*)adjoint_tma_kernel<256, 2>;
}
static int adj_threads(int shape) { return shape == 1 ? 544 : shape == 2 ? 512 : 288; }

cudaError_t adj_tma_prepare(int cap, int nst, int shape, int* ctas_per_sm)
{
    const size_t bytes = adj_stage_bytes(cap) * nst;
    cudaError_t e = cudaFuncSetAttribute(adj_kernel(shape), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, adj_kernel(shape), adj_threads(shape), bytes);
}

cudaError_t launch_adjoint_tma(const AdjointArgs& a, long long n_units, int cap, int nst, int shape, int grid,
                               cudaStream_t st)
{
    if (nst < 2 || nst > ADJ_MAX_STAGES) return cudaErrorInvalidValue;
    const size_t sm = adj_stage_bytes(cap) * nst;
    if (shape == 1) adjoint_tma_kernel<512, 1><<<grid, 544, sm, st>>>(a, n_units, cap, nst);
    else if (shape == 2) adjoint_tma_kernel<480, 1><<<grid, 512, sm, st>>>(a, n_units, cap, nst);
    else adjoint_tma_kernel<256, 2><<<grid, 288, sm, st>>>(a, n_units, cap, nst);
    return cudaGetLastError();
}

}  // namespace lbmbt
