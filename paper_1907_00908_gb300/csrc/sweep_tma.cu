// sweep_tma.cu -- the fused time step with bulk-copy (TMA) staging.
//
// Same arithmetic as sweep_kernel (sweep.cu), different data movement: the
// work unit is `rpu` consecutive x-rows of one z-plane of one member
// (L = rpu*nx sites).  For each unit one thread issues cp.async.bulk copies of
// the 7 source row-blocks (and the mask bytes) into a shared-memory stage;
// completion is tracked by an mbarrier (expect_tx / complete_tx).  A
// persistent CTA walks its units through a ring of 2-6 stages, filled by a
// producer warp and drained by 8 to 16 consumer warps, so the next units'
// copies are in flight while the current one is computed, without holding the
// data in registers.  A consumer first gathers the pulled populations of all
// its sites (phase 1, after which the stage is released), then reacts,
// collides and stores them with no branch between sites (phase 2), so the
// arithmetic of several sites interleaves.  The own-site values of planes
// 3 and 4 (membrane links in y) are prefetched into registers one unit
// ahead.  Those of planes 5 and 6 (membrane links in z) come in one of three
// forms, chosen per run (template parameter FORM): 0 prefetched like planes
// 3 and 4 (small planes: the rows are still in L2, and the smaller stage
// leaves more of the SM's memory to L1); 1 staged with the unit (the rows
// are otherwise first touched a whole plane later, and a load at a membrane
// lane waited on DRAM; they are read again when the neighbouring planes'
// units pull them); 2 z-marching: each CTA takes columns of zc units (the
// same rows of zc consecutive z-planes of one member) in z order.  There a
// unit stages the own rows of plane 5 in place of the rows of plane z-1,
// and every consumer keeps, per site, the plane-5 own value (the next
// unit's +z pull) and the plane-6 pull value (the next unit's own value) in
// registers, so each row is read once and no own value is loaded from
// global memory; the first unit of a column loads those two values itself.
//
// Source row-blocks of a unit starting at site s0 (all 16-byte aligned when
// nx is even; the mask copy needs nx % 16 == 0):
//   plane 0      [s0, s0+L)
//   plane 1 (+x) [s0-2, s0+L)      value for local l is at l+1, wrap at l+nx+1
//   plane 2 (-x) [s0, s0+L+2)      value for local l is at l+1, wrap at l-nx+1
//   plane 3 (+y) rows y-1 (row 0 of the grid: wrapped row, or the mirror
//                source: own row of plane 4)
//   plane 4 (-y) rows y+1 (last row: wrapped row, or own row of plane 3)
//   plane 5 (+z) plane z-1 (z = 0: wrapped plane, or own rows of plane 6);
//                z-marching: own rows of plane 5
//   plane 6 (-z) plane z+1 (last plane: wrapped, or own rows of plane 5)
//   own rows of planes 5 and 6 [s0, s0+L) (FORM 1 and geometries with membranes)
// The boundary factors (periodic phase, mirror conjugation and rewind) are
// applied per element after the copy, exactly as in the register kernel.
//
// Waits are bounded: a wait that has not completed after ~2 s sets the error
// word of the step control, the CTA waits (again bounded) for the copies it
// still has in flight, and returns.
#include "lbmbt_internal.cuh"
#include "sweep_common.cuh"
#include "tma_common.cuh"

namespace lbmbt {
namespace {

constexpr int TMA_MAX_STAGES = 6;

// Shared-memory stage (all parts 16-byte aligned): 7 pull rows of (cap + 2)
// complex values (the sources listed above), with FORM 1 the own rows of planes
// 5 and 6 (slots 7 and 8), capx spare complex values (0 in use), then cap
// mask bytes.
__host__ __device__ __forceinline__ size_t stage_bytes(int cap, int capx, int form)
{
    return (((size_t)(form == 1 ? 9 : 7) * (cap + 2) + capx) * sizeof(float2) + cap + 127) / 128 * 128;
}
__device__ __forceinline__ float2* stage_plane(unsigned char* stage, int cap, int i)
{
    return reinterpret_cast<float2*>(stage) + (size_t)i * (cap + 2);
}
__device__ __forceinline__ uint8_t* stage_mask(unsigned char* stage, int cap, int capx, int form)
{
    return stage + ((size_t)(form == 1 ? 9 : 7) * (cap + 2) + capx) * sizeof(float2);
}

// Z-marching (FORM 2): the j-th unit of this CTA.  Columns cc = blockIdx +
// q gridDim (q = j / zc) of all members in order; unit index within the
// member cc_local * zc + zi.  n_units past the last column.  zc is a power
// of two (shifts and masks: no division in the unit loops).
__device__ __forceinline__ long long zm_unit(const SweepArgs& a, long long n_units, long long j)
{
    const long long cc = blockIdx.x + (j >> a.zc_log2) * (long long)gridDim.x;
    if (cc >= a.n_cc) return n_units;
    const int m = a.n_members == 1 ? 0 : find_member(a.cc_start, a.n_members, cc);
    const MemberDesc* __restrict__ d = a.members + m;
    return d->unit0 + ((cc - d->cc0) << a.zc_log2) + (j & (a.zc - 1));
}

// Where z-marching unit u lies; us is the index of the same rows in the
// plane-by-plane order, whose signal slots it fills.
__device__ __forceinline__ UnitGeo unit_geo_zm(const SweepArgs& a, long long u, long long* us)
{
    UnitGeo G;
    G.m = a.n_members == 1 ? 0 : find_member(a.tile_start, a.n_members, u);
    const MemberDesc* __restrict__ d = a.members + G.m;
    const int ny = d->ny, nx = d->nx, rpu = d->rpu;
    const int lu = (int)(u - d->unit0);
    const int upz = (ny + rpu - 1) / rpu;
    const int ccl = lu >> a.zc_log2, zi = lu & (a.zc - 1);
    const int yb = ccl % upz;
    G.z = (ccl / upz) * a.zc + zi;
    G.y0 = yb * rpu;
    G.rows = min(rpu, ny - G.y0);
    G.L = G.rows * nx;
    G.s0 = (unsigned)G.z * ((unsigned)nx * ny) + (unsigned)G.y0 * nx;
    *us = d->unit0 + (long long)G.z * upz + yb;
    return G;
}

// Thread 0: copies of unit u into `stage`, completion on `bar`.
template <int FORM>
__device__ void issue_unit(const SweepArgs& a, long long u, int k, int sbase, int smod, unsigned char* stage, int cap,
                           int capx, uint64_t* bar, UnitGeo* info, long long* info_us)
{
    constexpr bool OZ = FORM == 1;
    long long us = u;
    const UnitGeo G = FORM == 2 ? unit_geo_zm(a, u, &us) : unit_geo(a.members, a.tile_start, a.n_members, u);
    *info = G;   // published to the consumers by the mbarrier (release/acquire)
    *info_us = us;
    const int m = G.m, z = G.z, y0 = G.y0, rows = G.rows;
    const MemberDesc& d = a.members[m];
    const long long nx = d.nx, sxy = (long long)d.nx * d.ny;
    const long long L = rows * nx;
    const long long s0 = (long long)z * sxy + (long long)y0 * nx;
    const size_t P = (size_t)d.plane;
    const float2* src = d.state + (size_t)((k - sbase) % smod) * 7 * P;
    auto pl = [&](int i) { return src + (size_t)i * P; };
    const uint32_t rowb = (uint32_t)(nx * sizeof(float2));
    const uint32_t Lb = (uint32_t)(L * sizeof(float2));
    const bool oz = OZ && d.memb;
    const uint32_t total = 5 * Lb + 2 * (Lb + 16) + (uint32_t)L + (oz ? 2 * Lb : 0u);
    mbar_arrive_expect_tx(bar, total);
    if (oz) {   // own rows of planes 5 and 6 (membrane links in z)
        bulk_g2s(stage_plane(stage, cap, 7), pl(5) + s0, Lb, bar);
        bulk_g2s(stage_plane(stage, cap, 8), pl(6) + s0, Lb, bar);
    }
    // rest, +x, -x
    bulk_g2s(stage_plane(stage, cap, 0), pl(0) + s0, Lb, bar);
    bulk_g2s(stage_plane(stage, cap, 1), pl(1) + s0 - 2, Lb + 16, bar);
    bulk_g2s(stage_plane(stage, cap, 2), pl(2) + s0, Lb + 16, bar);
    // +y: rows y0-1 .. y0+rows-2
    {
        float2* dst = stage_plane(stage, cap, 3);
        if (y0 >= 1) {
            bulk_g2s(dst, pl(3) + s0 - nx, Lb, bar);
        } else {
            const float2* face = d.bc[1] == BC_PER ? pl(3) + (long long)z * sxy + (long long)(d.ny - 1) * nx
                                                    : pl(4) + s0;  // mirror: own row 0 of plane 4
            bulk_g2s(dst, face, rowb, bar);
            if (rows > 1) bulk_g2s(dst + nx, pl(3) + s0, Lb - rowb, bar);
        }
    }
    // -y: rows y0+1 .. y0+rows
    {
        float2* dst = stage_plane(stage, cap, 4);
        if (y0 + rows <= d.ny - 1) {
            bulk_g2s(dst, pl(4) + s0 + nx, Lb, bar);
        } else {
            if (rows > 1) bulk_g2s(dst, pl(4) + s0 + nx, Lb - rowb, bar);
            const long long last = s0 + (long long)(rows - 1) * nx;  // row ny-1
            const float2* face = d.bc[1] == BC_PER ? pl(4) + (long long)z * sxy : pl(3) + last;
            bulk_g2s(dst + (rows - 1) * nx, face, rowb, bar);
        }
    }
    // +z, -z (a slab face towards another slab: the halo plane's rows)
    {
        const float2* srcz;
        const int b0 = d.zbc[0], b1 = d.zbc[1];
        if (FORM == 2) srcz = pl(5) + s0;   // z-marching: the own rows (the next unit's pull rows)
        else if (z >= 1) srcz = pl(5) + s0 - sxy;
        else if (b0 == BC_HALO || b0 == BC_HALO_PER) srcz = d.halo[0] + (long long)y0 * nx;
        else srcz = b0 == BC_PER ? pl(5) + s0 + (long long)(d.nz - 1) * sxy : pl(6) + s0;
        bulk_g2s(stage_plane(stage, cap, 5), srcz, Lb, bar);
        if (z <= d.nz - 2) srcz = pl(6) + s0 + sxy;
        else if (b1 == BC_HALO || b1 == BC_HALO_PER) srcz = d.halo[1] + (long long)y0 * nx;
        else srcz = b1 == BC_PER ? pl(6) + (long long)y0 * nx : pl(5) + s0;
        bulk_g2s(stage_plane(stage, cap, 6), srcz, Lb, bar);
    }
    bulk_g2s(stage_mask(stage, cap, capx, FORM), d.mask + s0, (uint32_t)L, bar);
}


// Warp-specialised persistent sweep: warp TMA_CONSUMERS/32 is the producer
// (issues the bulk copies of every unit of this CTA into a ring of nst
// stages), the other warps consume.  Stage st has a "full" mbarrier (one
// arrival with the byte count, completed by the copies) and an "empty"
// mbarrier (one arrival per consumer warp when it is done with the stage).
// No block-wide barrier is used after set-up: every wait is an mbarrier wait
// with a time limit, so a failed wait ends each warp on its own.
template <int TMA_CONSUMERS, int TMA_SPT, int FORM>
__global__ void __launch_bounds__(TMA_CONSUMERS + 32, 1)
    sweep_tma_kernel(const SweepArgs a, long long n_units, int cap, int capx, int nst)
{
    constexpr bool OZ = FORM == 1;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t full[TMA_MAX_STAGES];
    __shared__ uint64_t empty[TMA_MAX_STAGES];
    __shared__ UnitGeo infos[TMA_MAX_STAGES];
    __shared__ long long infos_us[TMA_MAX_STAGES];   // signal slot index of the unit
    __shared__ uint64_t never;   // test of the timeout path: a barrier nothing completes
    __shared__ int s_abort;

    const size_t stb = stage_bytes(cap, capx, FORM);
    const int tid = threadIdx.x;
    const int k = __ldcg(&a.ctl->k);
    const int sbase = __ldcg(&a.ctl->slot_base), smod = __ldcg(&a.ctl->slot_mod);
    auto unit_of = [&](long long j) {
        return FORM == 2 ? zm_unit(a, n_units, j) : blockIdx.x + j * (long long)gridDim.x;
    };
    // z-marching: this CTA's units (its columns x zc); the consumers test
    // only this count, the producer walks the columns
    const long long n_mine = FORM == 2 && blockIdx.x < a.n_cc
                                 ? ((a.n_cc - 1 - blockIdx.x) / gridDim.x + 1) << a.zc_log2 : 0;
    auto has_unit = [&](long long j) { return FORM == 2 ? j < n_mine : unit_of(j) < n_units; };

    if (tid == 0) {
        for (int st = 0; st < nst; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], TMA_CONSUMERS / 32);
        }
        mbar_init(&never, 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    // every thread of this CTA has read the step word: take the CTA's ticket
    // (the last CTA of the launch advances it for the next sweep)
    if (tid == 0) step_done(a.ctl, k, gridDim.x, true);

    if (tid >= TMA_CONSUMERS) {
        // ---------------- producer warp (lane 0 issues)
        if (tid != TMA_CONSUMERS) return;
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
            issue_unit<FORM>(a, u, k, sbase, smod, smem + st * stb, cap, capx, &full[st], &infos[st], &infos_us[st]);
        }
        // wait (bounded) for the copies of the last stages before leaving
        for (long long q = j - 1; q >= 0 && q >= j - nst; --q)
            mbar_wait(&full[q % nst], (uint32_t)((q / nst) & 1));
        if (s_abort) atomicOr(&a.ctl->err, 1);
        return;
    }

    // ---------------- consumer warps
    const bool series = __ldcg(&a.ctl->series);
    const int sig_step = __ldcg(&a.ctl->sig_step), field_step = __ldcg(&a.ctl->field_step);
    const int lsrc = (k - sbase) % smod, ldst = (k + 1 - sbase) % smod;
    const int warp = tid >> 5, lane = tid & 31;

    // Own-site values of planes 3 and 4 on membrane links in y, prefetched
    // into registers one unit ahead for the lanes whose mask needs them.
    float2 own[TMA_SPT][4], nown[TMA_SPT][4];
    // (st, ph): unit j's stage and the parity of its fill
    auto prefetch = [&](long long j, int st, uint32_t ph, float2 (&o)[TMA_SPT][4]) -> bool {
        if (!has_unit(j)) return true;
        if (!mbar_wait(&full[st], ph)) return false;
        const UnitGeo G = infos[st];
        const MemberDesc* __restrict__ d = a.members + G.m;
        if (!d->memb) return true;   // geometry without membranes
        unsigned char* sb = smem + st * stb;
        const uint8_t* __restrict__ mk8 = stage_mask(sb, cap, capx, FORM);
        const unsigned P = (unsigned)d->plane;
        const float2* __restrict__ sp = d->state + (size_t)lsrc * 7 * P;
#pragma unroll
        for (int jj = 0; jj < TMA_SPT; ++jj) {
            const int l = tid + jj * TMA_CONSUMERS;
            if (l < G.L) {
                const unsigned mk = mk8[l];
                const unsigned s = G.s0 + (unsigned)l;
                if (mk & 4u) o[jj][0] = __ldg(sp + (size_t)3 * P + s);
                if (mk & 8u) o[jj][1] = __ldg(sp + (size_t)4 * P + s);
                if (FORM == 0) {
                    if (mk & 16u) o[jj][2] = __ldg(sp + (size_t)5 * P + s);
                    if (mk & 32u) o[jj][3] = __ldg(sp + (size_t)6 * P + s);
                }

            }
        }
        return true;
    };
    // Test of the timeout path (a test-only option): the first wait is on a
    // barrier that nothing completes, with a short limit; it runs out like a
    // lost copy would, and the warp takes the abort path below (the producer
    // keeps its normal bounds and drains its copies before the CTA exits).
    bool ok = a.test_wait_ns == 0 || mbar_wait(&never, 0u, a.test_wait_ns);
    ok = ok && prefetch(0, 0, 0u, own);

    // constants of the current member, reloaded only when the member changes
    int cm = -1, nx = 1, ny = 1, nz = 1, bcx = 0, bcy = 0, bcz0 = 0, bcz1 = 0;
    unsigned P = 0, dm0 = 0;
    int ds0 = 0;
    float sh = 0.f, om0 = 0.f, om1 = 0.f, om2 = 0.f, om3 = 0.f, ep0 = 0.f, ep1 = 0.f, ep2 = 0.f, ep3 = 0.f;
    float2* dstb = nullptr;
    float2* field = nullptr;
    float fk = 0.f;            // the member's f_k
    bool do_sig = false, do_field = false;
    const MemberDesc* __restrict__ sd = a.members;
    // z-marching: per site, this unit's +z pull value and own plane-6 value,
    // carried from the previous unit of the column
    float2 c5[TMA_SPT], c6[TMA_SPT];

    int st = 0, stn = 0;     // stage of unit i and of unit i + 1, and their fill parities
    uint32_t ph = 0, phn = 0;
    for (long long i = 0;; ++i, st = stn, ph = phn) {
        if (!has_unit(i)) break;
        const long long u = FORM == 2 ? 0 : unit_of(i);
        stn = st + 1 == nst ? 0 : st + 1;
        phn = stn == 0 ? ph ^ 1u : ph;
        ok = ok && prefetch(i + 1, stn, phn, nown);
        ok = ok && mbar_wait(&full[st], ph);
        if (!ok) {
            s_abort = 1;
            break;
        }
        const UnitGeo G = infos[st];
        const long long uslot = FORM == 2 ? infos_us[st] : u;   // the unit's signal slots
        unsigned char* sb = smem + st * stb;
        if (G.m != cm) {
            cm = G.m;
            sd = a.members + cm;
            nx = sd->nx; ny = sd->ny; nz = sd->nz;
            bcx = sd->bc[0]; bcy = sd->bc[1]; bcz0 = sd->zbc[0]; bcz1 = sd->zbc[1];
            P = (unsigned)sd->plane;
            dm0 = sd->div_m[0]; ds0 = sd->div_s[0];
            sh = sd->s_share;
            om0 = sd->omega[0]; om1 = sd->omega[1]; om2 = sd->omega[2]; om3 = sd->omega[3];
            ep0 = sd->eps[0]; ep1 = sd->eps[1]; ep2 = sd->eps[2]; ep3 = sd->eps[3];
            dstb = sd->state + (size_t)ldst * 7 * P;
            field = sd->field;
            fk = __ldg(sd->fw + k + a.scheme);   // the classical scheme collides with f_(k+1)
            // a member with an end step of its own gives its signal and field there
            const int es = sd->end_step;
            do_sig = series || k == (es >= 0 ? es : sig_step);
            do_field = field != nullptr && k == (es >= 0 ? es : field_step);
        }
        const float2* __restrict__ r0 = stage_plane(sb, cap, 0);
        const float2* __restrict__ r1 = stage_plane(sb, cap, 1);
        const float2* __restrict__ r2 = stage_plane(sb, cap, 2);
        const float2* __restrict__ r3 = stage_plane(sb, cap, 3);
        const float2* __restrict__ r4 = stage_plane(sb, cap, 4);
        const float2* __restrict__ r5 = stage_plane(sb, cap, 5);
        const float2* __restrict__ r6 = stage_plane(sb, cap, 6);
        const uint8_t* __restrict__ rm = stage_mask(sb, cap, capx, FORM);
        const float2* __restrict__ fac = a.fac + ((size_t)k * a.n_members + G.m) * 6;
        float2* __restrict__ dst = dstb;
        const int z = G.z;
        if (FORM == 2 && (z & (a.zc - 1)) == 0) {
            // first unit of a column: the carried values from memory (the
            // +z pull source as the other forms stage it, the own plane-6 value)
            const float2* __restrict__ sp = sd->state + (size_t)lsrc * 7 * P;
            const unsigned sxy = (unsigned)nx * ny;
#pragma unroll
            for (int j = 0; j < TMA_SPT; ++j) {
                const int l0 = tid + j * TMA_CONSUMERS;
                const int l = l0 < G.L ? l0 : 0;
                const unsigned s = G.s0 + (unsigned)l;
                const float2* p5;
                if (z >= 1) p5 = sp + (size_t)5 * P + (s - sxy);
                else if (bcz0 == BC_HALO || bcz0 == BC_HALO_PER) p5 = sd->halo[0] + (size_t)G.y0 * nx + l;
                else p5 = bcz0 == BC_PER ? sp + (size_t)5 * P + s + (size_t)(nz - 1) * sxy : sp + (size_t)6 * P + s;
                c5[j] = __ldg(p5);
                c6[j] = __ldg(sp + (size_t)6 * P + s);
            }
        }

        // Phase 1, every site of this thread: pulls with the face transforms
        // and the half-link membrane rule.  Lanes past the unit's end work on
        // site 0 of the stage and store nothing.
        float2 g[TMA_SPT][Q];
        unsigned mks[TMA_SPT];
        int xs[TMA_SPT], ys[TMA_SPT];
#pragma unroll
        for (int j = 0; j < TMA_SPT; ++j) {
            const int l0 = tid + j * TMA_CONSUMERS;
            const bool valid = l0 < G.L;
            const int l = valid ? l0 : 0;
            const int r = G.rows == 1 ? 0 : (int)fdiv((unsigned)l, dm0, ds0);
            const int x = l - r * nx;
            const int y = G.y0 + r;
            const unsigned mk = valid ? (unsigned)rm[l] : 0u;
            g[j][0] = r0[l];
            if (x == 0) g[j][1] = bcx == BC_PER ? cmul(r1[l + nx + 1], __ldg(fac + 0)) : face_fix(r2[l], bcx, __ldg(fac + 0));
            else g[j][1] = r1[l + 1];
            if (x == nx - 1) g[j][2] = bcx == BC_PER ? cmul(r2[l - nx + 1], __ldg(fac + 1)) : face_fix(r1[l + 2], bcx, __ldg(fac + 1));
            else g[j][2] = r2[l + 1];
            g[j][3] = r3[l];
            if (y == 0) g[j][3] = face_fix(g[j][3], bcy, __ldg(fac + 2));
            g[j][4] = r4[l];
            if (y == ny - 1) g[j][4] = face_fix(g[j][4], bcy, __ldg(fac + 3));
            g[j][5] = FORM == 2 ? c5[j] : r5[l];
            if (z == 0) g[j][5] = face_fix(g[j][5], bcz0, __ldg(fac + 4));
            g[j][6] = r6[l];
            if (z == nz - 1) g[j][6] = face_fix(g[j][6], bcz1, __ldg(fac + 5));

            // Half-link membrane (Eq. B5): A + s (B - A) with A = own
            // population sent towards the membrane.
            if (mk & 0x3fu) {
                if (mk & 2u) g[j][1] = mix(r2[l], g[j][1], sh);          // link to -x: own hat g_2
                if (mk & 1u) g[j][2] = mix(r1[l + 2], g[j][2], sh);      // link to +x: own hat g_1
                if (mk & 8u) g[j][3] = mix(own[j][1], g[j][3], sh);      // link to -y: own hat g_4
                if (mk & 4u) g[j][4] = mix(own[j][0], g[j][4], sh);      // link to +y: own hat g_3
                if (mk & 32u)   // -z: own hat g_6
                    g[j][5] = mix(FORM == 2 ? c6[j] : OZ ? stage_plane(sb, cap, 8)[l] : own[j][3], g[j][5], sh);
                if (mk & 16u)   // +z: own hat g_5
                    g[j][6] = mix(FORM == 2 ? r5[l] : OZ ? stage_plane(sb, cap, 7)[l] : own[j][2], g[j][6], sh);
            }
            if (FORM == 2) {   // carried to the next unit of the column (same rows, plane z + 1)
                c5[j] = r5[l];
                c6[j] = r6[l];
            }
            mks[j] = mk;
            xs[j] = x;
            ys[j] = y;
        }
        // this warp is done with the stage
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);

        // Phase 2: reaction (Eq. reaction_LBM), BGK collision
        // (Eq. collision_LBM) and the stores, with no branch between sites.
        // rot(j) gives exp(i theta) - 1 of site j; the forms below are chosen
        // once per unit and give the values of rotation_m1 (up to the sign of
        // a zero).
        float zr = 0.f, zi = 0.f;
        auto phase2 = [&](auto rot) {
#pragma unroll
            for (int j = 0; j < TMA_SPT; ++j) {
                const int l = tid + j * TMA_CONSUMERS;
                const bool valid = l < G.L;
                const int ph = mks[j] >> 6;
                const float ep = (ph & 2) ? ((ph & 1) ? ep3 : ep2) : ((ph & 1) ? ep1 : ep0);
                const float om = (ph & 2) ? ((ph & 1) ? om3 : om2) : ((ph & 1) ? om1 : om0);
                const float2 q = reaction_q(rot(j), ep);
                float mr, mi;
                react(g[j], q, mr, mi);
                collide(g[j], om, mr, mi);
                const unsigned s = G.s0 + (unsigned)l;
                if (valid) {
#pragma unroll
                    for (int i2 = 0; i2 < Q; ++i2) __stcs(dst + (size_t)i2 * P + s, g[j][i2]);
                    zr += mr;
                    zi += mi;
                    if (do_field) field[s] = make_float2(mr, mi);
                }
            }
        };
        // Classical scheme (Appendix A, Eq. A12): no reaction step; M = sum_i g_i
        // and the collision with the source dt R M, as in the register sweep
        auto phase2_classical = [&]() {
#pragma unroll
            for (int j = 0; j < TMA_SPT; ++j) {
                const int l = tid + j * TMA_CONSUMERS;
                const bool valid = l < G.L;
                const int ph = mks[j] >> 6;
                const float ep = (ph & 2) ? ((ph & 1) ? ep3 : ep2) : ((ph & 1) ? ep1 : ep0);
                const float om = (ph & 2) ? ((ph & 1) ? om3 : om2) : ((ph & 1) ? om1 : om0);
                float mr = 0.f, mi = 0.f;
#pragma unroll
                for (int i2 = 0; i2 < Q; ++i2) {
                    mr = __fadd_rn(mr, g[j][i2].x);
                    mi = __fadd_rn(mi, g[j][i2].y);
                }
                const float2 src = source_dtRM(ep, fk != 0.f ? theta_lin(sd, fk, xs[j], ys[j], z) : 0.f, mr, mi);
                collide_source_w(g[j], om, mr, mi, src.x, src.y, W0, WI, WI);
                const unsigned s = G.s0 + (unsigned)l;
                if (valid) {
#pragma unroll
                    for (int i2 = 0; i2 < Q; ++i2) __stcs(dst + (size_t)i2 * P + s, g[j][i2]);
                    zr += mr;
                    zi += mi;
                    if (do_field) field[s] = make_float2(mr, mi);
                }
            }
        };
        const int ax = sd->axes;
        const float2* __restrict__ et = sd->etab;
        if (a.scheme == 1) {
            phase2_classical();
        } else if (fk == 0.f) {
            phase2([&](int) { return make_float2(0.f, 0.f); });
        } else if (et != nullptr && (fk == 1.f || fk == -1.f) && (ax == 1 || ax == 2 || ax == 4)) {
            // one gradient axis: a single table entry per site
            const float2* __restrict__ base = et + (ax == 1 ? 0 : ax == 2 ? nx : nx + ny + z);
            const int cx = ax == 1, cy = ax == 2;
            const bool neg = fk < 0.f;
            phase2([&](int j) {
                float2 v = __ldg(base + xs[j] * cx + ys[j] * cy);
                if (neg) v.y = -v.y;
                return v;
            });
        } else if (et != nullptr && (fk == 1.f || fk == -1.f)) {
            // general direction: x and y entries per site, the z entry once
            // per unit (a disabled axis has an all-zero table)
            const float2 ez = __ldg(et + nx + ny + z);
            const bool neg = fk < 0.f;
            phase2([&](int j) {
                float2 v = cadd_prod(cadd_prod(__ldg(et + xs[j]), __ldg(et + nx + ys[j])), ez);
                if (neg) v.y = -v.y;
                return v;
            });
        } else {
            phase2([&](int j) { return rotation_m1(sd, fk, xs[j], ys[j], z); });
        }
#pragma unroll
        for (int j = 0; j < TMA_SPT; ++j)
#pragma unroll
            for (int p = 0; p < 4; ++p) own[j][p] = nown[j][p];
        if (do_sig) {   // unit-uniform; FP64 from the warp level up, one slot per warp
            double dr = zr, di = zi;
            for (int o = 16; o > 0; o >>= 1) {
                dr += __shfl_down_sync(0xffffffffu, dr, o);
                di += __shfl_down_sync(0xffffffffu, di, o);
            }
            if (lane == 0) a.partial[uslot * (TMA_CONSUMERS / 32) + warp] = make_double2(dr, di);
        }
    }
    if (s_abort && tid == 0) atomicOr(&a.ctl->err, 1);
}

}  // namespace

size_t tma_smem_bytes(int cap, int capx, int nst, int form) { return stage_bytes(cap, capx, form) * nst; }
// signal partial slots per unit: one per consumer warp of the variant
int tma_partials_per_unit(int variant) { return variant == 1 ? 12 : variant == 2 ? 8 : variant == 3 ? 11 : 16; }

// variant 0: 16 consumer warps x 2 sites, 1: 12 x 3, 2: 8 x 4, 3 (default):
// 11 x 3 (units <= 1024 sites).  The register file is split over the SM's 4
// sub-partitions: with the producer warp, 9 to 12 warps per CTA allow 168
// registers a thread, 13 to 16 warps 128 and 17 warps 96; the two-phase
// consumer needs about 150.  Each in two forms: with the own z rows staged
// (form 1), prefetched into registers (form 0), or z-marching (form 2).
template <int FORM>
static void* tma_kernel_form(int variant)
{
    switch (variant) {
    case 1: return (void*)sweep_tma_kernel<384, 3, FORM>;
    case 2: return (void*)sweep_tma_kernel<256, 4, FORM>;
    case 3: return (void*)sweep_tma_kernel<352, 3, FORM>;
    default: return (void*)sweep_tma_kernel<512, 2, FORM>;
    }
}
static void* tma_kernel(int variant, int form)
{
    return form == 2 ? tma_kernel_form<2>(variant) : form == 1 ? tma_kernel_form<1>(variant) : tma_kernel_form<0>(variant);
}
static int tma_threads(int variant)
{
    return variant == 1 ? 384 + 32 : variant == 2 ? 256 + 32 : variant == 3 ? 352 + 32 : 512 + 32;
}

cudaError_t tma_prepare(int cap, int capx, int nst, int variant, int form, int* ctas_per_sm)
{
    const size_t bytes = tma_smem_bytes(cap, capx, nst, form);
    void* fn = tma_kernel(variant, form);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fn, tma_threads(variant), bytes);
}

template <int FORM>
static void launch_form(const SweepArgs& a, long long n_units, int cap, int capx, int nst, int variant, int grid,
                        size_t sm, cudaStream_t st)
{
    switch (variant) {
    case 1: sweep_tma_kernel<384, 3, FORM><<<grid, 384 + 32, sm, st>>>(a, n_units, cap, capx, nst); break;
    case 2: sweep_tma_kernel<256, 4, FORM><<<grid, 256 + 32, sm, st>>>(a, n_units, cap, capx, nst); break;
    case 3: sweep_tma_kernel<352, 3, FORM><<<grid, 352 + 32, sm, st>>>(a, n_units, cap, capx, nst); break;
    default: sweep_tma_kernel<512, 2, FORM><<<grid, 512 + 32, sm, st>>>(a, n_units, cap, capx, nst); break;
    }
}

cudaError_t launch_sweep_tma(const SweepArgs& a, long long n_units, int cap, int capx, int nst, int variant, int form,
                             int grid, cudaStream_t st)
{
    if (nst < 2 || nst > TMA_MAX_STAGES) return cudaErrorInvalidValue;
    if (form == 2 && (a.zc < 1 || a.cc_start == nullptr)) return cudaErrorInvalidValue;
    const size_t sm = tma_smem_bytes(cap, capx, nst, form);
    if (form == 2)
        launch_form<2>(a, n_units, cap, capx, nst, variant, grid, sm, st);
    else if (form == 1)
        launch_form<1>(a, n_units, cap, capx, nst, variant, grid, sm, st);
    else
        launch_form<0>(a, n_units, cap, capx, nst, variant, grid, sm, st);
    return cudaGetLastError();
}

}  // namespace lbmbt
