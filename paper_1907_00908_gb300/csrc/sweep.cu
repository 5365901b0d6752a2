// sweep.cu -- forward kernels of the hybrid lattice-Boltzmann Bloch-Torrey
// scheme (arXiv 1907.00908) for sm_103a.
//
//  * build_mask_kernel : labels -> per-site membrane bits + phase (Sec. 2.4.2)
//  * init_kernel       : hat g_i = omega_i (M = 1 at equilibrium, Sec. 2.1)
//  * sweep_kernel      : one fused time step per site, pull form:
//        stream + outer BC + half-link membrane   (Eqs. streaming_LBM,
//                                                  collision_BC, B5, Sec. 2.4.4)
//        reaction (phase + T2 decay)             (Eq. reaction_LBM)
//        M = sum_i g_i, BGK collision            (Eqs. M'summation, collision_LBM)
//        optional FP64 signal partials / field   (Sec. 2.1 signal)
//    The loop state is the post-collision population hat g(t^k); one pass
//    maps hat g(t^k) -> hat g(t^{k+1}), i.e. the paper's step order re-cut at
//    the collision, so every site reads 7 complex values (one from each
//    upstream neighbour) and writes 7 (5 on the D2Q5 lattice, whose z
//    populations stay exactly 0 and are not touched).
//  * sweep_links_kernel: the same step with membranes at given positions on
//        the links (Eqs. B4a-B4c), the rule's links compacted per warp
//  * sweep_classical_kernel: the same pass for the classical LBM (Appendix A,
//        Eq. A12): stream + BCs + membrane, M = sum_i g_i, collision with
//        the reaction as a source term; no reaction step
//  * ctl_set_kernel    : sets the step word before a run of sweeps (the
//                        bulk-copy sweep's last CTA advances it; after a
//                        register sweep ctl_advance_kernel does)
//  * factor_table_kernel: FP64 boundary factors of every step, once per run
//  * reduce_kernel     : fixed-order FP64 sum of the per-tile partials.
//
// The work list of a launch is the concatenation of all members' tiles; a
// block finds its member by binary search over the tile prefix.
#include "lbmbt_internal.cuh"
#include "sweep_common.cuh"
#include "links.cuh"

namespace lbmbt {
namespace {

// ---------------------------------------------------------------- mask
__global__ void build_mask_kernel(const int32_t* __restrict__ labels, const uint8_t* __restrict__ pol,
                                  int n_labels, int nx, int ny, int nz, int bcx, int bcy, int bcz,
                                  uint8_t* __restrict__ mask, int* err)
{
    const unsigned N = (unsigned)nx * ny * nz;
    const int dims[3] = {nx, ny, nz};
    const int bc[3] = {bcx, bcy, bcz};
    const unsigned stride[3] = {1u, (unsigned)nx, (unsigned)nx * ny};
    for (unsigned s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const unsigned row = s / nx;
        const int c[3] = {(int)(s - row * nx), (int)(row % ny), (int)(row / ny)};
        const int L = labels[s];
        if (L < 0 || L >= n_labels) {
            atomicOr(err, 1);
            mask[s] = 0;
            continue;
        }
        unsigned m = (unsigned)pol[L] << 6;
#pragma unroll
        for (int b = 0; b < 6; ++b) {       // bit b: direction i = b+1
            const int ax = b >> 1;
            const int sg = (b & 1) ? -1 : 1;
            int cn = c[ax] + sg;
            long long nb;
            if (cn < 0 || cn >= dims[ax]) {
                if (bc[ax] != BC_PER) continue;  // mirror face: no neighbour
                nb = (long long)s + (long long)(sg > 0 ? -(dims[ax] - 1) : (dims[ax] - 1)) * stride[ax];
            } else {
                nb = (long long)s + (long long)sg * stride[ax];
            }
            if (labels[nb] != L) m |= 1u << b;
        }
        mask[s] = (uint8_t)m;
        if (m & 0x3fu) atomicOr(err, 2);   // bit 1: the geometry has membranes
    }
}

// ---------------------------------------------------------------- init
// Hybrid scheme: hat g(t^0) = g_eq = omega_i (M = 1).  Classical scheme: the
// loop state hat g(t^0) is the collision of g_eq with the source of step 0,
// omega_i (1 + dt R(x, t^0)), R = -i gamma x.G0 f_0 - 1/T2 (Eq. A12).
__global__ void init_kernel(const MemberDesc* __restrict__ members, const long long* __restrict__ tile_start,
                            int n_members, int spt, int slot, float w0, float wxy, float wz, int classical)
{
    __shared__ int sm;
    if (threadIdx.x == 0) sm = find_member(tile_start, n_members, blockIdx.x);
    __syncthreads();
    const MemberDesc& d = members[sm];
    const unsigned P = (unsigned)d.plane;
    float2* out = d.state + (size_t)slot * 7 * P;
    const unsigned base = (unsigned)(blockIdx.x - d.tile0) * blockDim.x * spt;
    for (int j = 0; j < spt; ++j) {
        const unsigned s = base + j * blockDim.x + threadIdx.x;
        if (s < (unsigned)d.N) {
            float2 src = make_float2(0.f, 0.f);   // dt R M with M = 1
            if (classical) {
                int x, y, z;
                coords(&d, s, d.nx, d.ny, x, y, z);
                const float f0 = __ldg(d.fw);
                src = source_dtRM(d.eps[d.mask[s] >> 6], f0 != 0.f ? theta_lin(&d, f0, x, y, z) : 0.f, 1.f, 0.f);
            }
            out[s] = make_float2(__fmaf_rn(w0, src.x, w0), __fmul_rn(w0, src.y));
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const float w = i < 5 ? wxy : wz;
                out[(size_t)i * P + s] = make_float2(__fmaf_rn(w, src.x, w), __fmul_rn(w, src.y));
            }
            // slab halo planes start at the neighbours' initial values
            if (s < (unsigned)(d.nx * d.ny))
                for (int h = 0; h < 2; ++h)
                    if (d.halo[h]) const_cast<float2*>(d.halo[h])[s] = make_float2(wz, 0.f);
        }
    }
}

// Warp-compacted membrane links (Eqs. B4a-B4c): the links of one warp's 32
// sites that take the position rule are listed in shared memory and shared
// out one per lane, so the rule's loads and coefficients run once per link
// instead of once per direction for the whole warp.  One list covers all SPT
// sites of the warp's threads.  Per warp: SPT * LINK_SLOTS results (float2)
// and as many items (site << 8 | lane << 3 | direction, 16 bits).  A site
// lists at most 3 links, one per axis: direction i needs a membrane on the
// link behind it and none on the link ahead, so i and its opposite exclude
// each other.
constexpr int LINK_SLOTS = 32 * 3;
inline size_t link_smem_bytes(int block, int spt)
{
    return (size_t)(block / 32) * spt * LINK_SLOTS * (sizeof(float2) + sizeof(uint16_t));
}

// LINKS: 0 half-link rule only, 1 membrane positions, 2 positions and angles.
// CLS: the classical scheme (Eq. A12) instead of the hybrid one.
template <int SPT, int LINKS, bool CLS = false>
__device__ __forceinline__ void sweep_body(const SweepArgs& a)
{
    __shared__ double2 s_red[32];
    extern __shared__ __align__(16) unsigned char s_link[];   // LINKS only: link_smem_bytes(blockDim.x, SPT)
    // Every thread looks up its member, step and flags itself (broadcast
    // loads): there is no per-block prologue to wait for.
    const int m = a.n_members == 1 ? 0 : find_member(a.tile_start, a.n_members, blockIdx.x);
    const MemberDesc* __restrict__ sd = a.members + m;
    const int k = __ldcg(&a.ctl->k);
    const int sbase = __ldcg(&a.ctl->slot_base), smod = __ldcg(&a.ctl->slot_mod);
    // a member with an end step of its own (shorter waveform in a batch)
    // gives its signal and field there
    const int es = sd->end_step;
    const bool do_sig = __ldcg(&a.ctl->series) || k == (es >= 0 ? es : __ldcg(&a.ctl->sig_step));
    float2* const field = sd->field;
    const bool do_field = k == (es >= 0 ? es : __ldcg(&a.ctl->field_step)) && field != nullptr;
    const float2* __restrict__ fac = a.fac + ((size_t)k * a.n_members + m) * 6;

    // classical: the collision of this pass carries the source of step k+1
    const float fk = __ldg(sd->fw + k + (CLS ? 1 : 0));
    const unsigned P = (unsigned)sd->plane;
    const float2* __restrict__ src = sd->state + (size_t)((k - sbase) % smod) * 7 * P;
    float2* __restrict__ dst = sd->state + (size_t)((k + 1 - sbase) % smod) * 7 * P;
    const uint8_t* __restrict__ mask = sd->mask;
    const int nx = sd->nx, ny = sd->ny, nz = sd->nz;
    const int bcx = sd->bc[0], bcy = sd->bc[1], bcz0 = sd->zbc[0], bcz1 = sd->zbc[1];
    const unsigned sxy = (unsigned)nx * ny;
    const unsigned N = (unsigned)sd->N;
    const unsigned base = (unsigned)(blockIdx.x - sd->tile0) * blockDim.x * SPT;
    const float sh = sd->s_share;
    float zr = 0.f, zi = 0.f;   // per-thread sums in FP32, FP64 from the warp level up
    // D2Q5 (the z populations carry weight 0): they are exactly 0 at the
    // start and stay 0, so the z planes are neither read nor written
    const bool zpl = a.wz != 0.f;

    // Membranes at given positions: the warp lists the links of all its
    // sites that take the position rule (those whose node behind s, s + e_i,
    // lies in s's compartment), shares the list out one link per lane and
    // leaves the results in shared memory, all before any pull: the pulled
    // values are then not live across the rule's loads and arithmetic.
    const bool links_on = LINKS && sd->dlt != nullptr;   // block-uniform
    const unsigned lane = threadIdx.x & 31u;
    unsigned cand[SPT], off[SPT];   // per site: listed directions (bits 1..6), first list slot
    float2* res = nullptr;
    if (links_on) {
        res = reinterpret_cast<float2*>(s_link) + (threadIdx.x >> 5) * (SPT * LINK_SLOTS);
        uint16_t* const item = reinterpret_cast<uint16_t*>(reinterpret_cast<float2*>(s_link) +
                                                           (blockDim.x >> 5) * (SPT * LINK_SLOTS)) +
                               (threadIdx.x >> 5) * (SPT * LINK_SLOTS);
        unsigned K = 0;
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
            const unsigned s_at = base + j * blockDim.x + threadIdx.x;
            unsigned c = 0;
            if (s_at < N) {
                const unsigned mk = mask[s_at];
                if (mk & 0x3fu) {
#pragma unroll
                    for (int i = 1; i < Q; ++i) {
                        const int ib = (i & 1) ? i + 1 : i - 1;
                        if ((mk & (1u << (ib - 1))) && !(mk & (1u << (i - 1)))) c |= 1u << i;
                    }
                }
            }
            unsigned incl = __popc(c);   // inclusive prefix of the warp's link counts
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (unsigned)o) incl += v;
            }
            cand[j] = c;
            off[j] = K + incl - __popc(c);
            unsigned o = off[j];
            for (unsigned cc = c; cc; cc &= cc - 1)
                item[o++] = (uint16_t)(((unsigned)j << 8) | (lane << 3) | (__ffs(cc) - 1));
            K += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (K != 0) {   // warp-uniform
            __syncwarp();
            const unsigned wbase = base + (threadIdx.x - lane);
            for (unsigned t0 = 0; t0 < K; t0 += 32) {   // warp-uniform
                const unsigned t = t0 + lane;
                if (t < K) {
                    const unsigned it = item[t];
                    const unsigned so = wbase + (it >> 8) * blockDim.x + ((it >> 3) & 31u);
                    int xo, yo, zo;
                    coords(sd, so, nx, ny, xo, yo, zo);
                    res[t] = link_population<LINKS == 2>(sd, src, fac, so, xo, yo, zo, (int)(it & 7));
                }
            }
            __syncwarp();
        }
    }

#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const unsigned s = base + j * blockDim.x + threadIdx.x;
        if (s >= N) break;
        int x, y, z;
        coords(sd, s, nx, ny, x, y, z);
        const unsigned mk = mask[s];
        const int ph = mk >> 6;

        float2 g[Q];
        g[0] = __ldg(src + s);
        g[1] = pull<0, +1>(src, P, s, x, nx, 1u, bcx, fac);
        g[2] = pull<0, -1>(src, P, s, x, nx, 1u, bcx, fac);
        g[3] = pull<1, +1>(src, P, s, y, ny, (unsigned)nx, bcy, fac);
        g[4] = pull<1, -1>(src, P, s, y, ny, (unsigned)nx, bcy, fac);
        if (zpl) {
            g[5] = pull<2, +1>(src, P, s, z, nz, sxy, bcz0, fac, &sd->halo[0]);
            g[6] = pull<2, -1>(src, P, s, z, nz, sxy, bcz1, fac, &sd->halo[1]);
        } else {
            g[5] = g[6] = make_float2(0.f, 0.f);
        }

        // Half-link membrane (Eq. B5): on a membrane link the arriving
        // population is r * (own population sent towards the membrane) +
        // s * (population streaming across), written A + s (B - A).
        // Bit (ibar - 1) marks the link to the upstream neighbour of i.
        // With positions, the listed links take the result left in shared
        // memory instead.
        if (links_on) {
            if (mk & 0x3fu) {   // node behind s in another compartment: half-link rule
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const int ib = (i & 1) ? i + 1 : i - 1;
                    if ((mk & (1u << (ib - 1))) && (mk & (1u << (i - 1))))
                        g[i] = mix(__ldg(src + (size_t)ib * P + s), g[i], sh);
                }
            }
            unsigned o = off[j];
#pragma unroll
            for (int i = 1; i < Q; ++i)
                if (cand[j] & (1u << i)) g[i] = res[o++];
        } else if (mk & 0x3fu) {
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int ib = (i & 1) ? i + 1 : i - 1;
                if (mk & (1u << (ib - 1))) g[i] = mix(__ldg(src + (size_t)ib * P + s), g[i], sh);
            }
        }

        // Reaction (Eq. reaction_LBM): g <- g exp(-i gamma x.G0 f_k dt) (1 - eps),
        // applied as g + g q with q = exp(i theta)(1 - eps) - 1 (minus-one
        // forms, no O(1) rounding); then M and the BGK collision
        // (Eqs. M'summation, collision_LBM).
        float mr, mi;
        if (CLS) {
            // Classical scheme (Eq. A12): no reaction step; M(t^(k+1)) =
            // sum_i g_i, then the collision with the source dt R M of t^(k+1)
            mr = 0.f;
            mi = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                mr = __fadd_rn(mr, g[i].x);
                mi = __fadd_rn(mi, g[i].y);
            }
            const float2 src = source_dtRM(sd->eps[ph], fk != 0.f ? theta_lin(sd, fk, x, y, z) : 0.f, mr, mi);
            collide_source_w(g, sd->omega[ph], mr, mi, src.x, src.y, a.w0, a.wxy, a.wz);
        } else {
            const float2 q = fk != 0.f ? reaction_q(rotation_m1(sd, fk, x, y, z), sd->eps[ph])
                                       : make_float2(-sd->eps[ph], 0.f);
            react(g, q, mr, mi);
            collide_w(g, sd->omega[ph], mr, mi, a.w0, a.wxy, a.wz);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (i < 5 || zpl) __stcs(dst + (size_t)i * P + s, g[i]);

        zr += mr;
        zi += mi;
        if (do_field) field[s] = make_float2(mr, mi);
    }

    if (do_sig) {   // block-uniform: the only barrier of the kernel
        double dr = zr, di = zi;
        for (int o = 16; o > 0; o >>= 1) {
            dr += __shfl_down_sync(0xffffffffu, dr, o);
            di += __shfl_down_sync(0xffffffffu, di, o);
        }
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) s_red[w] = make_double2(dr, di);
        __syncthreads();
        if (w == 0) {
            const int nw = blockDim.x >> 5;
            double2 v = l < nw ? s_red[l] : make_double2(0.0, 0.0);
            for (int o = 16; o > 0; o >>= 1) {
                v.x += __shfl_down_sync(0xffffffffu, v.x, o);
                v.y += __shfl_down_sync(0xffffffffu, v.y, o);
            }
            if (l == 0) a.partial[blockIdx.x] = v;
        }
    }
}

template <int SPT>
__global__ void __launch_bounds__(512) sweep_kernel(const SweepArgs a)
{
    sweep_body<SPT, 0>(a);
}

template <int SPT>
__global__ void __launch_bounds__(512) sweep_classical_kernel(const SweepArgs a)
{
    sweep_body<SPT, 0, true>(a);
}

// With membrane positions: two blocks of 512 per SM (64 registers), since
// the position rule's extra loads need more warps in flight to hide them.
// ANG: with membrane angles too (one-plane D2Q5 grids); the general-angle
// rule's 18 extrapolation reads would spill at 64 registers, so one block.
template <int SPT, bool ANG>
__global__ void __launch_bounds__(512, ANG ? 1 : 2) sweep_links_kernel(const SweepArgs a)
{
    sweep_body<SPT, ANG ? 2 : 1>(a);
}

// Control word: set before a run of sweeps.
__global__ void ctl_set_kernel(StepCtl* ctl, StepCtl v) { *ctl = v; }

// Step advance after a register sweep.  That sweep has one block per tile
// (~10^5 a step on large grids); a ticket per block at its end, as the
// persistent bulk-copy sweep takes one per CTA, made each block wait for its
// streaming stores before it retired: 25 % slower, measured.  A persistent
// form of the register sweep was 12 % slower than one block per tile.
__global__ void ctl_advance_kernel(StepCtl* ctl) { ctl->k = ctl->k + 1; }

// Boundary factors of all steps 0..K, in FP64 from each member's F_k:
// table[k][m][6] (forward sweeps and adjoint sweeps).
__global__ void factor_table_kernel(const MemberDesc* __restrict__ members, int n_members, int F_shift, long long K,
                                    float2* __restrict__ table)
{
    const long long n = (K + 1) * n_members;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const long long k = t / n_members;
        const int m = (int)(t - k * n_members);
        boundary_factors6(members[m], members[m].Fw[k + F_shift], table + t * 6);
    }
}

// ---------------------------------------------------------------- reduce
__global__ void reduce_kernel(const double2* __restrict__ partial, const long long* __restrict__ tile_start,
                              int per, double2* __restrict__ out, double2* __restrict__ series,
                              long long series_stride, const StepCtl* ctl)
{
    __shared__ double2 sh[256];
    const int m = blockIdx.x;
    const long long t0 = tile_start[m] * per, t1 = tile_start[m + 1] * per;
    double2 v = make_double2(0.0, 0.0);
    for (long long t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        v.x += partial[t].x;
        v.y += partial[t].y;
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[threadIdx.x].x += sh[threadIdx.x + o].x;
            sh[threadIdx.x].y += sh[threadIdx.x + o].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[m] = sh[0];
        if (series) series[m * series_stride + (__ldcg(&ctl->k) - 1)] = sh[0];
    }
}

}  // namespace

cudaError_t launch_ctl_set(StepCtl* ctl, const StepCtl& v, cudaStream_t st)
{
    ctl_set_kernel<<<1, 1, 0, st>>>(ctl, v);
    return cudaGetLastError();
}

cudaError_t launch_factor_table(const MemberDesc* members, int n_members, int F_shift, long long K,
                                float2* table, cudaStream_t st)
{
    const long long n = (K + 1) * n_members;
    long long grid = (n + 255) / 256;
    if (grid > 152LL * 32) grid = 152LL * 32;
    factor_table_kernel<<<(unsigned)grid, 256, 0, st>>>(members, n_members, F_shift, K, table);
    return cudaGetLastError();
}

cudaError_t launch_build_mask(const int32_t* labels, const uint8_t* phase_of_label, int n_labels, int nx,
                              int ny, int nz, const int bc[3], uint8_t* mask, int* err, cudaStream_t st)
{
    const long long N = (long long)nx * ny * nz;
    const int block = 256;
    long long grid = (N + block - 1) / block;
    if (grid > 152LL * 64) grid = 152LL * 64;
    build_mask_kernel<<<(unsigned)grid, block, 0, st>>>(labels, phase_of_label, n_labels, nx, ny, nz, bc[0],
                                                        bc[1], bc[2], mask, err);
    return cudaGetLastError();
}

cudaError_t launch_init(const SweepArgs& a, long long n_tiles, int block, int spt, int slot, cudaStream_t st)
{
    init_kernel<<<(unsigned)n_tiles, block, 0, st>>>(a.members, a.tile_start, a.n_members, spt, slot, a.w0, a.wxy,
                                                     a.wz, a.scheme);
    return cudaGetLastError();
}

// The membrane-position kernels take up to link_smem_bytes(512, 4) of
// dynamic shared memory (above the default 48 KB); set once per run set-up.
cudaError_t links_prepare()
{
    const int bytes = (int)link_smem_bytes(512, 4);
    const void* k[6] = {(const void*)sweep_links_kernel<1, false>, (const void*)sweep_links_kernel<2, false>,
                        (const void*)sweep_links_kernel<4, false>, (const void*)sweep_links_kernel<1, true>,
                        (const void*)sweep_links_kernel<2, true>, (const void*)sweep_links_kernel<4, true>};
    for (const void* f : k) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t launch_sweep_blocks(const SweepArgs& a, long long n_tiles, int block, int spt, cudaStream_t st);

cudaError_t launch_sweep(const SweepArgs& a, long long n_tiles, int block, int spt, cudaStream_t st)
{
    cudaError_t e = launch_sweep_blocks(a, n_tiles, block, spt, st);
    if (e != cudaSuccess) return e;
    ctl_advance_kernel<<<1, 1, 0, st>>>(a.ctl);
    return cudaGetLastError();
}

static cudaError_t launch_sweep_blocks(const SweepArgs& a, long long n_tiles, int block, int spt, cudaStream_t st)
{
    if (a.scheme == 1) {   // classical scheme: half-link rule only (positions are refused at set-up)
        switch (spt) {
        case 1: sweep_classical_kernel<1><<<(unsigned)n_tiles, block, 0, st>>>(a); break;
        case 2: sweep_classical_kernel<2><<<(unsigned)n_tiles, block, 0, st>>>(a); break;
        case 4: sweep_classical_kernel<4><<<(unsigned)n_tiles, block, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (spt) {
    case 1:
        if (a.links == 2) sweep_links_kernel<1, true><<<(unsigned)n_tiles, block, link_smem_bytes(block, 1), st>>>(a);
        else if (a.links) sweep_links_kernel<1, false><<<(unsigned)n_tiles, block, link_smem_bytes(block, 1), st>>>(a);
        else sweep_kernel<1><<<(unsigned)n_tiles, block, 0, st>>>(a);
        break;
    case 2:
        if (a.links == 2) sweep_links_kernel<2, true><<<(unsigned)n_tiles, block, link_smem_bytes(block, 2), st>>>(a);
        else if (a.links) sweep_links_kernel<2, false><<<(unsigned)n_tiles, block, link_smem_bytes(block, 2), st>>>(a);
        else sweep_kernel<2><<<(unsigned)n_tiles, block, 0, st>>>(a);
        break;
    case 4:
        if (a.links == 2) sweep_links_kernel<4, true><<<(unsigned)n_tiles, block, link_smem_bytes(block, 4), st>>>(a);
        else if (a.links) sweep_links_kernel<4, false><<<(unsigned)n_tiles, block, link_smem_bytes(block, 4), st>>>(a);
        else sweep_kernel<4><<<(unsigned)n_tiles, block, 0, st>>>(a);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double2* partial, const long long* tile_start, int per, int n_members, double2* out,
                          double2* series, long long series_stride, const StepCtl* ctl, cudaStream_t st)
{
    reduce_kernel<<<n_members, 256, 0, st>>>(partial, tile_start, per, out, series, series_stride, ctl);
    return cudaGetLastError();
}

}  // namespace lbmbt
