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
//    upstream neighbour) and writes 7.
//  * reduce_kernel     : fixed-order FP64 sum of the per-tile partials.
//
// The work list of a launch is the concatenation of all members' tiles; a
// block finds its member by binary search over the tile prefix.
#include "lbmbt_internal.cuh"
#include "sweep_common.cuh"

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
    }
}

// ---------------------------------------------------------------- init
__global__ void init_kernel(const MemberDesc* __restrict__ members, const long long* __restrict__ tile_start,
                            int n_members, int spt, int slot)
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
            out[s] = make_float2(W0, 0.f);
#pragma unroll
            for (int i = 1; i < Q; ++i) out[(size_t)i * P + s] = make_float2(WI, 0.f);
        }
    }
}

template <int SPT>
__global__ void __launch_bounds__(512) sweep_kernel(const SweepArgs a)
{
    __shared__ MemberDesc sd;
    __shared__ float2 sfac[3][2];
    __shared__ int s_k, s_flags, s_src, s_dst;
    __shared__ double2 s_red[32];

    if (threadIdx.x == 0) {
        const int m = find_member(a.tile_start, a.n_members, blockIdx.x);
        sd = a.members[m];
        const int k = __ldcg(&a.ctl->k);
        const int base = __ldcg(&a.ctl->slot_base), mod = __ldcg(&a.ctl->slot_mod);
        s_k = k;
        s_src = (k - base) % mod;
        s_dst = (k + 1 - base) % mod;
        int flags = 0;
        if (__ldcg(&a.ctl->series) || k == __ldcg(&a.ctl->sig_step)) flags |= 1;
        if (k == __ldcg(&a.ctl->field_step) && sd.field != nullptr) flags |= 2;
        s_flags = flags;
        boundary_factors(sd, a.F[k], sfac);
    }
    __syncthreads();

    const int k = s_k;
    const int flags = s_flags;
    const float fk = __ldg(a.f + k);
    const unsigned P = (unsigned)sd.plane;
    const float2* __restrict__ src = sd.state + (size_t)s_src * 7 * P;
    float2* __restrict__ dst = sd.state + (size_t)s_dst * 7 * P;
    const int nx = sd.nx, ny = sd.ny, nz = sd.nz;
    const unsigned sxy = (unsigned)nx * ny;
    const unsigned N = (unsigned)sd.N;
    const unsigned base = (unsigned)(blockIdx.x - sd.tile0) * blockDim.x * SPT;
    const float sh = sd.s_share;
    double zr = 0.0, zi = 0.0;

#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const unsigned s = base + j * blockDim.x + threadIdx.x;
        if (s >= N) break;
        const unsigned row = s / nx;
        const int x = (int)(s - row * nx);
        const int z = (int)(row / ny);
        const int y = (int)(row - (unsigned)z * ny);
        const unsigned mk = sd.mask[s];
        const int ph = mk >> 6;

        float2 g[Q];
        g[0] = __ldg(src + s);
        g[1] = pull<0, +1>(src, P, s, x, nx, 1u, sd.bc[0], sfac[0][0]);
        g[2] = pull<0, -1>(src, P, s, x, nx, 1u, sd.bc[0], sfac[0][1]);
        g[3] = pull<1, +1>(src, P, s, y, ny, (unsigned)nx, sd.bc[1], sfac[1][0]);
        g[4] = pull<1, -1>(src, P, s, y, ny, (unsigned)nx, sd.bc[1], sfac[1][1]);
        g[5] = pull<2, +1>(src, P, s, z, nz, sxy, sd.bc[2], sfac[2][0]);
        g[6] = pull<2, -1>(src, P, s, z, nz, sxy, sd.bc[2], sfac[2][1]);

        // Half-link membrane (Eq. B5): on a membrane link the arriving
        // population is r * (own population sent towards the membrane) +
        // s * (population streaming across), written A + s (B - A).
        // Bit (ibar - 1) marks the link to the upstream neighbour of i.
        if (mk & 0x3fu) {
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int ib = (i & 1) ? i + 1 : i - 1;
                if (mk & (1u << (ib - 1))) {
                    const float2 o = __ldg(src + (size_t)ib * P + s);
                    g[i].x = o.x + sh * (g[i].x - o.x);
                    g[i].y = o.y + sh * (g[i].y - o.y);
                }
            }
        }

        // Reaction (Eq. reaction_LBM): g <- g exp(-i gamma x.G0 f_k dt) (1 - eps),
        // applied as g + g q with q = exp(i theta)(1 - eps) - 1 and
        // cos(theta) - 1 = -2 sin^2(theta/2), so no O(1) rounding enters.
        const float ep = sd.eps[ph];
        float qr = -ep, qi = 0.f;
        if (fk != 0.f) {
            const float th = fk * (sd.ctheta[0] * (float)x + sd.ctheta[1] * (float)y + sd.ctheta[2] * (float)z);
            float sh2, ch2;
            sincosf(0.5f * th, &sh2, &ch2);
            const float cm1 = -2.f * sh2 * sh2;
            qr = cm1 - ep * (1.f + cm1);
            qi = 2.f * sh2 * ch2 * (1.f - ep);
        }
        float mr = 0.f, mi = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float gr = g[i].x, gi = g[i].y;
            g[i].x = gr + (gr * qr - gi * qi);
            g[i].y = gi + (gr * qi + gi * qr);
            mr += g[i].x;
            mi += g[i].y;
        }

        // BGK collision (Eq. collision_LBM) with g_eq = w_i M (Eq. g_eq).
        const float om = sd.omega[ph];
        __stcs(dst + s, make_float2(g[0].x + om * (W0 * mr - g[0].x), g[0].y + om * (W0 * mi - g[0].y)));
#pragma unroll
        for (int i = 1; i < Q; ++i)
            __stcs(dst + (size_t)i * P + s,
                   make_float2(g[i].x + om * (WI * mr - g[i].x), g[i].y + om * (WI * mi - g[i].y)));

        if (flags & 1) { zr += mr; zi += mi; }
        if (flags & 2) sd.field[s] = make_float2(mr, mi);
    }

    if (flags & 1) {
        for (int o = 16; o > 0; o >>= 1) {
            zr += __shfl_down_sync(0xffffffffu, zr, o);
            zi += __shfl_down_sync(0xffffffffu, zi, o);
        }
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) s_red[w] = make_double2(zr, zi);
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

    // Advance the step counter once every block of this launch has finished.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&a.ctl->done, 1u);
        if (prev == gridDim.x - 1) {
            a.ctl->done = 0;
            a.ctl->k = k + 1;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------- reduce
__global__ void reduce_kernel(const double2* __restrict__ partial, const long long* __restrict__ tile_start,
                              double2* __restrict__ out, double2* __restrict__ series, long long series_stride,
                              const StepCtl* ctl)
{
    __shared__ double2 sh[256];
    const int m = blockIdx.x;
    const long long t0 = tile_start[m], t1 = tile_start[m + 1];
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

// The control word is written by a kernel so its value travels as a launch
// argument (stream-ordered, no host staging buffer to keep alive).
__global__ void set_ctl_kernel(StepCtl* ctl, StepCtl v) { *ctl = v; }

}  // namespace

cudaError_t launch_set_ctl(StepCtl* ctl, const StepCtl& v, cudaStream_t st)
{
    set_ctl_kernel<<<1, 1, 0, st>>>(ctl, v);
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
    init_kernel<<<(unsigned)n_tiles, block, 0, st>>>(a.members, a.tile_start, a.n_members, spt, slot);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepArgs& a, long long n_tiles, int block, int spt, cudaStream_t st)
{
    switch (spt) {
    case 1: sweep_kernel<1><<<(unsigned)n_tiles, block, 0, st>>>(a); break;
    case 2: sweep_kernel<2><<<(unsigned)n_tiles, block, 0, st>>>(a); break;
    case 4: sweep_kernel<4><<<(unsigned)n_tiles, block, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double2* partial, const long long* tile_start, int n_members, double2* out,
                          double2* series, long long series_stride, const StepCtl* ctl, cudaStream_t st)
{
    reduce_kernel<<<n_members, 256, 0, st>>>(partial, tile_start, out, series, series_stride, ctl);
    return cudaGetLastError();
}

}  // namespace lbmbt
