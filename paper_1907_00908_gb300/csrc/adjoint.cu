// adjoint.cu -- reverse-time (adjoint) sweep of the hybrid LBM step for
// d S / d(D_p, T2_p, kappa), S = |Z|/N, Z = sum_x M(x, t^K).
//
// One forward step k maps the post-collision state u^k to u^(k+1):
//   g'^k    = S_k u^k               stream + outer BC + membranes (real-linear)
//   g^(k+1) = (1 + q_k) g'^k        reaction, q_k = exp(i theta)(1 - eps) - 1
//   u^(k+1) = C g^(k+1)             BGK collision, real coefficients
// With lambda^k = dS/du^k held as complex numbers (d/dRe + i d/dIm), the
// transposes are
//   C^T:   mu_j = (1 - omega) lambda_j + omega sum_i w_i lambda_i
//   R^T:   nu   = conj(1 + q) mu
//   S^T:   lambda_j(y) = sum over the forward consumers of u_j(y):
//            plain link         -> conj(fac) nu_j(y + e_j)
//            membrane link      -> s conj(fac) nu_j(y + e_j) + r nu_jbar(y)
//            mirror, plain      -> nu_jbar(y)
//            mirror, conjugate  -> conj(nu_jbar(y)) fac    (the map z -> conj(z) c
//                                                          is its own transpose)
// and lambda^K = Z / (N |Z|) at every population.  The parameters enter
//   omega_p = 1/tau_p : d u/d omega = w M - g            (sites of phase p)
//   eps_p             : d g/d eps   = -exp(i theta) g'   (sites of phase p)
//   s = 1/(1+P)       : d g'_i/d s  = v_i - o_i          (membrane links; v the
//                       population streaming across, o = u_ibar of the site)
// so dS/d(omega, eps, s) = sum_k <adjoint, derivative>, <a, b> = Re(conj(a) b).
//
// adjoint_kernel performs nu^k -> nu^(k-1) in one pass per site: it pulls
// nu^k from the downstream neighbours (lambda^k), recomputes g'^(k-1) and
// g^k from u^(k-1) (an upstream pull, as the forward sweep), accumulates the
// three sensitivities and writes nu^(k-1).
#include "lbmbt_internal.cuh"
#include "sweep_common.cuh"

namespace lbmbt {
namespace {

__device__ __forceinline__ float dotc(float2 a, float2 b) { return a.x * b.x + a.y * b.y; }

// Transposed stream of direction J = 1 + 2*AX + (SIGN > 0 ? 0 : 1) into site y
// (index s): reads the adjoint of the population's consumer.
template <int AX, int SIGN>
__device__ __forceinline__ float2 adj_pull(const float2* __restrict__ nu, unsigned P, unsigned s, int coord, int dim,
                                           unsigned stride, int bc, const float2* __restrict__ fac, bool memb,
                                           float sh)
{
    constexpr int J = 1 + 2 * AX + (SIGN > 0 ? 0 : 1);
    constexpr int JB = (SIGN > 0) ? J + 1 : J - 1;
    const bool cr = (SIGN > 0) ? (coord == dim - 1) : (coord == 0);
    if (cr && bc != BC_PER) {
        // mirror: u_J(y) feeds g'_JB(y), which crosses the high face (J = +e)
        // or the low face (J = -e).
        float2 v = __ldg(nu + (size_t)JB * P + s);
        if (bc == BC_MIR_CONJ) {
            v.y = -v.y;
            v = cmul(v, __ldg(fac + 2 * AX + (SIGN > 0 ? 1 : 0)));
        }
        return v;
    }
    unsigned nb = (SIGN > 0) ? s + stride : s - stride;
    if (cr) nb = (SIGN > 0) ? s - (unsigned)(dim - 1) * stride : s + (unsigned)(dim - 1) * stride;
    float2 v = __ldg(nu + (size_t)J * P + nb);
    if (cr) {  // periodic: the consumer is the wrapped node, pulling across its face
        const float2 f = __ldg(fac + 2 * AX + (SIGN > 0 ? 0 : 1));
        v = cmul(v, make_float2(f.x, -f.y));
    }
    if (memb) {
        const float2 o = __ldg(nu + (size_t)JB * P + s);
        v.x = o.x + sh * (v.x - o.x);
        v.y = o.y + sh * (v.y - o.y);
    }
    return v;
}

__device__ __forceinline__ float2 pull_dir(int i, const float2* __restrict__ src, unsigned P, unsigned s, int x,
                                           int y, int z, int nx, int ny, int nz, unsigned sxy, int bcx, int bcy,
                                           int bcz, const float2* __restrict__ fac)
{
    switch (i) {
    case 1: return pull<0, +1>(src, P, s, x, nx, 1u, bcx, fac);
    case 2: return pull<0, -1>(src, P, s, x, nx, 1u, bcx, fac);
    case 3: return pull<1, +1>(src, P, s, y, ny, (unsigned)nx, bcy, fac);
    case 4: return pull<1, -1>(src, P, s, y, ny, (unsigned)nx, bcy, fac);
    case 5: return pull<2, +1>(src, P, s, z, nz, sxy, bcz, fac);
    default: return pull<2, -1>(src, P, s, z, nz, sxy, bcz, fac);
    }
}

// Each block takes a run of `run` consecutive tiles.  The gradient partials
// stay in registers over the tiles of one member and are reduced, once per
// member in the run, into the slot of the member's first tile of the run:
// the tile-to-block map is fixed, so every step adds the same groups in
// the same order.
template <int SPT>
__global__ void __launch_bounds__(256) adjoint_kernel(const AdjointArgs a, long long n_tiles, int run)
{
    __shared__ float s_red[NGACC][32];

    const float fk = a.fprev;
    // D2Q5: the z populations and their adjoints are exactly 0 (weight 0,
    // nothing couples them to the others), so their planes are not touched
    const bool zpl = a.wz != 0.f;
    float acc[NGACC];
#pragma unroll
    for (int j = 0; j < NGACC; ++j) acc[j] = 0.f;

    // block reduction: FP32 within warps, FP64 across warps and steps
    auto flush = [&](long long slot) {
#pragma unroll
        for (int j = 0; j < NGACC; ++j)
            for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_down_sync(0xffffffffu, acc[j], o);
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0)
#pragma unroll
            for (int j = 0; j < NGACC; ++j) s_red[j][w] = acc[j];
        __syncthreads();
        if (threadIdx.x < NGACC) {
            double t = 0.0;
            const int nw = blockDim.x >> 5;
            for (int q = 0; q < nw; ++q) t += (double)s_red[threadIdx.x][q];
            a.gacc[(size_t)slot * NGACC + threadIdx.x] += t;
        }
        __syncthreads();   // s_red is free again
#pragma unroll
        for (int j = 0; j < NGACC; ++j) acc[j] = 0.f;
    };

    // constants of the current member, reloaded when the member changes
    int m = -1;
    long long t_first = 0;
    const MemberDesc* __restrict__ sd = a.members;
    const float2* __restrict__ facP = nullptr;   // boundary factors of step k-1
    const float2* __restrict__ facK = nullptr;   // and of step k
    float2 sL = make_float2(0.f, 0.f);
    unsigned P = 0, sxy = 0, N = 0;
    const float2* __restrict__ u = nullptr;
    const float2* __restrict__ nu = nullptr;
    float2* __restrict__ out = nullptr;
    const uint8_t* __restrict__ mask = nullptr;
    int nx = 1, ny = 1, nz = 1, bcx = 0, bcy = 0, bcz = 0;
    float sh = 0.f;

    const long long t0 = (long long)blockIdx.x * run, t1 = min(t0 + run, n_tiles);
    for (long long t = t0; t < t1; ++t) {   // block-uniform
        const int mt = a.n_members == 1 ? 0 : find_member(a.tile_start, a.n_members, t);
        if (mt != m) {
            if (m >= 0) flush(t_first);
            m = mt;
            t_first = t;
            sd = a.members + m;
            facP = a.ftab + ((size_t)(a.k - 1) * a.n_members + m) * 6;
            facK = a.ftab + ((size_t)a.k * a.n_members + m) * 6;
            if (a.first) {
                const double2 L = a.lam_init[m];
                sL = make_float2((float)L.x, (float)L.y);
            }
            P = (unsigned)sd->plane;
            u = sd->state + (size_t)a.fwd_slot * 7 * P;
            nu = sd->adj + (size_t)a.lam_parity * 7 * P;
            out = sd->adj + (size_t)(a.lam_parity ^ 1) * 7 * P;
            mask = sd->mask;
            nx = sd->nx; ny = sd->ny; nz = sd->nz;
            bcx = sd->bc[0]; bcy = sd->bc[1]; bcz = sd->bc[2];
            sxy = (unsigned)nx * ny;
            N = (unsigned)sd->N;
            sh = sd->s_share;
        }
        const unsigned base = (unsigned)(t - sd->tile0) * blockDim.x * SPT;

#pragma unroll
        for (int jj = 0; jj < SPT; ++jj) {
            const unsigned s = base + jj * blockDim.x + threadIdx.x;
            if (s >= N) break;
            int x, y, z;
            coords(sd, s, nx, ny, x, y, z);
            const unsigned mk = mask[s];
            const int ph = mk >> 6;

            // forward recompute of g'^(k-1) at this site (as the forward sweep)
            float2 gp[Q];
            gp[0] = __ldg(u + s);
            gp[1] = pull<0, +1>(u, P, s, x, nx, 1u, bcx, facP);
            gp[2] = pull<0, -1>(u, P, s, x, nx, 1u, bcx, facP);
            gp[3] = pull<1, +1>(u, P, s, y, ny, (unsigned)nx, bcy, facP);
            gp[4] = pull<1, -1>(u, P, s, y, ny, (unsigned)nx, bcy, facP);
            if (zpl) {
                gp[5] = pull<2, +1>(u, P, s, z, nz, sxy, bcz, facP);
                gp[6] = pull<2, -1>(u, P, s, z, nz, sxy, bcz, facP);
            } else {
                gp[5] = gp[6] = make_float2(0.f, 0.f);
            }
            if (mk & 0x3fu) {
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const int ib = (i & 1) ? i + 1 : i - 1;
                    if (mk & (1u << (ib - 1))) gp[i] = mix(__ldg(u + (size_t)ib * P + s), gp[i], sh);
                }
            }
            const float ep = sd->eps[ph];
            const float2 rot = fk != 0.f ? rotation_m1(sd, fk, x, y, z) : make_float2(0.f, 0.f);
            const float2 q = fk != 0.f ? reaction_q(rot, ep) : make_float2(-ep, 0.f);
            const float cm1 = rot.x, sn = rot.y;

            // lambda^k at this site
            float2 lam[Q];
            if (a.first) {
#pragma unroll
                for (int i = 0; i < Q; ++i) lam[i] = sL;
            } else {
                lam[0] = __ldg(nu + s);
                lam[1] = adj_pull<0, +1>(nu, P, s, x, nx, 1u, bcx, facK, mk & 1u, sh);
                lam[2] = adj_pull<0, -1>(nu, P, s, x, nx, 1u, bcx, facK, mk & 2u, sh);
                lam[3] = adj_pull<1, +1>(nu, P, s, y, ny, (unsigned)nx, bcy, facK, mk & 4u, sh);
                lam[4] = adj_pull<1, -1>(nu, P, s, y, ny, (unsigned)nx, bcy, facK, mk & 8u, sh);
                if (zpl) {
                    lam[5] = adj_pull<2, +1>(nu, P, s, z, nz, sxy, bcz, facK, mk & 16u, sh);
                    lam[6] = adj_pull<2, -1>(nu, P, s, z, nz, sxy, bcz, facK, mk & 32u, sh);
                } else {
                    lam[5] = lam[6] = make_float2(0.f, 0.f);
                }
            }

            // The reacted populations g_i = (1 + q) g'_i and mu = C^T lambda enter
            // only through sums over i: Sg = sum g'_i (M = (1 + q) Sg),
            // D = sum conj(lambda_i) g'_i (sum <lambda_i, g_i> = Re((1 + q) D)) and
            // lw = sum w_i lambda_i (mu_i = (1 - omega) lambda_i + omega lw).
            float sgr = 0.f, sgi = 0.f, dr = 0.f, di = 0.f, lwr = 0.f, lwi = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float w = i == 0 ? a.w0 : i < 5 ? a.wxy : a.wz;
                sgr += gp[i].x;
                sgi += gp[i].y;
                dr += lam[i].x * gp[i].x + lam[i].y * gp[i].y;
                di += lam[i].x * gp[i].y - lam[i].y * gp[i].x;
                lwr += w * lam[i].x;
                lwi += w * lam[i].y;
            }
            const float q1r = 1.f + q.x, q1i = q.y;
            const float Mr = q1r * sgr - q1i * sgi, Mi = q1r * sgi + q1i * sgr;
            // d/d omega: sum_i <lambda_i, w_i M - g_i> = Re(conj(lw) M) - Re((1 + q) D)
            const float dOm = (lwr * Mr + lwi * Mi) - (q1r * dr - q1i * di);
            const float om = sd->omega[ph], om1 = 1.f - om;
            const float er = 1.f + cm1, ei = sn;
            // d/d eps: -Re(exp(i theta) c), c = sum_i conj(mu_i) g'_i = (1 - omega) D + omega conj(lw) Sg
            const float cr = om1 * dr + om * (lwr * sgr + lwi * sgi);
            const float ci = om1 * di + om * (lwr * sgi - lwi * sgr);
            const float dEp = -(er * cr - ei * ci);
            // nu_i = conj(1 + q) mu_i = a lambda_i + b, a = conj(1 + q)(1 - omega), b = conj(1 + q) omega lw
            const float ar = q1r * om1, ai = -q1i * om1;
            const float br = om * (q1r * lwr + q1i * lwi), bi = om * (q1r * lwi - q1i * lwr);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float2 l = lam[i];
                lam[i] = make_float2(ar * l.x - ai * l.y + br, ar * l.y + ai * l.x + bi);
                if (i < 5 || zpl) __stcs(out + (size_t)i * P + s, lam[i]);
            }
            // d/d s on membrane links of step k-1: <nu_i, v_i - o_i>
            float dS = 0.f;
            if (mk & 0x3fu) {
                for (int i = 1; i < Q; ++i) {
                    const int ib = (i & 1) ? i + 1 : i - 1;
                    if (mk & (1u << (ib - 1))) {
                        const float2 v = pull_dir(i, u, P, s, x, y, z, nx, ny, nz, sxy, bcx, bcy, bcz, facP);
                        const float2 o = __ldg(u + (size_t)ib * P + s);
                        dS += dotc(lam[i], make_float2(v.x - o.x, v.y - o.y));
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                acc[p] += (ph == p) ? dOm : 0.f;
                acc[4 + p] += (ph == p) ? dEp : 0.f;
            }
            acc[8] += dS;
        }
    }
    if (m >= 0) flush(t_first);
}

__global__ void reduce_grad_kernel(const double* __restrict__ gacc, const long long* __restrict__ tile_start, int per,
                                   double* __restrict__ out)
{
    __shared__ double sh[NGACC][128];
    const int m = blockIdx.x;
    double v[NGACC];
#pragma unroll
    for (int j = 0; j < NGACC; ++j) v[j] = 0.0;
    for (long long t = tile_start[m] * per + threadIdx.x; t < tile_start[m + 1] * per; t += blockDim.x)
#pragma unroll
        for (int j = 0; j < NGACC; ++j) v[j] += gacc[t * NGACC + j];
#pragma unroll
    for (int j = 0; j < NGACC; ++j) sh[j][threadIdx.x] = v[j];
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < o)
#pragma unroll
            for (int j = 0; j < NGACC; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < NGACC) out[m * NGACC + threadIdx.x] = sh[threadIdx.x][0];
}

}  // namespace

cudaError_t launch_adjoint(const AdjointArgs& a, long long n_tiles, int block, int spt, int run, cudaStream_t st)
{
    if (block > 256 || run < 1) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)((n_tiles + run - 1) / run);
    switch (spt) {
    case 1: adjoint_kernel<1><<<grid, block, 0, st>>>(a, n_tiles, run); break;
    case 2: adjoint_kernel<2><<<grid, block, 0, st>>>(a, n_tiles, run); break;
    case 4: adjoint_kernel<4><<<grid, block, 0, st>>>(a, n_tiles, run); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce_grad(const double* gacc, const long long* tile_start, int per, int n_members, double* out,
                               cudaStream_t st)
{
    reduce_grad_kernel<<<n_members, 128, 0, st>>>(gacc, tile_start, per, out);
    return cudaGetLastError();
}

}  // namespace lbmbt
