// noalloc.cu -- lbmbt_sweep_noalloc: the plain sweep for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs where the device memory
// is owned by someone else's allocator (a framework's caching pool, a
// real-time loop that must not touch the driver's allocator, an embedding
// that forbids allocation after start-up).  This entry point runs the same
// kernels as lbmbt_run on buffers the caller already owns (mask, state) and
// keeps its own small working data -- member descriptor, tile prefix, step
// control word, waveform and boundary-factor tables, per-tile signal
// partials -- in one
// file-scope __device__ array of fixed size, which every GPU that loads the
// library holds until the process exits.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>

#include "lbmbt.h"
#include "lbmbt_internal.cuh"

using namespace lbmbt;

namespace {

constexpr int NA_BLOCK = 256;                       // fixed launch shape
constexpr int NA_SPT = 2;
constexpr long long NA_TILE = (long long)NA_BLOCK * NA_SPT;
constexpr long long NA_MAX_SITES = 1LL << 24;       // 16,777,216 sites (256^3)
constexpr long long NA_MAX_STEPS = 1LL << 15;       // 32,768 waveform samples
constexpr long long NA_MAX_TILES = NA_MAX_SITES / NA_TILE;

// byte offsets inside the scratch array
constexpr size_t OFF_CTL = 0;
constexpr size_t OFF_DESC = 256;
constexpr size_t OFF_TS = 768;
constexpr size_t OFF_Z = 1024;
constexpr size_t OFF_PH = 1056;                      // largest phase id in the caller's mask
constexpr size_t OFF_F64 = 1280;
constexpr size_t OFF_F32 = OFF_F64 + NA_MAX_STEPS * sizeof(double);
constexpr size_t OFF_FCUM = OFF_F32 + NA_MAX_STEPS * sizeof(float);
// boundary factors of every step, [K+1][1][6]
constexpr size_t OFF_FTAB = (OFF_FCUM + (NA_MAX_STEPS + 1) * sizeof(double) + 255) / 256 * 256;
constexpr size_t OFF_PART = (OFF_FTAB + (NA_MAX_STEPS + 1) * 6 * sizeof(float2) + 255) / 256 * 256;
constexpr size_t NA_SCRATCH_BYTES = OFF_PART + NA_MAX_TILES * sizeof(double2);
static_assert(sizeof(StepCtl) <= OFF_DESC - OFF_CTL, "control word does not fit");
static_assert(sizeof(MemberDesc) <= OFF_TS - OFF_DESC, "descriptor does not fit");
// 2,754,304 bytes (2.63 MiB), the figure the header states
static_assert(NA_SCRATCH_BYTES == 2754304, "scratch size differs from the documented figure");

// The scratch.  Host code must not pass `na_scratch` itself to a kernel: on
// the host it names a stand-in object, not device memory.  Its device address
// comes from cudaGetSymbolAddress (na_scratch_ptr below).
static __device__ __align__(256) unsigned char na_scratch[NA_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex na_mutex;
unsigned char* na_ptr[NA_MAX_DEVICES] = {};

__global__ void na_setup_kernel(unsigned char* base, MemberDesc d, long long n_tiles, int K, double dt)
{
    // descriptor and tile prefix
    *reinterpret_cast<MemberDesc*>(base + OFF_DESC) = d;
    long long* ts = reinterpret_cast<long long*>(base + OFF_TS);
    ts[0] = 0;
    ts[1] = n_tiles;
    // waveform tables from the caller's samples (copied to OFF_F64):
    // f_k as float and F_k = sum_{m<k} f_m dt in FP64, summed in order
    *reinterpret_cast<int*>(base + OFF_PH) = 0;   // cleared every call
    const double* f64 = reinterpret_cast<const double*>(base + OFF_F64);
    float* f32 = reinterpret_cast<float*>(base + OFF_F32);
    double* F = reinterpret_cast<double*>(base + OFF_FCUM);
    double acc = 0.0;
    for (int k = 0; k < K; ++k) {
        f32[k] = (float)f64[k];
        F[k] = acc;
        acc += f64[k] * dt;
    }
    F[K] = acc;
}

// Largest phase id (mask bits 6..7) over the caller's mask.
__global__ void na_phase_kernel(const uint8_t* __restrict__ mask, long long N, int* out)
{
    unsigned mx = 0;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x)
        mx = max(mx, (unsigned)(mask[s] >> 6));
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, (int)mx);
}

int na_fail(char* errbuf, size_t errlen, int code, const char* msg)
{
    if (errbuf && errlen) snprintf(errbuf, errlen, "%s", msg);
    return code;
}

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does it; it must not be inside a stream
// capture).
int na_scratch_ptr(int dev, unsigned char** out, char* errbuf, size_t errlen)
{
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(errbuf, errlen, LBMBT_EINVAL, "device ordinal too large");
    std::lock_guard<std::mutex> lk(na_mutex);
    if (!na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
        if (e != cudaSuccess || !p) {
            char m[256];
            snprintf(m, sizeof m, "cudaGetSymbolAddress of the scratch failed: %s", cudaGetErrorString(e));
            return na_fail(errbuf, errlen, LBMBT_ECUDA, m);
        }
        na_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = na_ptr[dev];
    return LBMBT_OK;
}

}  // namespace

extern "C" int lbmbt_sweep_noalloc(int nx, int ny, int nz, double dx_um, const uint8_t* mask_dev, const int bc[3],
                                   int n_phases, const double* D_um2_ms, const double* T2_ms, double kappa_um_ms,
                                   double dt_ms, int64_t n_total_steps, const double* f, const double gamma_G0[3],
                                   void* state_dev, int64_t k0, int64_t n_steps, int init, double* signal_out,
                                   void* cuda_stream, char* errbuf, size_t errlen)
{
    if (errbuf && errlen) errbuf[0] = 0;
    if (!mask_dev || !bc || !D_um2_ms || !T2_ms || !f || !gamma_G0 || !state_dev || !signal_out)
        return na_fail(errbuf, errlen, LBMBT_EINVAL, "NULL argument");
    if (nx < 1 || ny < 1 || nz < 1) return na_fail(errbuf, errlen, LBMBT_EINVAL, "grid sizes must be >= 1");
    const long long N = (long long)nx * ny * nz;
    if (N > NA_MAX_SITES)
        return na_fail(errbuf, errlen, LBMBT_EINVAL,
                       "grid larger than the no-allocation limit of 16,777,216 sites (use lbmbt_run)");
    if (n_total_steps < 1 || n_total_steps > NA_MAX_STEPS)
        return na_fail(errbuf, errlen, LBMBT_EINVAL,
                       "sequence longer than the no-allocation limit of 32,768 steps (use lbmbt_run)");
    if (k0 < 0 || n_steps < 1 || k0 + n_steps > n_total_steps)
        return na_fail(errbuf, errlen, LBMBT_EINVAL, "need 0 <= k0 and k0 + n_steps <= n_total_steps, n_steps >= 1");
    if (init && k0 != 0) return na_fail(errbuf, errlen, LBMBT_EINVAL, "init requires k0 = 0");
    if (!(dx_um > 0) || !(dt_ms > 0) || !(kappa_um_ms >= 0))
        return na_fail(errbuf, errlen, LBMBT_EINVAL, "dx, dt must be positive and kappa >= 0");
    if (n_phases < 1 || n_phases > 4) return na_fail(errbuf, errlen, LBMBT_EINVAL, "need 1..4 phases");
    for (int a = 0; a < 3; ++a)
        if ((bc[a] != LBMBT_BC_PERIODIC && bc[a] != LBMBT_BC_MIRROR) || !std::isfinite(gamma_G0[a]))
            return na_fail(errbuf, errlen, LBMBT_EINVAL, "bad boundary code or gradient");

    MemberDesc d;
    memset(&d, 0, sizeof d);
    d.mask = mask_dev;
    d.N = N;
    d.plane = (N + 63) / 64 * 64;
    d.nx = nx; d.ny = ny; d.nz = nz;
    d.dx = dx_um;
    d.state = static_cast<float2*>(state_dev);
    for (int a = 0; a < 3; ++a) {
        d.gG[a] = gamma_G0[a];
        d.ctheta[a] = (float)(-gamma_G0[a] * dx_um * dt_ms);
        if (bc[a] == LBMBT_BC_PERIODIC) d.bc[a] = BC_PER;
        else if (gamma_G0[a] == 0.0) d.bc[a] = BC_MIR;
        else {
            for (int b = 0; b < 3; ++b)
                if (b != a && gamma_G0[b] != 0.0)
                    return na_fail(errbuf, errlen, LBMBT_EUNSUPPORTED,
                                   "mirror face with a gradient neither normal nor parallel to it");
            d.bc[a] = BC_MIR_CONJ;
        }
    }
    for (int p = 0; p < 4; ++p) {
        const double Dp = p < n_phases ? D_um2_ms[p] : 1.0;
        const double T2p = p < n_phases ? T2_ms[p] : INFINITY;
        const double tau = 0.5 + dt_ms * Dp / (EPS_D * dx_um * dx_um);
        if (p < n_phases && !(tau > 0.5)) return na_fail(errbuf, errlen, LBMBT_EUNSTABLE, "tau <= 1/2");
        if (p < n_phases && !(T2p > 0)) return na_fail(errbuf, errlen, LBMBT_EINVAL, "T2 must be positive");
        d.omega[p] = (float)(1.0 / tau);
        d.eps[p] = std::isinf(T2p) ? 0.f : (float)(-std::expm1(-dt_ms / T2p));
    }
    const double cP = EPS_D * dx_um / (2.0 * dt_ms);
    d.s_share = std::isinf(kappa_um_ms) ? 1.f : (float)(kappa_um_ms / (kappa_um_ms + cP));
    d.axes = 0;
    for (int a = 0; a < 3; ++a)
        if (d.ctheta[a] != 0.f) d.axes |= 1 << a;
    d.nzg = nz;        // the whole grid (z0 = 0, no halo planes)
    d.zbc[0] = d.zbc[1] = d.bc[2];
    d.etab = nullptr;  // no tables here: the reaction angle uses sincosf
    d.memb = 1;        // the mask is the caller's: assume membranes may be present
    const unsigned dv[2] = {(unsigned)nx, (unsigned)ny};
    for (int j = 0; j < 2; ++j) {  // exact n / d for n < 2^28 (multiply-shift)
        int l = 0;
        while ((1ull << l) < dv[j]) ++l;
        d.div_m[j] = (unsigned)((1ull << (28 + l)) / dv[j] + 1);
        d.div_s[j] = 28 + l;
    }
    const long long n_tiles = (N + NA_TILE - 1) / NA_TILE;
    d.end_step = -1;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(errbuf, errlen, LBMBT_ECUDA, cudaGetErrorString(e));
    unsigned char* base = nullptr;
    int rc = na_scratch_ptr(dev, &base, errbuf, errlen);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    d.fw = reinterpret_cast<const float*>(base + OFF_F32);      // the waveform tables in the scratch
    d.Fw = reinterpret_cast<const double*>(base + OFF_FCUM);

    StepCtl c;
    memset(&c, 0, sizeof c);   // ticket counters start at zero every call
    c.k = (int)k0;
    c.done = 0;                                  // must start at zero every call
    c.sig_step = (int)(k0 + n_steps - 1);
    c.field_step = -1;
    c.slot_base = 0;
    c.slot_mod = 2;
    c.series = 0;
    c.err = 0;
    e = cudaMemcpyAsync(base + OFF_F64, f, n_total_steps * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        na_setup_kernel<<<1, 1, 0, st>>>(base, d, n_tiles, (int)n_total_steps, dt_ms);
        e = cudaGetLastError();
    }
    // every phase id in the mask must name one of the n_phases phases given;
    // checked before any state is touched
    int max_ph = 0;
    if (e == cudaSuccess) {
        const long long blocks = std::min<long long>((N + 255) / 256, 152LL * 8);
        na_phase_kernel<<<(unsigned)blocks, 256, 0, st>>>(mask_dev, N, reinterpret_cast<int*>(base + OFF_PH));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&max_ph, base + OFF_PH, sizeof max_ph, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return na_fail(errbuf, errlen, LBMBT_ECUDA, cudaGetErrorString(e));
    if (max_ph >= n_phases) {
        char m[128];
        snprintf(m, sizeof m, "the mask uses phase %d but %d phases are given", max_ph, n_phases);
        return na_fail(errbuf, errlen, LBMBT_ESTATE, m);
    }
    SweepArgs a;
    a.members = reinterpret_cast<const MemberDesc*>(base + OFF_DESC);
    a.tile_start = reinterpret_cast<const long long*>(base + OFF_TS);
    a.n_members = 1;
    a.ctl = reinterpret_cast<StepCtl*>(base + OFF_CTL);
    a.f = reinterpret_cast<const float*>(base + OFF_F32);
    a.F = reinterpret_cast<const double*>(base + OFF_FCUM);
    a.partial = reinterpret_cast<double2*>(base + OFF_PART);
    float2* ftab = reinterpret_cast<float2*>(base + OFF_FTAB);
    a.fac = ftab;
    a.links = 0;
    a.w0 = W0; a.wxy = WI; a.wz = WI;   // D3Q7
    a.scheme = 0;                       // the hybrid scheme
    a.test_wait_ns = 0;
    a.zc = 0;   // the register sweep: no z-marching columns
    a.zc_log2 = 0;
    a.n_cc = 0;
    a.cc_start = nullptr;
    MemberDesc* dd = reinterpret_cast<MemberDesc*>(base + OFF_DESC);
    // control word (done counter and step start from the values above every
    // call; each sweep's last block advances the step) and the boundary
    // factors of every step of the waveform
    if (e == cudaSuccess) e = launch_ctl_set(a.ctl, c, st);
    if (e == cudaSuccess) e = launch_factor_table(dd, 1, 0, n_total_steps, ftab, st);
    if (e == cudaSuccess && init) e = launch_init(a, n_tiles, NA_BLOCK, NA_SPT, 0, st);
    for (long long k = 0; e == cudaSuccess && k < n_steps; ++k) e = launch_sweep(a, n_tiles, NA_BLOCK, NA_SPT, st);
    double2* Zd = reinterpret_cast<double2*>(base + OFF_Z);
    if (e == cudaSuccess) e = launch_reduce(a.partial, a.tile_start, 1, 1, Zd, nullptr, 0, a.ctl, st);
    double2 Z = make_double2(0.0, 0.0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&Z, Zd, sizeof Z, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return na_fail(errbuf, errlen, LBMBT_ECUDA, cudaGetErrorString(e));
    signal_out[0] = Z.x;
    signal_out[1] = Z.y;
    signal_out[2] = std::hypot(Z.x, Z.y) / (double)N;
    return LBMBT_OK;
}
