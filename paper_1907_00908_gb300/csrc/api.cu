// api.cu -- host side of the C ABI declared in include/lbmbt.h.
//
// A context owns: the geometries (device mask bytes), the phase table, the
// sequence tables (f_k as float, F_k = sum_{m<k} f_m dt as double, both on
// the device), and the work of the current prepared run: member descriptors,
// the tile prefix of the work list, state buffers, per-tile partial sums and
// the step-control word.  Time steps are issued as sweep launches; with the
// graph option a chunk of sweeps is captured once per prepared run and
// replayed (the step index lives on the device, so one graph serves any k).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "lbmbt.h"
#include "lbmbt_internal.cuh"

using namespace lbmbt;

namespace {

struct Geom {
    int nx = 0, ny = 0, nz = 0;
    double dx = 0;
    int bc[3] = {0, 0, 0};
    long long N = 0;
    int max_phase = 0;
    int has_membranes = 0;
    uint8_t* d_mask = nullptr;
    // slab of a larger grid (z planes z0 .. z0+nz-1 of nzg); face kinds
    // LBMBT_FACE_OWN / _HALO / _HALO_WRAP of the low and high z face
    int slab = 0, z0 = 0, nzg = 0;
    int zkind[2] = {0, 0};
    float* d_dlt = nullptr;       // membrane positions on the links, [6][plane], or nullptr
    float* d_dth = nullptr;       // membrane angles on the links (2-D), [6][plane], or nullptr
};

constexpr int GRAPH_CHUNK = 16;

}  // namespace

struct lbmbt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t owned_stream = nullptr;
    std::string err;
    std::vector<Geom> geoms;
    int n_phases = 0;
    double D[4] = {0, 0, 0, 0};
    double T2[4] = {0, 0, 0, 0};
    double kappa = INFINITY;
    // sequence
    double dt = 0;
    long long n_steps = 0;
    std::vector<double> f;
    double gG[3] = {0, 0, 0};
    float* d_f = nullptr;
    double* d_F = nullptr;
    // options
    int use_graph = 1;
    int autotune = 0;
    int kernel_opt = 0;           // 0 auto, 1 register sweep, 2 bulk-copy sweep
    int block = 256;
    int spt = 2;
    long long launches = 0;
    // prepared run
    int n_members = 0;
    std::vector<lbmbt_member> members;
    std::vector<MemberDesc> descs;
    std::vector<long long> tile_start;
    long long n_tiles = 0;
    std::vector<long long> unit_start;
    long long n_units = 0;
    long long* d_unit_start = nullptr;
    size_t cap_us = 0;
    std::vector<long long> adj_unit_start;
    long long n_adj_units = 0;
    long long* d_adj_unit_start = nullptr;
    size_t cap_aus = 0;
    bool adj_tma_ok = false;
    int adj_cap = 0;
    int adjoint_opt = 0;          // 0 auto, 1 register adjoint, 2 bulk-copy adjoint
    int lattice = 0;              // 0 D3Q7, 1 D2Q5 (Sec. 2.3; grids of one z plane)
    int scheme = 0;               // 0 hybrid, 1 classical LBM with a reaction source (Eq. A12)
    int substeps = 1;             // reaction sub-steps folded into the waveform (hybrid only)
    int adj_shape = 2;            // bulk-copy adjoint consumer shape (15 warps x 1 site)
    int adj_shape_used = 2;       // the shape of the prepared run (2 falls back to 1 when an nx > 480)
    bool use_tma = false;
    int tma_cap = 0;
    int tma_capx = 0;
    int tma_stages = 3;
    int tma_variant = 3;
    int tma_form = 0;             // own z values: 0 prefetched, 1 staged, 2 z-marching columns
    int oz_opt = 0;               // 0 auto, 1 prefetch, 2 stage, 3 z-marching
    int tma_zc = 0;               // z-marching: units per column
    int zc_opt = 0;               // z-marching column length: 0 auto, else a power of two
    long long n_cc = 0;           // z-marching: columns of all members
    std::vector<long long> cc_start;
    long long* d_cc_start = nullptr;
    size_t cap_cc = 0;
    int tuned_kernel = 0;         // 0: untuned, 1 register, 2 bulk copy (auto follows it)
    int tuned_oz = 0;             // 0: untuned, else the own-z form the tuner chose (2 staged, 3 z-marching)
    struct Tuned { int kernel, block, spt, variant, stages, oz; };
    std::map<std::string, Tuned> tune_cache;
    int tma_grid = 0;
    int sm_count = 0;
    int tile_block = 0, tile_spt = 0;
    MemberDesc* d_desc = nullptr;
    long long* d_tile_start = nullptr;
    size_t cap_desc = 0, cap_ts = 0;
    double2* d_partial = nullptr;
    size_t cap_partial = 0;
    float2* d_ftab = nullptr;     // boundary factors of every step, [K+1][n_members][6]
    size_t cap_ftab = 0;
    bool ftab_valid = false;      // d_ftab holds the prepared members' factors
    int grad_groups = 0;          // member groups of the last lbmbt_grad_batch
    long long test_wait_ns = 0;   // tests of the bulk-copy sweep's timeout path (0: off)
    float2* d_etab = nullptr;     // per-member rotation tables
    size_t cap_etab = 0;
    float2* d_halo = nullptr;     // slab halo planes, [member][2][nx*ny]
    size_t cap_halo = 0;
    std::vector<size_t> halo_off; // per member offset into d_halo (elements)
    double2* d_Z = nullptr;
    size_t cap_Z = 0;
    double2* d_series = nullptr;
    size_t cap_series = 0;
    float2* d_state = nullptr;
    size_t cap_state = 0;  // bytes
    int n_slots = 2;
    StepCtl* d_ctl = nullptr;
    int* d_err = nullptr;
    long long k_cur = 0;
    bool prepared = false;
    bool series_mode = false;
    void* field_dev = nullptr;
    void* field_req = nullptr;    // lbmbt_set_field: field buffer for the next lbmbt_prepare
    cudaGraphExec_t graph = nullptr;
    int graph_series = -1;
    // adjoint buffers
    float2* d_ck = nullptr;
    size_t cap_ck = 0;
    float2* d_seg = nullptr;
    size_t cap_seg = 0;
    double* d_gacc = nullptr;
    size_t cap_gacc = 0;
    double* d_gout = nullptr;
    size_t cap_gout = 0;
    double2* d_laminit = nullptr;
    size_t cap_laminit = 0;
    // members' own waveforms (lbmbt_run_batch_ex): f [K+1] and F [K+2] per such member
    float* d_wf = nullptr;
    size_t cap_wf = 0;
    double* d_wF = nullptr;
    size_t cap_wF = 0;
};

static std::string g_create_error;

// Exact division of n < 2^28 by d (Granlund-Montgomery with 28-bit
// dividends): l = ceil(log2 d), m = floor(2^(28+l)/d) + 1, q = (n*m) >> (28+l).
static void div_magic(unsigned d, unsigned* m, int* s)
{
    int l = 0;
    while ((1ull << l) < d) ++l;
    *m = (unsigned)((1ull << (28 + l)) / d + 1);
    *s = 28 + l;
}

// Per-axis rotation table of one member: (cos(c n) - 1, sin(c n)), c = -gG_a dx dt.
static void rotation_table(const double gG[3], double dx, double dt, const int dims[3], int z0,
                           std::vector<float2>& out)
{
    for (int a = 0; a < 3; ++a) {
        const double c = -gG[a] * dx * dt;
        for (int n = 0; n < dims[a]; ++n) {
            const double t = c * (n + (a == 2 ? z0 : 0));
            const double h = std::sin(0.5 * t);
            out.push_back(make_float2((float)(-2.0 * h * h), (float)std::sin(t)));
        }
    }
}

static int fail(lbmbt_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_create_error = buf;
    return code;
}

#define CU(c, call)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail((c), e_ == cudaErrorMemoryAllocation ? LBMBT_ENOMEM : LBMBT_ECUDA,       \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);   \
    } while (0)

template <class T>
static int grow(lbmbt_ctx* c, T** p, size_t* cap, size_t bytes)
{
    if (*cap >= bytes && *p) return LBMBT_OK;
    if (*p) { cudaFree(*p); *p = nullptr; *cap = 0; }
    if (bytes == 0) return LBMBT_OK;
    CU(c, cudaMalloc((void**)p, bytes));
    *cap = bytes;
    return LBMBT_OK;
}

static void drop_graph(lbmbt_ctx* c)
{
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    c->graph_series = -1;
}

static int set_device(lbmbt_ctx* c)
{
    CU(c, cudaSetDevice(c->device));
    return LBMBT_OK;
}

// ------------------------------------------------------------------ basics
extern "C" const char* lbmbt_version(void) { return "lbmbt 0.1 (sm_103a)"; }

extern "C" int lbmbt_create(lbmbt_ctx** out, int device, void* cuda_stream)
{
    if (!out) return fail(nullptr, LBMBT_EINVAL, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return fail(nullptr, LBMBT_ECUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= n) return fail(nullptr, LBMBT_EINVAL, "device %d out of range (%d)", device, n);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, LBMBT_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    lbmbt_ctx* c = new lbmbt_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (!c->stream) {
        // The legacy default stream cannot be captured into a graph; use an
        // owned blocking stream, which still orders with the legacy stream.
        if (cudaStreamCreate(&c->owned_stream) != cudaSuccess) {
            delete c;
            return fail(nullptr, LBMBT_ECUDA, "stream creation failed");
        }
        c->stream = c->owned_stream;
    }
    if (cudaMalloc(&c->d_ctl, sizeof(StepCtl)) != cudaSuccess ||
        cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess) {
        lbmbt_destroy(c);
        return fail(nullptr, LBMBT_ENOMEM, "allocation of control words failed");
    }
    *out = c;
    return LBMBT_OK;
}

extern "C" int lbmbt_destroy(lbmbt_ctx* c)
{
    if (!c) return LBMBT_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
    drop_graph(c);
    for (auto& g : c->geoms) { cudaFree(g.d_mask); cudaFree(g.d_dlt); cudaFree(g.d_dth); }
    cudaFree(c->d_f); cudaFree(c->d_F);
    cudaFree(c->d_desc); cudaFree(c->d_tile_start); cudaFree(c->d_partial); cudaFree(c->d_Z);
    cudaFree(c->d_series); cudaFree(c->d_state); cudaFree(c->d_ctl); cudaFree(c->d_err);
    cudaFree(c->d_ftab); cudaFree(c->d_unit_start); cudaFree(c->d_etab); cudaFree(c->d_cc_start);
    cudaFree(c->d_adj_unit_start); cudaFree(c->d_halo);
    cudaFree(c->d_ck); cudaFree(c->d_seg); cudaFree(c->d_gacc); cudaFree(c->d_gout); cudaFree(c->d_laminit);
    if (c->owned_stream) cudaStreamDestroy(c->owned_stream);
    delete c;
    return LBMBT_OK;
}

extern "C" const char* lbmbt_last_error(const lbmbt_ctx* c)
{
    return c ? c->err.c_str() : g_create_error.c_str();
}

static int sync(lbmbt_ctx* c)
{
    CU(c, cudaStreamSynchronize(c->stream));
    return LBMBT_OK;
}

// ---------------------------------------------------------------- geometry
static int make_geom(lbmbt_ctx* c, int nx, int ny, int nz, double dx, const int32_t* labels, int on_dev,
                     int n_labels, const uint8_t* pol, const int bc[3], Geom* out)
{
    if (nx < 1 || ny < 1 || nz < 1) return fail(c, LBMBT_EINVAL, "grid sizes must be >= 1");
    const long long N = (long long)nx * ny * nz;
    if (N > (1LL << 28)) return fail(c, LBMBT_EINVAL, "grid of %lld sites exceeds 2^28", N);
    if (!(dx > 0) || !std::isfinite(dx)) return fail(c, LBMBT_EINVAL, "dx must be positive");
    if (!labels || !pol || !bc || n_labels < 1) return fail(c, LBMBT_EINVAL, "labels/phase table missing");
    int maxp = 0;
    for (int i = 0; i < n_labels; ++i) {
        if (pol[i] > 3) return fail(c, LBMBT_EINVAL, "phase_of_label[%d] = %d > 3", i, (int)pol[i]);
        if (pol[i] > maxp) maxp = pol[i];
    }
    for (int a = 0; a < 3; ++a)
        if (bc[a] != LBMBT_BC_PERIODIC && bc[a] != LBMBT_BC_MIRROR)
            return fail(c, LBMBT_EINVAL, "bc[%d] = %d invalid", a, bc[a]);
    int rc = set_device(c);
    if (rc) return rc;
    int32_t* d_lab = nullptr;
    uint8_t* d_pol = nullptr;
    uint8_t* d_mask = nullptr;
    auto cleanup = [&]() { cudaFree(d_lab); cudaFree(d_pol); };
    if (!on_dev) {
        if (cudaMalloc(&d_lab, N * sizeof(int32_t)) != cudaSuccess) { cleanup(); return fail(c, LBMBT_ENOMEM, "label buffer"); }
        if (cudaMemcpyAsync(d_lab, labels, N * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
            cleanup(); return fail(c, LBMBT_ECUDA, "label upload failed");
        }
    }
    if (cudaMalloc(&d_pol, n_labels) != cudaSuccess || cudaMalloc(&d_mask, N) != cudaSuccess) {
        cleanup(); cudaFree(d_mask); return fail(c, LBMBT_ENOMEM, "mask buffer");
    }
    cudaMemcpyAsync(d_pol, pol, n_labels, cudaMemcpyHostToDevice, c->stream);
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    cudaError_t e = launch_build_mask(on_dev ? labels : d_lab, d_pol, n_labels, nx, ny, nz, bc, d_mask, c->d_err,
                                      c->stream);
    c->launches++;
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cleanup();
    if (e != cudaSuccess) { cudaFree(d_mask); return fail(c, LBMBT_ECUDA, "mask build: %s", cudaGetErrorString(e)); }
    if (herr & 1) { cudaFree(d_mask); return fail(c, LBMBT_EDEVICE, "a label is outside [0, %d)", n_labels); }
    out->nx = nx; out->ny = ny; out->nz = nz; out->dx = dx; out->N = N; out->max_phase = maxp;
    out->has_membranes = (herr & 2) ? 1 : 0;
    for (int a = 0; a < 3; ++a) out->bc[a] = bc[a];
    out->d_mask = d_mask;
    return LBMBT_OK;
}

static void invalidate_run(lbmbt_ctx* c)
{
    c->prepared = false;
    c->ftab_valid = false;
    drop_graph(c);
}

extern "C" int lbmbt_set_geometry(lbmbt_ctx* c, int nx, int ny, int nz, double dx, const int32_t* labels,
                                  int on_dev, int n_labels, const uint8_t* pol, const int bc[3])
{
    if (!c) return LBMBT_EINVAL;
    Geom g;
    int rc = make_geom(c, nx, ny, nz, dx, labels, on_dev, n_labels, pol, bc, &g);
    if (rc) return rc;
    invalidate_run(c);
    for (auto& o : c->geoms) { cudaFree(o.d_mask); cudaFree(o.d_dlt); cudaFree(o.d_dth); }
    c->geoms.clear();
    c->geoms.push_back(g);
    return LBMBT_OK;
}

extern "C" int lbmbt_add_geometry(lbmbt_ctx* c, int nx, int ny, int nz, double dx, const int32_t* labels,
                                  int on_dev, int n_labels, const uint8_t* pol, const int bc[3], int* index_out)
{
    if (!c) return LBMBT_EINVAL;
    Geom g;
    int rc = make_geom(c, nx, ny, nz, dx, labels, on_dev, n_labels, pol, bc, &g);
    if (rc) return rc;
    invalidate_run(c);
    c->geoms.push_back(g);
    if (index_out) *index_out = (int)c->geoms.size() - 1;
    return LBMBT_OK;
}

// Slab of a grid cut along z (the strips of Sec. 2.5): labels_ext holds
// nz + 2 planes, the plane below the slab, the slab's nz planes, the plane
// above.  The mask is built over the extended block (z wrapped, which only
// the ghost planes see) and its nz interior planes are kept, so the links of
// the face planes compare with the neighbouring slab's labels.  A face of
// kind OWN is the global mirror face: its ghost plane is replaced by a copy
// of the face plane first, so the face links carry no membrane bit.
extern "C" int lbmbt_set_geometry_slab(lbmbt_ctx* c, int nx, int ny, int nz, double dx, const int32_t* labels_ext,
                                       int on_dev, int n_labels, const uint8_t* pol, const int bc[3], int z0,
                                       int nz_global, int lo_kind, int hi_kind)
{
    if (!c) return LBMBT_EINVAL;
    if (!labels_ext || !bc) return fail(c, LBMBT_EINVAL, "labels/bc missing");
    if (nx < 1 || ny < 1 || nz < 1) return fail(c, LBMBT_EINVAL, "grid sizes must be >= 1");
    if (z0 < 0 || nz_global < 1 || z0 + nz > nz_global)
        return fail(c, LBMBT_EINVAL, "slab planes [%d, %d) outside the grid of %d planes", z0, z0 + nz, nz_global);
    const int kinds[2] = {lo_kind, hi_kind};
    for (int h = 0; h < 2; ++h) {
        const int k = kinds[h];
        if (k != LBMBT_FACE_OWN && k != LBMBT_FACE_HALO && k != LBMBT_FACE_HALO_WRAP)
            return fail(c, LBMBT_EINVAL, "face kind %d invalid", k);
        if (k == LBMBT_FACE_OWN && bc[2] != LBMBT_BC_MIRROR)
            return fail(c, LBMBT_EINVAL, "a slab face of its own must be a global mirror face (a periodic whole "
                                         "grid is a plain geometry)");
        if (k == LBMBT_FACE_HALO_WRAP && bc[2] != LBMBT_BC_PERIODIC)
            return fail(c, LBMBT_EINVAL, "a wrapping halo face needs a periodic z axis");
    }
    if (bc[2] == LBMBT_BC_MIRROR &&
        ((lo_kind == LBMBT_FACE_OWN) != (z0 == 0) || (hi_kind == LBMBT_FACE_OWN) != (z0 + nz == nz_global)))
        return fail(c, LBMBT_EINVAL, "a face is the global mirror face iff the slab touches it");
    if ((lo_kind == LBMBT_FACE_HALO_WRAP) != (z0 == 0 && bc[2] == LBMBT_BC_PERIODIC) ||
        (hi_kind == LBMBT_FACE_HALO_WRAP) != (z0 + nz == nz_global && bc[2] == LBMBT_BC_PERIODIC))
        return fail(c, LBMBT_EINVAL, "the faces on the periodic global face must wrap, the others must not");
    if (nx % 2) return fail(c, LBMBT_EINVAL, "a slab needs an even nx");
    const long long sxy = (long long)nx * ny;
    const long long Next = sxy * (nz + 2);
    if (Next > (1LL << 28)) return fail(c, LBMBT_EINVAL, "slab of %lld sites (with ghost planes) exceeds 2^28", Next);
    int rc = set_device(c);
    if (rc) return rc;
    int32_t* d_lab = nullptr;
    if (cudaMalloc(&d_lab, Next * sizeof(int32_t)) != cudaSuccess) return fail(c, LBMBT_ENOMEM, "label buffer");
    auto kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(d_lab, labels_ext, Next * sizeof(int32_t), kind, c->stream);
    if (e == cudaSuccess && lo_kind == LBMBT_FACE_OWN)
        e = cudaMemcpyAsync(d_lab, d_lab + sxy, sxy * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && hi_kind == LBMBT_FACE_OWN)
        e = cudaMemcpyAsync(d_lab + (nz + 1) * sxy, d_lab + nz * sxy, sxy * sizeof(int32_t),
                            cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) {
        cudaFree(d_lab);
        return fail(c, LBMBT_ECUDA, "label upload: %s", cudaGetErrorString(e));
    }
    const int bce[3] = {bc[0], bc[1], LBMBT_BC_PERIODIC};
    Geom ext;
    rc = make_geom(c, nx, ny, nz + 2, dx, d_lab, 1, n_labels, pol, bce, &ext);
    cudaFree(d_lab);
    if (rc) return rc;
    uint8_t* d_mask = nullptr;
    if (cudaMalloc(&d_mask, sxy * nz) != cudaSuccess) {
        cudaFree(ext.d_mask);
        return fail(c, LBMBT_ENOMEM, "mask buffer");
    }
    e = cudaMemcpyAsync(d_mask, ext.d_mask + sxy, sxy * nz, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(ext.d_mask);
    if (e != cudaSuccess) {
        cudaFree(d_mask);
        return fail(c, LBMBT_ECUDA, "mask copy: %s", cudaGetErrorString(e));
    }
    Geom g = ext;
    g.nz = nz;
    g.N = sxy * nz;
    for (int a = 0; a < 3; ++a) g.bc[a] = bc[a];
    g.d_mask = d_mask;
    g.slab = 1;
    g.z0 = z0;
    g.nzg = nz_global;
    g.zkind[0] = lo_kind;
    g.zkind[1] = hi_kind;
    invalidate_run(c);
    for (auto& o : c->geoms) { cudaFree(o.d_mask); cudaFree(o.d_dlt); cudaFree(o.d_dth); }
    c->geoms.clear();
    c->geoms.push_back(g);
    return LBMBT_OK;
}

extern "C" int lbmbt_get_mask(lbmbt_ctx* c, int index, uint8_t* mask_out)
{
    if (!c) return LBMBT_EINVAL;
    if (index < 0 || index >= (int)c->geoms.size()) return fail(c, LBMBT_EINVAL, "geometry %d not set", index);
    if (!mask_out) return fail(c, LBMBT_EINVAL, "mask_out is NULL");
    int rc = set_device(c);
    if (rc) return rc;
    const Geom& g = c->geoms[index];
    CU(c, cudaMemcpyAsync(mask_out, g.d_mask, g.N, cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
}

// Membrane positions on the links of geometry `index` (theta = 0 rule,
// Eqs. B4a-B4c): delta [6][nz][ny][nx] float32, entry j-1 at a node is the
// distance in dx from the node to the membrane on its link to node + e_j,
// read on membrane links only.  NULL removes them (half-link rule, Eq. B5).
extern "C" int lbmbt_set_link_distances(lbmbt_ctx* c, int index, const float* delta, int on_device)
{
    if (!c) return LBMBT_EINVAL;
    if (index < 0 || index >= (int)c->geoms.size()) return fail(c, LBMBT_EINVAL, "geometry %d not set", index);
    int rc = set_device(c);
    if (rc) return rc;
    Geom& g = c->geoms[index];
    invalidate_run(c);
    cudaFree(g.d_dlt);
    g.d_dlt = nullptr;
    if (!delta) {   // the angles go with the positions
        cudaFree(g.d_dth);
        g.d_dth = nullptr;
        return LBMBT_OK;
    }
    if (g.slab) return fail(c, LBMBT_EUNSUPPORTED, "membrane positions on a slab are not supported");
    if (!on_device)
        for (long long i = 0; i < 6 * g.N; ++i)
            if (!(delta[i] > 0.f && delta[i] < 1.f))
                return fail(c, LBMBT_EINVAL, "membrane position %g at entry %lld outside (0, 1)", (double)delta[i], i);
    const long long plane = (g.N + 63) / 64 * 64;
    CU(c, cudaMalloc(&g.d_dlt, sizeof(float) * 6 * plane));
    const auto kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int j = 0; j < 6; ++j)
        CU(c, cudaMemcpyAsync(g.d_dlt + j * plane, delta + j * g.N, sizeof(float) * g.N, kind, c->stream));
    return sync(c);
}

// Smallest tau (every phase) at which runs with membrane angles are accepted.
constexpr double ANGLE_TAU_MIN = 0.75;

// Membrane angles on the links of a one-plane geometry `index` (the
// general-angle rule of Appendix B): theta [6][1][ny][nx] float32, entry j-1
// at a node is the signed angle between the membrane normal (from the node's
// compartment to the neighbour's) and its link to the neighbour across +e_j,
// normal = cos(theta) e_j + sin(theta) e_perp with e_perp = +y for x links,
// +x for y links; |theta| < pi/2.  Needs the positions first.  NULL removes
// them.
extern "C" int lbmbt_set_link_angles(lbmbt_ctx* c, int index, const float* theta, int on_device)
{
    if (!c) return LBMBT_EINVAL;
    if (index < 0 || index >= (int)c->geoms.size()) return fail(c, LBMBT_EINVAL, "geometry %d not set", index);
    int rc = set_device(c);
    if (rc) return rc;
    Geom& g = c->geoms[index];
    invalidate_run(c);
    cudaFree(g.d_dth);
    g.d_dth = nullptr;
    if (!theta) return LBMBT_OK;
    if (!g.d_dlt) return fail(c, LBMBT_EINVAL, "membrane angles need the membrane positions first");
    if (g.nz != 1) return fail(c, LBMBT_EINVAL, "membrane angles are defined on one-plane (2-D) grids only");
    if (!on_device)
        for (long long i = 0; i < 6 * g.N; ++i)
            if (!(std::fabs(theta[i]) < 1.5707963f))
                return fail(c, LBMBT_EINVAL, "membrane angle %g at entry %lld not in (-pi/2, pi/2)",
                            (double)theta[i], i);
    const long long plane = (g.N + 63) / 64 * 64;
    CU(c, cudaMalloc(&g.d_dth, sizeof(float) * 6 * plane));
    const auto kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int j = 0; j < 6; ++j)
        CU(c, cudaMemcpyAsync(g.d_dth + j * plane, theta + j * g.N, sizeof(float) * g.N, kind, c->stream));
    return sync(c);
}

// ------------------------------------------------------------ physics setup
extern "C" int lbmbt_set_phases(lbmbt_ctx* c, int n, const double* D, const double* T2)
{
    if (!c) return LBMBT_EINVAL;
    if (n < 1 || n > 4 || !D || !T2) return fail(c, LBMBT_EINVAL, "need 1..4 phases with D and T2");
    for (int p = 0; p < n; ++p) {
        if (!(D[p] > 0) || !std::isfinite(D[p])) return fail(c, LBMBT_EINVAL, "D[%d] must be positive", p);
        if (!(T2[p] > 0)) return fail(c, LBMBT_EINVAL, "T2[%d] must be positive", p);
    }
    c->n_phases = n;
    for (int p = 0; p < 4; ++p) { c->D[p] = p < n ? D[p] : 1.0; c->T2[p] = p < n ? T2[p] : INFINITY; }
    invalidate_run(c);
    return LBMBT_OK;
}

extern "C" int lbmbt_set_permeability(lbmbt_ctx* c, double kappa)
{
    if (!c) return LBMBT_EINVAL;
    if (!(kappa >= 0)) return fail(c, LBMBT_EINVAL, "kappa must be >= 0 (INFINITY allowed)");
    c->kappa = kappa;
    invalidate_run(c);
    return LBMBT_OK;
}

extern "C" int lbmbt_set_sequence(lbmbt_ctx* c, double dt, int64_t n_steps, const double* f, const double gG[3])
{
    if (!c) return LBMBT_EINVAL;
    if (!(dt > 0) || !std::isfinite(dt)) return fail(c, LBMBT_EINVAL, "dt must be positive");
    if (n_steps < 1 || n_steps > (1LL << 30)) return fail(c, LBMBT_EINVAL, "n_steps out of range");
    if (!f || !gG) return fail(c, LBMBT_EINVAL, "f / gamma_G0 missing");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(gG[a])) return fail(c, LBMBT_EINVAL, "gamma_G0 not finite");
    for (long long k = 0; k < n_steps; ++k)
        if (!std::isfinite(f[k])) return fail(c, LBMBT_EINVAL, "f[%lld] not finite", k);
    int rc = set_device(c);
    if (rc) return rc;
    invalidate_run(c);
    c->dt = dt;
    c->n_steps = n_steps;
    c->f.assign(f, f + n_steps);
    for (int a = 0; a < 3; ++a) c->gG[a] = gG[a];
    c->substeps = 1;
    // f_k and F_k with one entry past the end (f_K = 0, F_(K+1) = F_K): the
    // classical scheme's pass k reads them one step ahead
    std::vector<float> ff(n_steps + 1, 0.f);
    std::vector<double> FF(n_steps + 2);
    double F = 0.0;
    for (long long k = 0; k < n_steps; ++k) {
        ff[k] = (float)f[k];
        FF[k] = F;                  // F_k = sum_{m<k} f_m dt (Eq. periodic_phi)
        F += f[k] * dt;
    }
    FF[n_steps] = F;
    FF[n_steps + 1] = F;
    cudaFree(c->d_f); cudaFree(c->d_F);
    c->d_f = nullptr; c->d_F = nullptr;
    CU(c, cudaMalloc(&c->d_f, (n_steps + 1) * sizeof(float)));
    CU(c, cudaMalloc(&c->d_F, (n_steps + 2) * sizeof(double)));
    CU(c, cudaMemcpyAsync(c->d_f, ff.data(), (n_steps + 1) * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CU(c, cudaMemcpyAsync(c->d_F, FF.data(), (n_steps + 2) * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    return sync(c);
}

// Reaction sub-steps (Sec. 2.3, dt = k dt'): k reaction steps of dt' after
// each diffusion step.  The reaction factors of one site are scalars that
// commute, so the k sub-steps equal one reaction with the step-mean waveform
// exp(-i gamma x.G0 dt' sum_j f_j) (the T2 factors multiply to exp(-dt/T2)),
// and F_k = sum f dt' is unchanged: the sequence becomes the step means.
extern "C" int lbmbt_set_sequence_substeps(lbmbt_ctx* c, double dt, int64_t n_steps, int substeps,
                                           const double* f_fine, const double gG[3])
{
    if (!c) return LBMBT_EINVAL;
    if (substeps < 1) return fail(c, LBMBT_EINVAL, "substeps must be >= 1");
    if (!f_fine) return fail(c, LBMBT_EINVAL, "f missing");
    if (n_steps < 1 || n_steps > (1LL << 30) / substeps) return fail(c, LBMBT_EINVAL, "n_steps out of range");
    std::vector<double> fm(n_steps);
    for (long long k = 0; k < n_steps; ++k) {
        double acc = 0.0;
        for (int j = 0; j < substeps; ++j) acc += f_fine[k * substeps + j];
        fm[k] = acc / substeps;
    }
    const int rc = lbmbt_set_sequence(c, dt, n_steps, fm.data(), gG);
    if (rc == LBMBT_OK) c->substeps = substeps;
    return rc;
}

extern "C" int lbmbt_pgse(double b, double delta, double Delta, double dt, const double dir[3], double gG_out[3],
                          int64_t* n_steps_out, double* f_out)
{
    if (!dir || !gG_out || !n_steps_out) return LBMBT_EINVAL;
    if (!(dt > 0) || !(delta > 0) || !(Delta >= delta) || !(b >= 0)) return LBMBT_EINVAL;
    const double nd = delta / dt, nD = Delta / dt;
    if (std::fabs(nd - std::round(nd)) > 1e-9 * std::fmax(1.0, nd) ||
        std::fabs(nD - std::round(nD)) > 1e-9 * std::fmax(1.0, nD))
        return LBMBT_EINVAL;
    const long long id = (long long)std::llround(nd), iD = (long long)std::llround(nD);
    const double nrm = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    if (!(nrm > 0)) return LBMBT_EINVAL;
    // b [s/mm^2] * 1e-3 = b [ms/um^2];  b = (gamma G0)^2 delta^2 (Delta - delta/3)  (Sec. 2.1)
    const double g = b > 0 ? std::sqrt(b * 1e-3 / (delta * delta * (Delta - delta / 3.0))) : 0.0;
    for (int a = 0; a < 3; ++a) gG_out[a] = g * dir[a] / nrm;
    *n_steps_out = iD + id;
    if (f_out)
        for (long long k = 0; k < iD + id; ++k) f_out[k] = k < id ? 1.0 : (k >= iD ? -1.0 : 0.0);
    return LBMBT_OK;
}

// ------------------------------------------------------------- run set-up
// Row units of the bulk-copy sweep: rpu x-rows of one z-plane, about 512
// sites per unit.  Eligible when every member has nx % 16 == 0 (16-byte
// aligned rows and mask bytes) and a unit fits the shared-memory stages.
static constexpr int TMA_TARGET_SITES = 1024;
static constexpr int TMA_MAX_CAP = 1024;
// Planes from this many sites on: the own z rows of a membrane geometry are
// staged with the unit (a register prefetch of them would wait on DRAM, the
// rows being next touched a plane later); below it the register prefetch is
// faster (the rows are still in L2, and the smaller stage leaves more L1).
static constexpr long long TMA_OZ_PLANE = 1LL << 17;

static bool tma_eligible(const lbmbt_ctx* c)
{
    if (c->lattice != 0) return false;   // the bulk-copy sweep has the D3Q7 weights built in
    for (auto& d : c->descs)
        if (d.nx % 16 != 0 || d.nx > TMA_MAX_CAP || d.dlt != nullptr) return false;
    return true;
}

// Offset into the F_k tables of the boundary-factor table: the
// hybrid scheme streams before step k's reaction (F_k); the classical
// scheme's streamed populations already hold step k's source, so its faces
// take F_(k+1).
static int ctl_F_shift(const lbmbt_ctx* c) { return c->scheme == 1 ? 1 : 0; }

static int build_worklist(lbmbt_ctx* c, int block, int spt)
{
    const long long tile = (long long)block * spt;
    c->tile_start.assign(c->n_members + 1, 0);
    c->unit_start.assign(c->n_members + 1, 0);
    c->adj_unit_start.assign(c->n_members + 1, 0);
    int adj_cap = 16;
    bool adj_ok = true;
    c->adj_shape_used = c->adj_shape;
    for (auto& d : c->descs)
        if (c->adj_shape == 2 && d.nx > adj_tma_max_sites(2)) c->adj_shape_used = 1;
    const int adj_sites = adj_tma_max_sites(c->adj_shape_used);
    const bool want = c->kernel_opt == 2 || (c->kernel_opt == 0 && c->tuned_kernel != 1);
    const bool tma = want && tma_eligible(c);
    if (c->kernel_opt == 2 && !tma)
        return fail(c, LBMBT_EINVAL, "bulk-copy sweep needs nx %% 16 == 0 and nx <= %d for every member, no "
                                     "membrane positions and the D3Q7 lattice", TMA_MAX_CAP);
    int cap = 16, capx = 0;
    for (int m = 0; m < c->n_members; ++m) {
        MemberDesc& d = c->descs[m];
        d.tile0 = c->tile_start[m];
        c->tile_start[m + 1] = c->tile_start[m] + (d.N + tile - 1) / tile;
        d.rpu = std::max(1, std::min(d.ny, TMA_TARGET_SITES / std::max(1, d.nx)));
        d.unit0 = c->unit_start[m];
        c->unit_start[m + 1] = c->unit_start[m] + (long long)d.nz * ((d.ny + d.rpu - 1) / d.rpu);
        d.rpu_adj = std::max(1, std::min(d.ny, adj_sites / std::max(1, d.nx)));
        d.unit0_adj = c->adj_unit_start[m];
        c->adj_unit_start[m + 1] = c->adj_unit_start[m] + (long long)d.nz * ((d.ny + d.rpu_adj - 1) / d.rpu_adj);
        adj_cap = std::max(adj_cap, d.rpu_adj * d.nx);
        if (d.nx > adj_sites) adj_ok = false;
        cap = std::max(cap, d.rpu * d.nx);
        (void)capx;   // the x rotation table is read through L1, not staged
    }
    c->n_tiles = c->tile_start[c->n_members];
    c->n_units = c->unit_start[c->n_members];
    c->n_adj_units = c->adj_unit_start[c->n_members];
    c->adj_tma_ok = adj_ok && tma_eligible(c);
    c->adj_cap = (adj_cap + 15) / 16 * 16;
    if (c->n_tiles > 0x7fffffffLL) return fail(c, LBMBT_EINVAL, "work list too long");
    c->use_tma = tma;
    if (tma) {
        c->tma_cap = (cap + 15) / 16 * 16;
        c->tma_capx = (capx + 15) / 16 * 16;
        if (!c->sm_count) CU(c, cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
        // where the own z values of membrane lanes come from: on large planes
        // with membranes z-marching columns (each row read once, no own value
        // from global memory) when the grid gives enough columns of >= 8
        // planes, else staged with the unit; otherwise prefetched
        bool large = false;
        for (auto& d : c->descs)
            if (d.memb && (long long)d.nx * d.ny >= TMA_OZ_PLANE) large = true;
        int gz = 0;   // column length must divide every member's nz
        for (auto& d : c->descs) gz = std::gcd(gz, d.nz);
        auto columns = [&](int zc) {
            long long n = 0;
            for (auto& d : c->descs) n += (long long)(d.nz / zc) * ((d.ny + d.rpu - 1) / d.rpu);
            return n;
        };
        int zc = 0;   // the longest column (a power of two <= 32) that leaves >= 32 columns a SM
        for (int t = 32; t >= 1 && !zc; t >>= 1)
            if (gz % t == 0 && columns(t) >= 32LL * c->sm_count) zc = t;
        if (c->oz_opt == 3 && !zc)
            for (int t = 32; t >= 1 && !zc; t >>= 1)
                if (gz % t == 0) zc = t;
        // the caller's choice, else the tuner's (large planes), else the rule
        const int ozo = c->oz_opt != 0 ? c->oz_opt : large ? c->tuned_oz : 0;
        c->tma_form = ozo == 1 ? 0 : ozo == 2 ? 1 : ozo == 3 ? 2 : !large ? 0 : zc >= 8 ? 2 : 1;
        if (c->tma_form == 2 && c->zc_opt) {   // a column length set by the caller
            if (gz % c->zc_opt != 0)
                return fail(c, LBMBT_EINVAL, "column of %d planes does not divide every member's nz", c->zc_opt);
            zc = c->zc_opt;
        }
        c->tma_zc = c->tma_form == 2 ? zc : 0;
        c->n_cc = 0;
        c->cc_start.assign(c->n_members + 1, 0);
        if (c->tma_form == 2)
            for (int m = 0; m < c->n_members; ++m) {
                MemberDesc& d = c->descs[m];
                d.cc0 = c->cc_start[m];
                c->cc_start[m + 1] = d.cc0 + (long long)(d.nz / zc) * ((d.ny + d.rpu - 1) / d.rpu);
            }
        c->n_cc = c->cc_start[c->n_members];
        int per_sm = 0;
        const cudaError_t pe = tma_prepare(c->tma_cap, c->tma_capx, c->tma_stages, c->tma_variant, c->tma_form,
                                           &per_sm);
        if (pe == cudaErrorInvalidValue) {   // more shared memory than a block may have
            cudaGetLastError();
            return fail(c, LBMBT_EINVAL, "%d bulk-copy stages of %d sites (%zu bytes) do not fit in shared memory",
                        c->tma_stages, c->tma_cap,
                        tma_smem_bytes(c->tma_cap, c->tma_capx, c->tma_stages, c->tma_form));
        }
        CU(c, pe);
        if (per_sm < 1) return fail(c, LBMBT_EINVAL, "bulk-copy sweep does not fit on an SM");
        c->tma_grid = (int)std::min<long long>((long long)c->sm_count * per_sm,
                                               c->tma_form == 2 ? c->n_cc : c->n_units);
    }
    for (auto& d : c->descs)
        if (d.dlt) {
            CU(c, links_prepare());
            break;
        }
    const long long n_part = std::max(c->n_tiles, c->n_units * tma_partials_per_unit(c->tma_variant));
    int rc = grow(c, &c->d_desc, &c->cap_desc, sizeof(MemberDesc) * c->n_members);
    if (!rc) rc = grow(c, &c->d_tile_start, &c->cap_ts, sizeof(long long) * (c->n_members + 1));
    if (!rc) rc = grow(c, &c->d_unit_start, &c->cap_us, sizeof(long long) * (c->n_members + 1));
    if (!rc) rc = grow(c, &c->d_adj_unit_start, &c->cap_aus, sizeof(long long) * (c->n_members + 1));
    if (!rc) rc = grow(c, &c->d_partial, &c->cap_partial, sizeof(double2) * n_part);
    if (!rc) rc = grow(c, &c->d_cc_start, &c->cap_cc, sizeof(long long) * (c->n_members + 1));
    if (rc) return rc;
    CU(c, cudaMemcpyAsync(c->d_desc, c->descs.data(), sizeof(MemberDesc) * c->n_members, cudaMemcpyHostToDevice,
                          c->stream));
    if (!c->ftab_valid) {
        // FP64 boundary factors of every step for every member, once per run
        // (the sweeps and the adjoint read them by step index)
        const size_t tb = sizeof(float2) * 6 * (size_t)(c->n_steps + 1) * c->n_members;
        if (tb > (4ull << 30))
            return fail(c, LBMBT_ENOMEM, "boundary-factor table of %zu bytes (steps x members too large; split the "
                                         "batch)", tb);
        rc = grow(c, &c->d_ftab, &c->cap_ftab, tb);
        if (rc) return rc;
        CU(c, launch_factor_table(c->d_desc, c->n_members, ctl_F_shift(c), c->n_steps, c->d_ftab, c->stream));
        c->launches++;
        c->ftab_valid = true;
    }
    CU(c, cudaMemcpyAsync(c->d_tile_start, c->tile_start.data(), sizeof(long long) * (c->n_members + 1),
                          cudaMemcpyHostToDevice, c->stream));
    CU(c, cudaMemcpyAsync(c->d_unit_start, c->unit_start.data(), sizeof(long long) * (c->n_members + 1),
                          cudaMemcpyHostToDevice, c->stream));
    CU(c, cudaMemcpyAsync(c->d_adj_unit_start, c->adj_unit_start.data(), sizeof(long long) * (c->n_members + 1),
                          cudaMemcpyHostToDevice, c->stream));
    if (c->use_tma && c->tma_form == 2)
        CU(c, cudaMemcpyAsync(c->d_cc_start, c->cc_start.data(), sizeof(long long) * (c->n_members + 1),
                              cudaMemcpyHostToDevice, c->stream));
    c->tile_block = block;
    c->tile_spt = spt;
    drop_graph(c);
    return sync(c);
}

// Work list the signal partials of the current sweep kernel are indexed by.
static const long long* part_start(const lbmbt_ctx* c) { return c->use_tma ? c->d_unit_start : c->d_tile_start; }
static int part_per(const lbmbt_ctx* c) { return c->use_tma ? tma_partials_per_unit(c->tma_variant) : 1; }

static SweepArgs sweep_args(lbmbt_ctx* c)
{
    SweepArgs a;
    a.members = c->d_desc;
    a.tile_start = c->d_tile_start;
    a.n_members = c->n_members;
    a.ctl = c->d_ctl;
    a.f = c->d_f;
    a.F = c->d_F;
    a.scheme = c->scheme;
    a.test_wait_ns = (unsigned long long)c->test_wait_ns;
    a.partial = c->d_partial;
    a.fac = c->d_ftab;
    const bool zm = c->use_tma && c->tma_form == 2;
    a.zc = zm ? c->tma_zc : 0;
    a.zc_log2 = 0;
    while (a.zc > (1 << a.zc_log2)) ++a.zc_log2;
    a.n_cc = zm ? c->n_cc : 0;
    a.cc_start = zm ? c->d_cc_start : nullptr;
    a.links = 0;
    for (auto& d : c->descs) {
        if (d.dth) a.links = 2;
        else if (d.dlt && a.links == 0) a.links = 1;
    }
    if (c->lattice == 1) {
        // D2Q5 weights 1/3, 1/6 are not binary fractions: take w0 = 1 - 4 wxy
        // (exact in FP32) so the FP32 weights sum to exactly 1; with
        // fl(1/3) + 4 fl(1/6) = 1 + 3e-8 every collision would scale M by
        // 1 + omega 3e-8 (0.5 % over 1.5e5 steps)
        a.wxy = 1.f / 6.f;
        a.w0 = 1.f - 4.f * a.wxy;
        a.wz = 0.f;
    }
    else { a.w0 = W0; a.wxy = WI; a.wz = WI; }
    return a;
}


static int write_ctl(lbmbt_ctx* c, int sig_step, int field_step, int slot_base = 0, int slot_mod = 2)
{
    StepCtl h;
    memset(&h, 0, sizeof h);   // counters start at zero
    h.k = (int)c->k_cur;
    h.done = 0;
    h.sig_step = sig_step;
    h.field_step = field_step;
    h.slot_base = slot_base;
    h.slot_mod = slot_mod;
    h.series = c->series_mode ? 1 : 0;
    h.err = 0;
    CU(c, launch_ctl_set(c->d_ctl, h, c->stream));
    c->launches++;
    return LBMBT_OK;
}

static int init_state(lbmbt_ctx* c)
{
    SweepArgs a = sweep_args(c);
    CU(c, launch_init(a, c->n_tiles, c->tile_block, c->tile_spt, 0, c->stream));
    c->launches++;
    c->k_cur = 0;
    return LBMBT_OK;
}

// Issue one step: the sweep (its last block advances the step word), plus
// the per-step reduce in series mode.
static int issue_step(lbmbt_ctx* c)
{
    SweepArgs a = sweep_args(c);
    if (c->use_tma) {
        a.tile_start = c->d_unit_start;
        CU(c, launch_sweep_tma(a, c->n_units, c->tma_cap, c->tma_capx, c->tma_stages, c->tma_variant, c->tma_form,
                               c->tma_grid, c->stream));
    } else {
        CU(c, launch_sweep(a, c->n_tiles, c->tile_block, c->tile_spt, c->stream));
    }
    c->launches += c->use_tma ? 1 : 2;   // the register sweep is followed by the step advance
    if (c->series_mode) {
        CU(c, launch_reduce(c->d_partial, part_start(c), part_per(c), c->n_members, c->d_Z, c->d_series, c->n_steps, c->d_ctl,
                            c->stream));
        c->launches++;
    }
    return LBMBT_OK;
}

// Times a few steps of every launch shape that fits -- register sweep block x
// sites per thread, bulk-copy sweep consumer shape x stages -- and keeps the
// fastest for this problem shape (cached per shape for the context's life).
static int autotune(lbmbt_ctx* c)
{
    std::string key = std::to_string(c->n_members);
    for (auto& d : c->descs) key += "/" + std::to_string(d.nx) + "x" + std::to_string(d.ny) + "x" + std::to_string(d.nz);
    auto it = c->tune_cache.find(key);
    if (it == c->tune_cache.end()) {
        struct Cand { int kernel, block, spt, variant, stages, oz; };
        std::vector<Cand> cand;
        if (c->kernel_opt != 2)
            for (auto bs : {std::make_pair(128, 1), std::make_pair(256, 1), std::make_pair(512, 1),
                            std::make_pair(128, 2), std::make_pair(256, 2), std::make_pair(512, 2),
                            std::make_pair(128, 4), std::make_pair(256, 4)})
                cand.push_back({1, bs.first, bs.second, c->tma_variant, c->tma_stages, c->oz_opt});
        // on large planes with membranes the staging and the z-marching forms
        // are both timed (which is faster varies from GPU to GPU by a few %)
        bool large = false;
        for (auto& d : c->descs)
            if (d.memb && (long long)d.nx * d.ny >= TMA_OZ_PLANE) large = true;
        std::vector<int> forms;
        if (c->oz_opt == 0 && large) forms = {2, 3};
        else forms = {c->oz_opt};
        if (c->kernel_opt != 1 && tma_eligible(c))
            for (int oz : forms)
                for (int v = 0; v < 4; ++v)
                    for (int st = 2; st <= 4; ++st) cand.push_back({2, c->block, c->spt, v, st, oz});
        const int saved_opt = c->kernel_opt, saved_block = c->block, saved_spt = c->spt;
        const int saved_var = c->tma_variant, saved_st = c->tma_stages, saved_oz = c->oz_opt;
        const bool saved_series = c->series_mode;
        c->series_mode = false;
        cudaEvent_t e0, e1;
        CU(c, cudaEventCreate(&e0));
        CU(c, cudaEventCreate(&e1));
        float best = 1e30f;
        Cand win = {0, saved_block, saved_spt, saved_var, saved_st, 0};
        for (const Cand& cd : cand) {
            c->kernel_opt = cd.kernel;
            c->tma_variant = cd.variant;
            c->tma_stages = cd.stages;
            c->oz_opt = cd.oz;
            if (build_worklist(c, cd.block, cd.spt) != LBMBT_OK) {  // e.g. stages do not fit
                c->err.clear();
                cudaGetLastError();
                continue;
            }
            // one warm step, then batches of steps from k = 0 (never past
            // the end of the schedule), growing until a batch takes 1 ms
            int rc = init_state(c);
            if (!rc) rc = write_ctl(c, -1, -1);
            if (!rc) rc = issue_step(c);
            if (rc) break;
            const long long r_max = std::min<long long>(c->n_steps, 256);
            long long r = std::min<long long>(4, r_max);
            float per_step = 0.f;
            for (;;) {
                rc = write_ctl(c, -1, -1);
                CU(c, cudaEventRecord(e0, c->stream));
                for (long long q = 0; q < r && !rc; ++q) rc = issue_step(c);
                CU(c, cudaEventRecord(e1, c->stream));
                CU(c, cudaEventSynchronize(e1));
                float ms = 0;
                CU(c, cudaEventElapsedTime(&ms, e0, e1));
                per_step = ms / (float)r;
                if (rc || ms >= 1.f || r >= r_max) break;
                r = std::min<long long>(r * 4, r_max);
            }
            if (!rc && per_step < best) { best = per_step; win = cd; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->kernel_opt = saved_opt;
        c->block = saved_block;
        c->spt = saved_spt;
        c->tma_variant = saved_var;
        c->tma_stages = saved_st;
        c->oz_opt = saved_oz;
        c->series_mode = saved_series;
        it = c->tune_cache.emplace(key, lbmbt_ctx::Tuned{win.kernel, win.block, win.spt, win.variant, win.stages,
                                                         win.kernel == 2 ? win.oz : 0}).first;
    }
    const lbmbt_ctx::Tuned& t = it->second;
    c->tuned_kernel = t.kernel;
    c->tuned_oz = t.oz;
    c->block = t.block;
    c->spt = t.spt;
    c->tma_variant = t.variant;
    c->tma_stages = t.stages;
    return LBMBT_OK;
}

static bool any_slab(const lbmbt_ctx* c);

// ex (optional, [n_members]): each member's own waveform (f, n_steps; f NULL
// for the run's) and field output.
static int prepare(lbmbt_ctx* c, int n_members, const lbmbt_member* mem, bool series, void* field_dev,
                   const lbmbt_member_ex* ex = nullptr)
{
    if (c->geoms.empty()) return fail(c, LBMBT_ESTATE, "no geometry set");
    if (c->n_phases == 0) return fail(c, LBMBT_ESTATE, "phases not set");
    if (c->n_steps == 0) return fail(c, LBMBT_ESTATE, "sequence not set");
    if (n_members < 1) return fail(c, LBMBT_EINVAL, "n_members must be >= 1");
    if (field_dev && n_members != 1) return fail(c, LBMBT_EINVAL, "field output needs a single member");
    if (c->scheme == 1) {
        if (any_slab(c)) return fail(c, LBMBT_EUNSUPPORTED, "the classical scheme does not run on slabs");
        if (c->substeps != 1)
            return fail(c, LBMBT_EINVAL, "the classical scheme has no reaction step to sub-step");
    }
    int rc = set_device(c);
    if (rc) return rc;
    std::vector<MemberDesc> descs(n_members);
    size_t max_plane = 0;
    for (int m = 0; m < n_members; ++m) {
        const lbmbt_member& mm = mem[m];
        if (mm.geometry < 0 || mm.geometry >= (int)c->geoms.size())
            return fail(c, LBMBT_EINVAL, "member %d: geometry %d not set", m, mm.geometry);
        const Geom& g = c->geoms[mm.geometry];
        if (g.max_phase >= c->n_phases)
            return fail(c, LBMBT_ESTATE, "geometry %d uses phase %d but %d phases are set", mm.geometry, g.max_phase,
                        c->n_phases);
        if (!(mm.kappa_um_ms >= 0)) return fail(c, LBMBT_EINVAL, "member %d: kappa must be >= 0", m);
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(mm.gamma_G0[a])) return fail(c, LBMBT_EINVAL, "member %d: gradient not finite", m);
        MemberDesc& d = descs[m];
        memset(&d, 0, sizeof d);
        d.mask = g.d_mask;
        d.N = g.N;
        d.plane = (g.N + 63) / 64 * 64;
        d.nx = g.nx; d.ny = g.ny; d.nz = g.nz;
        d.z0 = g.slab ? g.z0 : 0;
        d.nzg = g.slab ? g.nzg : g.nz;
        d.dx = g.dx;
        for (int a = 0; a < 3; ++a) {
            d.gG[a] = mm.gamma_G0[a];
            d.ctheta[a] = (float)(-mm.gamma_G0[a] * g.dx * c->dt);
            if (g.bc[a] == LBMBT_BC_PERIODIC) d.bc[a] = BC_PER;
            else if (mm.gamma_G0[a] == 0.0) d.bc[a] = BC_MIR;
            else {
                for (int b = 0; b < 3; ++b)
                    if (b != a && mm.gamma_G0[b] != 0.0)
                        return fail(c, LBMBT_EUNSUPPORTED,
                                    "member %d: mirror face on axis %d with a gradient neither normal nor parallel "
                                    "to it (Sec. 2.4.4)", m, a);
                d.bc[a] = BC_MIR_CONJ;
            }
        }
        for (int h = 0; h < 2; ++h)
            d.zbc[h] = (!g.slab || g.zkind[h] == LBMBT_FACE_OWN) ? d.bc[2]
                       : g.zkind[h] == LBMBT_FACE_HALO          ? BC_HALO
                                                                : BC_HALO_PER;
        const double eps = c->lattice == 1 ? EPS_D2 : EPS_D;
        if (c->lattice == 1 && (g.nz != 1 || g.slab))
            return fail(c, LBMBT_EINVAL, "the D2Q5 lattice needs geometries of one z plane (geometry %d has %d)",
                        mm.geometry, g.nz);
        for (int p = 0; p < 4; ++p) {
            const double tau = 0.5 + c->dt * c->D[p] / (eps * g.dx * g.dx);   // Eq. tau_def
            if (p < c->n_phases && !(tau > 0.5))
                return fail(c, LBMBT_EUNSTABLE, "phase %d: tau = %.17g <= 1/2", p, tau);
            d.omega[p] = (float)(1.0 / tau);
            if (c->scheme == 1)   // the classical source's decay rate: dt/T2 (Eq. A12)
                d.eps[p] = std::isinf(c->T2[p]) ? 0.f : (float)(c->dt / c->T2[p]);
            else
                d.eps[p] = std::isinf(c->T2[p]) ? 0.f : (float)(-std::expm1(-c->dt / c->T2[p]));
        }
        const double kap = mm.kappa_um_ms;
        const double cP = eps * g.dx / (2.0 * c->dt);   // P = cP / kappa  (Eq. P_def)
        d.s_share = std::isinf(kap) ? 1.f : (float)(kap / (kap + cP));
        d.axes = 0;
        for (int a = 0; a < 3; ++a)
            if (d.ctheta[a] != 0.f) d.axes |= 1 << a;
        d.memb = g.has_membranes;
        if (g.d_dlt && !std::isinf(kap)) {
            if (g.slab) return fail(c, LBMBT_EUNSUPPORTED, "membrane positions on a slab are not supported");
            if (c->scheme == 1)
                return fail(c, LBMBT_EUNSUPPORTED, "the classical scheme takes the half-link membrane rule only");
            d.dlt = g.d_dlt;
            d.lrho = (float)(kap * c->dt / (eps * g.dx));
            if (g.d_dth) {
                if (c->lattice != 1)
                    return fail(c, LBMBT_EUNSUPPORTED, "membrane angles need the D2Q5 lattice (LBMBT_OPT_LATTICE 1)");
                // the general-angle rule's extrapolation is unstable for tau
                // near 1/2 (measured: diverging at tau 0.65, and at 0.7 with
                // grazing links of high permeability)
                for (int p = 0; p < c->n_phases; ++p) {
                    const double tau = 0.5 + c->dt * c->D[p] / (eps * g.dx * g.dx);
                    if (!(tau >= ANGLE_TAU_MIN))
                        return fail(c, LBMBT_EUNSTABLE, "membrane angles need tau >= %.2f in every phase (phase %d: %.4g)",
                                    ANGLE_TAU_MIN, p, tau);
                }
                d.dth = g.d_dth;
            }
        }
        div_magic((unsigned)g.nx, &d.div_m[0], &d.div_s[0]);
        div_magic((unsigned)g.ny, &d.div_m[1], &d.div_s[1]);
        if ((size_t)d.plane > max_plane) max_plane = d.plane;
        d.fw = c->d_f;
        d.Fw = c->d_F;
        d.end_step = -1;
        if (ex) {
            if (ex[m].f && (ex[m].n_steps < 1 || ex[m].n_steps > c->n_steps))
                return fail(c, LBMBT_EINVAL, "member %d: waveform of %lld steps, the run has %lld", m,
                            (long long)ex[m].n_steps, c->n_steps);
            if (ex[m].f)
                for (long long k = 0; k < ex[m].n_steps; ++k)
                    if (!std::isfinite(ex[m].f[k])) return fail(c, LBMBT_EINVAL, "member %d: f[%lld] not finite", m, k);
            d.end_step = (int)((ex[m].f ? ex[m].n_steps : c->n_steps) - 1);
        }
    }
    invalidate_run(c);
    c->n_members = n_members;
    c->members.assign(mem, mem + n_members);
    c->descs = descs;
    c->series_mode = series;
    c->n_slots = 2;
    // state: n_slots * 7 planes per member
    size_t total = 0;
    for (auto& d : c->descs) total += (size_t)c->n_slots * 7 * d.plane * sizeof(float2);
    rc = grow(c, &c->d_state, &c->cap_state, total);
    if (rc) return rc;
    size_t off = 0;
    for (auto& d : c->descs) {
        d.state = c->d_state + off / sizeof(float2);
        off += (size_t)c->n_slots * 7 * d.plane * sizeof(float2);
    }
    if (field_dev) c->descs[0].field = (float2*)field_dev;
    if (ex) {
        // members' own waveforms: f_k (zero past the member's end, one entry
        // past the run's) and F_k = sum_{m<k} f_m dt, as lbmbt_set_sequence
        // builds the shared ones
        const long long K = c->n_steps;
        int n_own = 0;
        for (int m = 0; m < n_members; ++m) n_own += ex[m].f != nullptr;
        if (n_own) {
            rc = grow(c, &c->d_wf, &c->cap_wf, sizeof(float) * (size_t)n_own * (K + 1));
            if (!rc) rc = grow(c, &c->d_wF, &c->cap_wF, sizeof(double) * (size_t)n_own * (K + 2));
            if (rc) return rc;
            std::vector<float> wf((size_t)n_own * (K + 1), 0.f);
            std::vector<double> wF((size_t)n_own * (K + 2));
            int j = 0;
            for (int m = 0; m < n_members; ++m) {
                if (!ex[m].f) continue;
                float* fj = wf.data() + (size_t)j * (K + 1);
                double* Fj = wF.data() + (size_t)j * (K + 2);
                double F = 0.0;
                for (long long k = 0; k < K; ++k) {
                    const double fk = k < ex[m].n_steps ? ex[m].f[k] : 0.0;
                    fj[k] = (float)fk;
                    Fj[k] = F;
                    F += fk * c->dt;
                }
                Fj[K] = F;
                Fj[K + 1] = F;
                c->descs[m].fw = c->d_wf + (size_t)j * (K + 1);
                c->descs[m].Fw = c->d_wF + (size_t)j * (K + 2);
                ++j;
            }
            CU(c, cudaMemcpyAsync(c->d_wf, wf.data(), sizeof(float) * wf.size(), cudaMemcpyHostToDevice, c->stream));
            CU(c, cudaMemcpyAsync(c->d_wF, wF.data(), sizeof(double) * wF.size(), cudaMemcpyHostToDevice, c->stream));
            CU(c, cudaStreamSynchronize(c->stream));
        }
        for (int m = 0; m < n_members; ++m) c->descs[m].field = static_cast<float2*>(ex[m].field_dev);
    }
    {   // slab halo planes: two of nx*ny complex values per slab member
        c->halo_off.assign(n_members, 0);
        size_t hn = 0;
        for (int m = 0; m < n_members; ++m)
            if (c->geoms[mem[m].geometry].slab) {
                c->halo_off[m] = hn;
                hn += 2 * (size_t)c->descs[m].nx * c->descs[m].ny;   // nx even: planes stay 16-byte aligned
            }
        if (hn) {
            rc = grow(c, &c->d_halo, &c->cap_halo, hn * sizeof(float2));
            if (rc) return rc;
            for (int m = 0; m < n_members; ++m)
                if (c->geoms[mem[m].geometry].slab) {
                    const size_t sxy = (size_t)c->descs[m].nx * c->descs[m].ny;
                    c->descs[m].halo[0] = c->d_halo + c->halo_off[m];
                    c->descs[m].halo[1] = c->d_halo + c->halo_off[m] + sxy;
                }
        }
    }
    {   // rotation tables
        std::vector<float2> et;
        std::vector<size_t> off(n_members);
        for (int m = 0; m < n_members; ++m) {
            off[m] = et.size();
            const MemberDesc& d = c->descs[m];
            const int dims[3] = {d.nx, d.ny, d.nz};
            rotation_table(d.gG, d.dx, c->dt, dims, d.z0, et);
            if (et.size() & 1) et.push_back(make_float2(0.f, 0.f));  // 16-byte aligned tables
        }
        rc = grow(c, &c->d_etab, &c->cap_etab, et.size() * sizeof(float2));
        if (rc) return rc;
        CU(c, cudaMemcpyAsync(c->d_etab, et.data(), et.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream));
        for (int m = 0; m < n_members; ++m) c->descs[m].etab = c->d_etab + off[m];
        CU(c, cudaStreamSynchronize(c->stream));
    }
    rc = grow(c, &c->d_Z, &c->cap_Z, sizeof(double2) * n_members);
    if (!rc && series) rc = grow(c, &c->d_series, &c->cap_series, sizeof(double2) * n_members * c->n_steps);
    if (rc) return rc;
    if (c->autotune) {
        rc = autotune(c);
        if (rc) return rc;
    }
    rc = build_worklist(c, c->block, c->spt);
    if (rc) return rc;
    rc = init_state(c);
    if (rc) return rc;
    c->field_dev = field_dev;
    c->prepared = true;
    return LBMBT_OK;
}

static int capture_graph(lbmbt_ctx* c)
{
    drop_graph(c);
    cudaGraph_t g;
    CU(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const long long before = c->launches;
    for (int i = 0; i < GRAPH_CHUNK; ++i) {
        int rc = issue_step(c);
        if (rc) {
            cudaStreamEndCapture(c->stream, &g);
            return rc;
        }
    }
    c->launches = before;  // counted when replayed
    CU(c, cudaStreamEndCapture(c->stream, &g));
    cudaError_t e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { c->graph = nullptr; return fail(c, LBMBT_ECUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
    c->graph_series = c->series_mode ? 1 : 0;
    return LBMBT_OK;
}

static bool any_slab(const lbmbt_ctx* c)
{
    for (auto& g : c->geoms)
        if (g.slab) return true;
    return false;
}

// Advance n steps; the signal (and field) of the last step is produced when asked.
static int advance(lbmbt_ctx* c, long long n, bool want_signal)
{
    if (!c->prepared) return fail(c, LBMBT_ESTATE, "no prepared run");
    if (n < 0 || c->k_cur + n > c->n_steps)
        return fail(c, LBMBT_EINVAL, "advance past the end of the sequence (%lld + %lld > %lld)", c->k_cur, n,
                    c->n_steps);
    if (n == 0) return LBMBT_OK;
    if (n > 1 && any_slab(c))
        return fail(c, LBMBT_EINVAL, "a slab advances one step at a time, with a halo exchange between steps");
    const long long last = c->k_cur + n - 1;
    int rc = write_ctl(c, want_signal ? (int)last : -1, (c->field_dev && last == c->n_steps - 1) ? (int)last : -1);
    if (rc) return rc;
    long long left = n;
    if (c->use_graph && n >= GRAPH_CHUNK) {
        if (!c->graph || c->graph_series != (c->series_mode ? 1 : 0)) {
            rc = capture_graph(c);
            if (rc) return rc;
        }
        const int per = (c->use_tma ? 1 : 2) + (c->series_mode ? 1 : 0);
        while (left >= GRAPH_CHUNK) {
            CU(c, cudaGraphLaunch(c->graph, c->stream));
            c->launches += GRAPH_CHUNK * per;
            left -= GRAPH_CHUNK;
        }
    }
    while (left > 0) {
        rc = issue_step(c);
        if (rc) return rc;
        --left;
    }
    c->k_cur += n;
    if (want_signal && !c->series_mode) {
        CU(c, launch_reduce(c->d_partial, part_start(c), part_per(c), c->n_members, c->d_Z, nullptr, 0, c->d_ctl, c->stream));
        c->launches++;
    }
    return LBMBT_OK;
}

// Device-side error word of the step control (a bounded wait that timed out).
static int check_device_error(lbmbt_ctx* c)
{
    int err = 0;
    CU(c, cudaMemcpyAsync(&err, &c->d_ctl->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(c, cudaStreamSynchronize(c->stream));
    if (err) return fail(c, LBMBT_EDEVICE, "a device-side wait timed out (error word %d)", err);
    return LBMBT_OK;
}

static int fetch_signal(lbmbt_ctx* c, double* signal_out, double* series_out)
{
    int rc0 = check_device_error(c);
    if (rc0) return rc0;
    std::vector<double2> Z(c->n_members);
    CU(c, cudaMemcpyAsync(Z.data(), c->d_Z, sizeof(double2) * c->n_members, cudaMemcpyDeviceToHost, c->stream));
    std::vector<double2> ser;
    if (series_out && c->series_mode) {
        ser.resize((size_t)c->n_members * c->n_steps);
        CU(c, cudaMemcpyAsync(ser.data(), c->d_series, sizeof(double2) * ser.size(), cudaMemcpyDeviceToHost,
                              c->stream));
    }
    int rc = sync(c);
    if (rc) return rc;
    for (int m = 0; m < c->n_members; ++m) {
        const double N = (double)c->descs[m].N;
        if (signal_out) {
            signal_out[3 * m] = Z[m].x;
            signal_out[3 * m + 1] = Z[m].y;
            signal_out[3 * m + 2] = std::hypot(Z[m].x, Z[m].y) / N;
        }
    }
    if (series_out && c->series_mode)
        for (size_t i = 0; i < ser.size(); ++i) { series_out[2 * i] = ser[i].x; series_out[2 * i + 1] = ser[i].y; }
    // series mode reduces every step, so the last reduction is of the last
    // step: a member that ends earlier takes its signal from its own step
    if (signal_out && c->series_mode && !ser.empty())
        for (int m = 0; m < c->n_members; ++m) {
            const int es = c->descs[m].end_step;
            if (es < 0 || es == c->n_steps - 1) continue;
            const double2 z = ser[(size_t)m * c->n_steps + es];
            signal_out[3 * m] = z.x;
            signal_out[3 * m + 1] = z.y;
            signal_out[3 * m + 2] = std::hypot(z.x, z.y) / (double)c->descs[m].N;
        }
    return LBMBT_OK;
}

// ---------------------------------------------------------------- runs
static lbmbt_member plain_member(lbmbt_ctx* c)
{
    lbmbt_member m;
    for (int a = 0; a < 3; ++a) m.gamma_G0[a] = c->gG[a];
    m.geometry = 0;
    m.kappa_um_ms = c->kappa;
    return m;
}

extern "C" int lbmbt_run(lbmbt_ctx* c, double* signal_out, void* field_out_dev, double* series_out)
{
    if (!c) return LBMBT_EINVAL;
    if (!signal_out) return fail(c, LBMBT_EINVAL, "signal_out is NULL");
    if (any_slab(c)) return fail(c, LBMBT_ESTATE, "a slab runs with lbmbt_prepare and lbmbt_advance(1) per step");
    lbmbt_member m = plain_member(c);
    int rc = prepare(c, 1, &m, series_out != nullptr, field_out_dev);
    if (!rc) rc = advance(c, c->n_steps, true);
    if (!rc) rc = fetch_signal(c, signal_out, series_out);
    return rc;
}

extern "C" int lbmbt_run_batch(lbmbt_ctx* c, int n_members, const lbmbt_member* members, double* signal_out,
                               double* series_out)
{
    if (!c) return LBMBT_EINVAL;
    if (!members || !signal_out) return fail(c, LBMBT_EINVAL, "members / signal_out is NULL");
    if (any_slab(c)) return fail(c, LBMBT_ESTATE, "a slab runs with lbmbt_prepare and lbmbt_advance(1) per step");
    int rc = prepare(c, n_members, members, series_out != nullptr, nullptr);
    if (!rc) rc = advance(c, c->n_steps, true);
    if (!rc) rc = fetch_signal(c, signal_out, series_out);
    return rc;
}

extern "C" int lbmbt_run_batch_ex(lbmbt_ctx* c, int n_members, const lbmbt_member_ex* members, double* signal_out,
                                  double* series_out)
{
    if (!c) return LBMBT_EINVAL;
    if (!members || !signal_out) return fail(c, LBMBT_EINVAL, "members / signal_out is NULL");
    if (any_slab(c)) return fail(c, LBMBT_ESTATE, "a slab runs with lbmbt_prepare and lbmbt_advance(1) per step");
    if (n_members < 1) return fail(c, LBMBT_EINVAL, "n_members must be >= 1");
    std::vector<lbmbt_member> base(n_members);
    for (int m = 0; m < n_members; ++m) {
        for (int a = 0; a < 3; ++a) base[m].gamma_G0[a] = members[m].gamma_G0[a];
        base[m].geometry = members[m].geometry;
        base[m].kappa_um_ms = members[m].kappa_um_ms;
    }
    int rc = prepare(c, n_members, base.data(), series_out != nullptr, nullptr, members);
    if (!rc) rc = advance(c, c->n_steps, true);
    if (!rc) rc = fetch_signal(c, signal_out, series_out);
    // the run stands at its end: no later step writes the members' fields
    return rc;
}

extern "C" int lbmbt_prepare(lbmbt_ctx* c, int n_members, const lbmbt_member* members)
{
    if (!c) return LBMBT_EINVAL;
    if (n_members == 0) {
        lbmbt_member m = plain_member(c);
        int rc = prepare(c, 1, &m, false, c->field_req);
        return rc ? rc : sync(c);
    }
    if (!members) return fail(c, LBMBT_EINVAL, "members is NULL");
    int rc = prepare(c, n_members, members, false, c->field_req);
    return rc ? rc : sync(c);
}

extern "C" int lbmbt_set_field(lbmbt_ctx* c, void* field_dev)
{
    if (!c) return LBMBT_EINVAL;
    c->field_req = field_dev;
    return LBMBT_OK;
}

extern "C" int lbmbt_advance(lbmbt_ctx* c, int64_t n_steps, int want_signal, double* signal_out)
{
    if (!c) return LBMBT_EINVAL;
    int rc = advance(c, n_steps, want_signal != 0);
    if (rc) return rc;
    if (want_signal && signal_out) return fetch_signal(c, signal_out, nullptr);
    return check_device_error(c);
}

// Slab faces of member m at the current step (before the next sweep): the
// population leaving through each z face, hat g_6 of plane 0 (for the slab
// below) and hat g_5 of plane nz-1 (for the slab above).
extern "C" int lbmbt_slab_faces(lbmbt_ctx* c, int member, void* lo_out, void* hi_out)
{
    if (!c) return LBMBT_EINVAL;
    if (!c->prepared) return fail(c, LBMBT_ESTATE, "no prepared run");
    if (member < 0 || member >= c->n_members) return fail(c, LBMBT_EINVAL, "member %d out of range", member);
    const MemberDesc& d = c->descs[member];
    if (!d.halo[0]) return fail(c, LBMBT_ESTATE, "member %d is not on a slab", member);
    int rc = set_device(c);
    if (rc) return rc;
    const size_t sxy = (size_t)d.nx * d.ny, P = (size_t)d.plane;
    const float2* lvl = d.state + (size_t)(c->k_cur % 2) * 7 * P;
    if (lo_out) CU(c, cudaMemcpyAsync(lo_out, lvl + 6 * P, sxy * sizeof(float2), cudaMemcpyDefault, c->stream));
    if (hi_out)
        CU(c, cudaMemcpyAsync(hi_out, lvl + 5 * P + (size_t)(d.nz - 1) * sxy, sxy * sizeof(float2), cudaMemcpyDefault,
                              c->stream));
    return LBMBT_OK;
}

// Halo planes of member m for the next sweep: lo_in = hat g_5 of the plane
// below the slab, hi_in = hat g_6 of the plane above (the neighbours' faces).
extern "C" int lbmbt_slab_set_halos(lbmbt_ctx* c, int member, const void* lo_in, const void* hi_in)
{
    if (!c) return LBMBT_EINVAL;
    if (!c->prepared) return fail(c, LBMBT_ESTATE, "no prepared run");
    if (member < 0 || member >= c->n_members) return fail(c, LBMBT_EINVAL, "member %d out of range", member);
    const MemberDesc& d = c->descs[member];
    if (!d.halo[0]) return fail(c, LBMBT_ESTATE, "member %d is not on a slab", member);
    int rc = set_device(c);
    if (rc) return rc;
    const size_t sxy = (size_t)d.nx * d.ny;
    if (lo_in)
        CU(c, cudaMemcpyAsync(const_cast<float2*>(d.halo[0]), lo_in, sxy * sizeof(float2), cudaMemcpyDefault, c->stream));
    if (hi_in)
        CU(c, cudaMemcpyAsync(const_cast<float2*>(d.halo[1]), hi_in, sxy * sizeof(float2), cudaMemcpyDefault, c->stream));
    return LBMBT_OK;
}

extern "C" int lbmbt_set_option(lbmbt_ctx* c, int opt, int64_t v)
{
    if (!c) return LBMBT_EINVAL;
    switch (opt) {
    case LBMBT_OPT_GRAPH: c->use_graph = v != 0; break;
    case LBMBT_OPT_AUTOTUNE:
        c->autotune = v != 0;
        if (!c->autotune) c->tuned_kernel = c->tuned_oz = 0;
        break;
    case LBMBT_OPT_BLOCK:
        if (v < 64 || v > 512 || (v & 31)) return fail(c, LBMBT_EINVAL, "block must be a multiple of 32 in 64..512");
        c->block = (int)v;
        break;
    case LBMBT_OPT_SPT:
        if (v != 1 && v != 2 && v != 4) return fail(c, LBMBT_EINVAL, "sites per thread must be 1, 2 or 4");
        c->spt = (int)v;
        break;
    case LBMBT_OPT_KERNEL:
        if (v < 0 || v > 2) return fail(c, LBMBT_EINVAL, "kernel must be 0 (auto), 1 (register) or 2 (bulk copy)");
        c->kernel_opt = (int)v;
        break;
    case LBMBT_OPT_STAGES:
        if (v < 2 || v > 6) return fail(c, LBMBT_EINVAL, "stages must be 2..6");
        c->tma_stages = (int)v;
        break;
    case LBMBT_OPT_TMA_SHAPE:
        if (v < 0 || v > 3) return fail(c, LBMBT_EINVAL, "bulk-copy shape must be 0, 1, 2 or 3");
        c->tma_variant = (int)v;
        break;
    case LBMBT_OPT_ADJOINT_KERNEL:
        if (v < 0 || v > 2) return fail(c, LBMBT_EINVAL, "adjoint kernel must be 0 (auto), 1 or 2");
        c->adjoint_opt = (int)v;
        break;
    case LBMBT_OPT_ADJOINT_SHAPE:
        if (v < 0 || v > 2) return fail(c, LBMBT_EINVAL, "adjoint shape must be 0, 1 or 2");
        c->adj_shape = (int)v;
        break;
    case LBMBT_OPT_LATTICE:
        if (v != 0 && v != 1) return fail(c, LBMBT_EINVAL, "lattice must be 0 (D3Q7) or 1 (D2Q5)");
        invalidate_run(c);
        c->lattice = (int)v;
        break;
    case LBMBT_OPT_STAGE_OWN_Z:
        if (v < 0 || v > 3) return fail(c, LBMBT_EINVAL, "own-z source must be 0 (auto), 1, 2 or 3");
        c->oz_opt = (int)v;
        break;
    case LBMBT_OPT_SCHEME:
        if (v != 0 && v != 1) return fail(c, LBMBT_EINVAL, "scheme must be 0 (hybrid) or 1 (classical)");
        c->scheme = (int)v;
        break;
    case LBMBT_OPT_TEST_WAIT_NS:
        if (v < 0 || v > 1000000000LL) return fail(c, LBMBT_EINVAL, "test wait must be 0 (off) .. 1e9 ns");
        c->test_wait_ns = v;
        break;
    case LBMBT_OPT_COLUMN_PLANES:
        if (v < 0 || v > 64 || (v & (v - 1)) != 0)
            return fail(c, LBMBT_EINVAL, "column planes must be 0 (auto) or a power of two <= 64");
        c->zc_opt = (int)v;
        break;
    default: return fail(c, LBMBT_EINVAL, "unknown option %d", opt);
    }
    invalidate_run(c);
    return LBMBT_OK;
}

extern "C" int lbmbt_get_option(lbmbt_ctx* c, int opt, int64_t* v)
{
    if (!c || !v) return LBMBT_EINVAL;
    switch (opt) {
    case LBMBT_OPT_GRAPH: *v = c->use_graph; break;
    case LBMBT_OPT_AUTOTUNE: *v = c->autotune; break;
    case LBMBT_OPT_BLOCK: *v = c->block; break;
    case LBMBT_OPT_SPT: *v = c->spt; break;
    case LBMBT_OPT_KERNEL: *v = c->kernel_opt; break;
    case LBMBT_OPT_STAGES: *v = c->tma_stages; break;
    case LBMBT_OPT_TMA_SHAPE: *v = c->tma_variant; break;
    case LBMBT_OPT_ADJOINT_KERNEL: *v = c->adjoint_opt; break;
    case LBMBT_OPT_ADJOINT_SHAPE: *v = c->adj_shape; break;
    case LBMBT_OPT_LATTICE: *v = c->lattice; break;
    case LBMBT_OPT_STAGE_OWN_Z: *v = c->oz_opt; break;
    case LBMBT_OPT_SCHEME: *v = c->scheme; break;
    case LBMBT_OPT_GRAD_GROUPS: *v = c->grad_groups; break;
    case LBMBT_OPT_TEST_WAIT_NS: *v = c->test_wait_ns; break;
    case LBMBT_OPT_COLUMN_PLANES: *v = c->zc_opt; break;
    case LBMBT_OPT_STAGE_OWN_Z_USED: *v = c->prepared && c->use_tma ? c->tma_form + 1 : 0; break;
    case LBMBT_OPT_KERNEL_USED: *v = c->prepared ? (c->use_tma ? 2 : 1) : 0; break;
    default: return fail(c, LBMBT_EINVAL, "unknown option %d", opt);
    }
    return LBMBT_OK;
}

extern "C" int lbmbt_launch_count(lbmbt_ctx* c, int64_t* out)
{
    if (!c || !out) return LBMBT_EINVAL;
    *out = c->launches;
    return LBMBT_OK;
}

// ---------------------------------------------------------------- adjoint
static size_t grad_bytes_per_member(const lbmbt_ctx* c, long long plane, int ck)
{
    const long long n_ck = (c->n_steps + ck - 1) / ck;
    return (size_t)(2 + n_ck + ck + 1) * 7 * plane * sizeof(float2);
}

// One group of members: checkpointed forward pass, then segments in reverse:
// recompute the segment's forward levels from its checkpoint, then run the
// adjoint sweep back through it.
static int grad_group(lbmbt_ctx* c, int n, const lbmbt_member* mem, int ck, double* sig, double* dD, double* dT2,
                      double* dk)
{
    const int saved_block = c->block;
    if (c->block > 256) c->block = 256;
    int rc = prepare(c, n, mem, false, nullptr);
    c->block = saved_block;
    if (rc) return rc;
    const long long K = c->n_steps;
    const long long n_ck = (K + ck - 1) / ck;
    size_t lvl_total = 0;
    for (auto& d : c->descs) lvl_total += (size_t)7 * d.plane;
    rc = grow(c, &c->d_ck, &c->cap_ck, lvl_total * n_ck * sizeof(float2));
    if (!rc) rc = grow(c, &c->d_seg, &c->cap_seg, lvl_total * (ck + 1) * sizeof(float2));
    const bool adj_tma = c->adjoint_opt == 2 || (c->adjoint_opt == 0 && c->adj_tma_ok);
    if (c->adjoint_opt == 2 && !c->adj_tma_ok)
        return fail(c, LBMBT_EINVAL, "bulk-copy adjoint needs nx %% 16 == 0 and nx <= %d", adj_tma_max_sites(1));
    const long long n_gslots = adj_tma ? c->n_adj_units * adj_tma_slots_per_unit() : c->n_tiles;
    if (!rc) rc = grow(c, &c->d_gacc, &c->cap_gacc, sizeof(double) * NGACC * n_gslots);
    if (!rc) rc = grow(c, &c->d_gout, &c->cap_gout, sizeof(double) * NGACC * n);
    if (!rc) rc = grow(c, &c->d_laminit, &c->cap_laminit, sizeof(double2) * n);
    if (rc) return rc;
    // per-member bases of checkpoints and segment levels
    std::vector<float2*> ckb(n), segb(n);
    {
        size_t oc = 0, os = 0;
        for (int m = 0; m < n; ++m) {
            const size_t lv = (size_t)7 * c->descs[m].plane;
            ckb[m] = c->d_ck + oc;
            segb[m] = c->d_seg + os;
            oc += lv * n_ck;
            os += lv * (ck + 1);
        }
    }
    auto copy_level = [&](int m, const float2* from, float2* to) -> int {
        const size_t lv = (size_t)7 * c->descs[m].plane;
        CU(c, cudaMemcpyAsync(to, from, lv * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
        return LBMBT_OK;
    };
    // forward with checkpoints u^0, u^ck, u^2ck, ...; from the last
    // segment's first step on it writes its levels straight into the segment
    // buffer (slot k - k_last), so that segment is not recomputed
    const long long k_last = (n_ck - 1) * ck;
    rc = write_ctl(c, (int)(K - 1), -1);
    if (rc) return rc;
    if (n_ck > 1)
        for (int m = 0; m < n; ++m)
            if ((rc = copy_level(m, c->descs[m].state, ckb[m]))) return rc;
    for (long long k = 0; k < K; ++k) {
        if (k == k_last) {
            std::vector<MemberDesc> fd = c->descs;
            for (int m = 0; m < n; ++m) {
                const size_t lv = (size_t)7 * c->descs[m].plane;
                if ((rc = copy_level(m, c->descs[m].state + (k & 1) * lv, segb[m]))) return rc;
                fd[m].state = segb[m];
            }
            CU(c, cudaMemcpyAsync(c->d_desc, fd.data(), sizeof(MemberDesc) * n, cudaMemcpyHostToDevice, c->stream));
            c->k_cur = k;
            if ((rc = write_ctl(c, (int)(K - 1), -1, (int)k, ck + 1))) return rc;
        }
        if ((rc = issue_step(c))) return rc;
        const long long kn = k + 1;
        if (kn % ck == 0 && kn < k_last)
            for (int m = 0; m < n; ++m) {
                const size_t lv = (size_t)7 * c->descs[m].plane;
                if ((rc = copy_level(m, c->descs[m].state + (kn & 1) * lv, ckb[m] + (kn / ck) * lv))) return rc;
            }
    }
    c->k_cur = K;
    CU(c, launch_reduce(c->d_partial, part_start(c), part_per(c), n, c->d_Z, nullptr, 0, c->d_ctl, c->stream));
    c->launches++;
    std::vector<double2> Z(n);
    CU(c, cudaMemcpyAsync(Z.data(), c->d_Z, sizeof(double2) * n, cudaMemcpyDeviceToHost, c->stream));
    if ((rc = sync(c))) return rc;
    std::vector<double2> L(n);
    for (int m = 0; m < n; ++m) {
        const double N = (double)c->descs[m].N;
        const double a = std::hypot(Z[m].x, Z[m].y);
        sig[3 * m] = Z[m].x;
        sig[3 * m + 1] = Z[m].y;
        sig[3 * m + 2] = a / N;
        L[m] = a > 0 ? make_double2(Z[m].x / (N * a), Z[m].y / (N * a)) : make_double2(0.0, 0.0);
    }
    CU(c, cudaMemcpyAsync(c->d_laminit, L.data(), sizeof(double2) * n, cudaMemcpyHostToDevice, c->stream));
    // descriptors for the reverse pass: forward levels in the segment buffer,
    // adjoint ping-pong in the (now free) forward state
    std::vector<MemberDesc> rd = c->descs;
    for (int m = 0; m < n; ++m) {
        rd[m].adj = c->descs[m].state;
        rd[m].state = segb[m];
    }
    CU(c, cudaMemcpyAsync(c->d_desc, rd.data(), sizeof(MemberDesc) * n, cudaMemcpyHostToDevice, c->stream));
    CU(c, cudaMemsetAsync(c->d_gacc, 0, sizeof(double) * NGACC * n_gslots, c->stream));
    int adj_grid = 0;
    const int adj_stages = 3;
    // register adjoint: runs of up to 16 tiles per block, keeping >= 32
    // blocks per SM
    if (!c->sm_count) CU(c, cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
    const int adj_run = (int)std::max<long long>(1, std::min<long long>(16, c->n_tiles / (32LL * c->sm_count)));
    if (adj_tma) {
        int per_sm = 0;
        CU(c, adj_tma_prepare(c->adj_cap, adj_stages, c->adj_shape_used, &per_sm));
        if (per_sm < 1) return fail(c, LBMBT_EINVAL, "bulk-copy adjoint does not fit on an SM");
        if (!c->sm_count) CU(c, cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
        adj_grid = (int)std::min<long long>((long long)c->sm_count * per_sm, c->n_adj_units);
    }
    AdjointArgs aa;   // the boundary factors of every step: the forward's table
    aa.members = c->d_desc;
    aa.tile_start = c->d_tile_start;
    aa.n_members = n;
    aa.lam_init = c->d_laminit;
    aa.gacc = c->d_gacc;
    aa.ftab = c->d_ftab;
    aa.unit_start = c->d_adj_unit_start;
    aa.ctl_err = &c->d_ctl->err;
    {
        const SweepArgs sa = sweep_args(c);   // the forward's equilibrium weights
        aa.w0 = sa.w0;
        aa.wxy = sa.wxy;
        aa.wz = sa.wz;
    }
    int parity = 1;
    for (long long seg = n_ck - 1; seg >= 0; --seg) {
        const long long k0 = seg * ck, k1 = std::min(K, k0 + ck);
        if (seg < n_ck - 1) {   // the last segment's levels are in place from the forward pass
            for (int m = 0; m < n; ++m) {
                const size_t lv = (size_t)7 * c->descs[m].plane;
                if ((rc = copy_level(m, ckb[m] + seg * lv, segb[m]))) return rc;
            }
        }
        if (seg < n_ck - 1 && k1 - k0 - 1 > 0) {
            c->k_cur = k0;
            if ((rc = write_ctl(c, -1, -1, (int)k0, ck + 1))) return rc;
            for (long long k = k0; k < k1 - 1; ++k)
                if ((rc = issue_step(c))) return rc;
        }
        for (long long k = k1; k > k0; --k) {
            aa.k = (int)k;
            aa.first = (k == K) ? 1 : 0;
            aa.fwd_slot = (int)(k - 1 - k0);
            aa.lam_parity = parity;
            aa.fprev = (float)c->f[k - 1];
            if (adj_tma)
                CU(c, launch_adjoint_tma(aa, c->n_adj_units, c->adj_cap, adj_stages, c->adj_shape_used, adj_grid,
                                         c->stream));
            else CU(c, launch_adjoint(aa, c->n_tiles, c->tile_block, c->tile_spt, adj_run, c->stream));
            c->launches++;
            parity ^= 1;
        }
    }
    if (adj_tma) CU(c, launch_reduce_grad(c->d_gacc, c->d_adj_unit_start, adj_tma_slots_per_unit(), n, c->d_gout,
                                          c->stream));
    else CU(c, launch_reduce_grad(c->d_gacc, c->d_tile_start, 1, n, c->d_gout, c->stream));
    c->launches++;
    std::vector<double> G((size_t)NGACC * n);
    CU(c, cudaMemcpyAsync(G.data(), c->d_gout, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, c->stream));
    if ((rc = check_device_error(c))) return rc;
    c->prepared = false;  // descriptors now describe the reverse pass
    // chain rule to the physical parameters
    const double eps = c->lattice == 1 ? EPS_D2 : EPS_D;
    for (int m = 0; m < n; ++m) {
        const double dx = c->descs[m].dx, dt = c->dt;
        const double* g = &G[(size_t)NGACC * m];
        for (int p = 0; p < c->n_phases; ++p) {
            const double tau = 0.5 + dt * c->D[p] / (eps * dx * dx);
            const double om = 1.0 / tau;
            dD[(size_t)m * c->n_phases + p] = g[p] * (-om * om * dt / (eps * dx * dx));
            const double T2 = c->T2[p];
            if (std::isinf(T2)) {
                dT2[(size_t)m * c->n_phases + p] = 0.0;
            } else {
                const double one_m_eps = std::exp(-dt / T2);
                dT2[(size_t)m * c->n_phases + p] = g[4 + p] * (-one_m_eps * dt / (T2 * T2));
            }
        }
        const double kap = mem[m].kappa_um_ms;
        const double cP = eps * dx / (2.0 * dt);
        dk[m] = std::isinf(kap) ? 0.0 : g[8] * cP / ((kap + cP) * (kap + cP));
    }
    return LBMBT_OK;
}

extern "C" int lbmbt_grad_batch(lbmbt_ctx* c, int n_members, const lbmbt_member* members, int checkpoint_every,
                                double* signal_out, double* dS_dD, double* dS_dT2, double* dS_dkappa)
{
    if (!c) return LBMBT_EINVAL;
    if (!members || !signal_out || !dS_dD || !dS_dT2 || !dS_dkappa)
        return fail(c, LBMBT_EINVAL, "NULL argument");
    if (n_members < 1) return fail(c, LBMBT_EINVAL, "n_members must be >= 1");
    if (c->geoms.empty() || c->n_phases == 0 || c->n_steps == 0) return fail(c, LBMBT_ESTATE, "set-up incomplete");
    if (any_slab(c)) return fail(c, LBMBT_EUNSUPPORTED, "the adjoint sweep does not run on slabs");
    if (c->scheme != 0) return fail(c, LBMBT_EUNSUPPORTED, "the adjoint sweep is of the hybrid scheme only");
    for (auto& g : c->geoms)
        if (g.d_dlt) return fail(c, LBMBT_EUNSUPPORTED, "the adjoint sweep does not take membrane positions");
    if (c->lattice != 0 && c->adjoint_opt == 2)
        return fail(c, LBMBT_EUNSUPPORTED, "the bulk-copy adjoint runs on the D3Q7 lattice only");
    const int ck = checkpoint_every > 0 ? checkpoint_every : 64;
    int rc = set_device(c);
    if (rc) return rc;
    // group members so one group's levels fit in the free device memory
    size_t free_b = 0, total_b = 0;
    CU(c, cudaMemGetInfo(&free_b, &total_b));
    const size_t held = c->cap_state + c->cap_ck + c->cap_seg;
    const size_t budget = (size_t)((double)(free_b + held) * 0.8);
    int m0 = 0;
    c->grad_groups = 0;
    while (m0 < n_members) {
        size_t used = 0;
        int m1 = m0;
        while (m1 < n_members) {
            const lbmbt_member& mm = members[m1];
            if (mm.geometry < 0 || mm.geometry >= (int)c->geoms.size())
                return fail(c, LBMBT_EINVAL, "member %d: geometry %d not set", m1, mm.geometry);
            const long long plane = (c->geoms[mm.geometry].N + 63) / 64 * 64;
            const size_t b = grad_bytes_per_member(c, plane, ck);
            if (m1 > m0 && used + b > budget) break;
            used += b;
            ++m1;
        }
        if (used > budget) return fail(c, LBMBT_ENOMEM, "one member needs %zu bytes for the adjoint", used);
        rc = grad_group(c, m1 - m0, members + m0, ck, signal_out + 3 * m0, dS_dD + (size_t)m0 * c->n_phases,
                        dS_dT2 + (size_t)m0 * c->n_phases, dS_dkappa + m0);
        if (rc) return rc;
        ++c->grad_groups;
        m0 = m1;
    }
    return LBMBT_OK;
}

extern "C" int lbmbt_grad(lbmbt_ctx* c, int checkpoint_every, double* signal_out, double* dS_dD, double* dS_dT2,
                          double* dS_dkappa)
{
    if (!c) return LBMBT_EINVAL;
    lbmbt_member m = plain_member(c);
    return lbmbt_grad_batch(c, 1, &m, checkpoint_every, signal_out, dS_dD, dS_dT2, dS_dkappa);
}
