// lbmbt_internal.cuh -- device-side descriptors shared by the kernels and the
// host side of liblbmbt (not part of the public C ABI).
//
// State layout in HBM (structure of arrays): for one member the post-collision
// populations hat g_i(x) of one time level are 7 planes of complex64
// (float2 = re, im), plane i at base + i*plane, site s = (z*ny + y)*nx + x.
// `plane` >= N is rounded up to a multiple of 64 sites so every plane starts
// 512-byte aligned.  A member owns `n_slots` such time levels back to back
// (stride 7*plane): 2 for the ping-pong of a run, c+1 for an adjoint segment.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lbmbt {

constexpr int Q = 7;
// D3Q7 weights with eps_D = 1/4 (Sec. 2.3 pattern: w0 = eps_D, wi = eps_D/2).
constexpr float W0 = 0.25f;
constexpr float WI = 0.125f;
constexpr double EPS_D = 0.25;
// D2Q5 (Sec. 2.3, Eq. omega_i): eps_D = 1/3, w0 = 1/3, w1..4 = 1/6; run as
// the first five D3Q7 velocities on a grid of one z plane, z weights 0.
constexpr double EPS_D2 = 1.0 / 3.0;

// Outer-boundary handling of one axis for one member.
enum BcMode : int {
    BC_PER = 0,       // modified periodic (Sec. 2.4.3): wrap with exp(+-i phi)
    BC_MIR = 1,       // mirror, G parallel to the face: hat g_i(x_m) = hat g_ibar(x_n)
    BC_MIR_CONJ = 2,  // mirror, G normal to the face: conjugate + rewind (Sec. 2.4.4)
    // z faces of a slab cut out of a larger grid (the strips of Sec. 2.5):
    BC_HALO = 3,      // the neighbouring slab: value from the halo plane
    BC_HALO_PER = 4   // the neighbouring slab across the periodic global face:
                      // halo value times the wrap factor exp(+-i phi)
};

struct MemberDesc {
    float2* state;        // n_slots time levels, each 7 planes
    float2* adj;          // adjoint sweep: 2 levels of 7 planes (or nullptr)
    float2* field;        // M(x) output (complex64 [N]) or nullptr
    const uint8_t* mask;  // per-site membrane bits 0..5 + phase bits 6..7
    long long N;          // sites
    long long plane;      // plane stride in sites
    long long tile0;      // first work-list tile of this member (site tiles)
    long long unit0;      // first row-unit of this member (bulk-copy sweep)
    long long cc0;        // first unit column of this member (bulk-copy sweep, z-marching form)
    int rpu;              // x-rows per unit of the bulk-copy sweep
    int rpu_adj;          // x-rows per unit of the bulk-copy adjoint sweep
    long long unit0_adj;  // first row-unit of this member (bulk-copy adjoint)
    int nx, ny, nz;
    int bc[3];            // BcMode per axis
    double gG[3];         // gamma*G0, rad/(um ms)
    double dx;            // um
    float ctheta[3];      // -gG_a*dx*dt: reaction angle = f_k * sum_a ctheta_a * n_a
    float omega[4];       // 1/tau_p (Eq. tau_def)
    float eps[4];         // 1 - exp(-dt/T2_p), from expm1 in FP64; for the
                          // classical scheme dt/T2_p (its Euler source)
    float s_share;        // 1/(1+P): crossing share of a membrane link (Eq. B5)
    int axes;             // bit a set iff ctheta[a] != 0
    int memb;             // the geometry has at least one membrane link
    // exact division of site indices (< 2^28) by nx and ny: q = (n*m) >> s
    unsigned div_m[2];
    int div_s[2];
    // per-axis rotation tables (FP64-built): etab[off_a + n] =
    // (cos(ctheta_a n_a) - 1, sin(ctheta_a n_a)), offsets 0, nx, nx+ny, with
    // n_z = z0 + n (global plane index); or nullptr
    const float2* etab;
    // z extent within the whole grid: the member covers planes z0 .. z0+nz-1
    // of nzg (z0 = 0, nzg = nz unless the geometry is a slab)
    int z0, nzg;
    int zbc[2];           // BcMode of the low and high z face (bc[2] unless a slab)
    const float2* halo[2];  // slab halo planes (nx*ny complex64): hat g_5 of the
                          // plane below, hat g_6 of the plane above; or nullptr
    // membrane positions on the links (theta = 0 rule, Eqs. B4a-B4c):
    // dlt[(j-1)*plane + s] = distance in dx from s to the membrane on its
    // link to s + e_j; nullptr = half-link rule (Eq. B5) everywhere
    const float* dlt;
    float lrho;           // kappa dt / (eps_D dx): the coefficients depend on it only
    // membrane angles (one-plane D2Q5 grids, general-angle rule of Appendix
    // B): dth[(j-1)*plane + s] = signed angle between the membrane normal and
    // the link from s to s + e_j; nullptr = theta = 0 everywhere
    const float* dth;
    // the member's waveform: fw[k] = f_k as float (one entry past the end,
    // 0), Fw[k] = F_k = sum_{m<k} f_m dt (two entries past the end); the
    // run's shared tables unless the member has a waveform of its own
    const float* fw;
    const double* Fw;
    // step whose end signal partials (and field, if any) are this member's
    // own: its echo when it is shorter than the run; -1: the step control's
    int end_step;
};

// Step control word in device memory.  Every block of a sweep reads k at its
// start.  The bulk-copy sweep's last CTA to be done with it (a two-level
// ticket, no waiting) advances k; after a register sweep a one-thread kernel
// does.  So a captured graph of steps replays from any step.  No kernel ever
// waits on it.
constexpr unsigned CTL_SHARDS = 32;   // first-level ticket counters (same-address atomics serialise)
struct StepCtl {
    int k;              // step index the next sweep performs
    unsigned done;      // shards of the current sweep whose blocks are all done (0 between sweeps)
    int sig_step;       // step whose end signal is reduced (-1: none)
    int field_step;     // step whose end field is written (-1: none)
    int slot_base;      // src slot = (k - slot_base) % slot_mod
    int slot_mod;       // dst slot = (k + 1 - slot_base) % slot_mod
    int series;         // 1: reduce the signal after every step
    int err;            // device-side error bits
    unsigned shard[CTL_SHARDS];   // blocks b % CTL_SHARDS == s of the current sweep that are done
};

struct SweepArgs {
    const MemberDesc* members;
    const long long* tile_start;  // n_members + 1 prefix of tiles
    int n_members;
    StepCtl* ctl;
    const float* f;               // waveform per step
    const double* F;              // F_k = sum_{m<k} f_m dt, per step
    double2* partial;             // per-tile (sum Re M, sum Im M)
    const float2* fac;            // [K+1][n_members][6] boundary factors of every step
    int links;                    // 1: a member has membrane positions (register sweep
                                  // variant with the Eqs. B4a-B4c rule); 2: and angles
    float w0, wxy, wz;            // equilibrium weights (register sweep, init):
                                  // D3Q7 1/4, 1/8, 1/8; D2Q5 1/3, 1/6, 0 (Sec. 2.3)
    unsigned long long test_wait_ns;  // bulk-copy sweep, tests of the timeout path only: > 0
                                  // makes each consumer warp first wait, with this limit,
                                  // on a barrier nothing completes (0: off)
    int zc;                       // bulk-copy sweep, z-marching form: units per column
                                  // (consecutive z-planes of the same rows; a power of two
                                  // that divides every member's nz), else 0
    int zc_log2;                  // log2(zc)
    long long n_cc;               // z-marching: columns of all members
    const long long* cc_start;    // z-marching: n_members + 1 prefix of columns
    int scheme;                   // 0 the hybrid scheme; 1 the classical LBM with the
                                  // reaction as a collision source (Appendix A, Eq. A12),
                                  // register sweep only: f and F are then read one step
                                  // ahead (f[k+1], F[k+1]), since the loop state hat g(t^k)
                                  // already holds step k's source
};

// ---- launchers (sweep.cu) ------------------------------------------------
cudaError_t launch_build_mask(const int32_t* labels, const uint8_t* phase_of_label, int n_labels,
                              int nx, int ny, int nz, const int bc[3], uint8_t* mask, int* err,
                              cudaStream_t st);
// Writes v to the control word (before a run of sweeps, which then advance
// it themselves).
cudaError_t launch_ctl_set(StepCtl* ctl, const StepCtl& v, cudaStream_t st);
// Boundary factors of every step 0..K for every member, table[k][m][6], from
// each member's F table at k + F_shift (1 for the classical scheme, whose
// streamed populations already hold step k's source).
cudaError_t launch_factor_table(const MemberDesc* members, int n_members, int F_shift, long long K,
                                float2* table, cudaStream_t st);
cudaError_t launch_init(const SweepArgs& a, long long n_tiles, int block, int spt, int slot,
                        cudaStream_t st);
// Register sweep (one block per tile), then the one-thread step advance.
cudaError_t launch_sweep(const SweepArgs& a, long long n_tiles, int block, int spt, cudaStream_t st);
cudaError_t links_prepare();   // dynamic shared memory of the membrane-position sweeps
// Sums partial[tile_start[m]*per .. tile_start[m+1]*per) per member.
cudaError_t launch_reduce(const double2* partial, const long long* tile_start, int per, int n_members,
                          double2* out, double2* series, long long series_stride,
                          const StepCtl* ctl, cudaStream_t st);

// ---- bulk-copy sweep (sweep_tma.cu) --------------------------------------
// oz: the own rows of planes 5 and 6 go through the stage (wanted where
// planes are large, so those rows would otherwise come from DRAM a plane
// later); without it they are prefetched into registers with planes 3 and 4.
size_t tma_smem_bytes(int cap, int capx, int nst, int form);
int tma_partials_per_unit(int variant);
cudaError_t tma_prepare(int cap, int capx, int nst, int variant, int form, int* ctas_per_sm);
cudaError_t launch_sweep_tma(const SweepArgs& a, long long n_units, int cap, int capx, int nst, int variant, int form,
                             int grid, cudaStream_t st);

// ---- adjoint (adjoint.cu) -------------------------------------------------
// Per-tile gradient accumulators: [0..3] sum <lambda, w M - g> per phase
// (d/d omega_p), [4..7] sum <mu, -exp(i theta) g'> per phase (d/d eps_p),
// [8] sum over membrane links <nu, v - o> (d/d s).
constexpr int NGACC = 9;

struct AdjointArgs {
    const MemberDesc* members;    // state = the segment of forward levels
    const long long* tile_start;
    int n_members;
    int k;                        // adjoint step: nu^k -> nu^(k-1)
    int first;                    // 1: lambda^K is uniform, lam_init[member]
    int fwd_slot;                 // level of u^(k-1) in the member's state
    int lam_parity;               // nu^k is adj level lam_parity
    const double2* lam_init;      // per member Z / (N |Z|)
    float fprev;                  // f_(k-1)
    double* gacc;                 // per tile NGACC doubles, accumulated
    const float2* ftab;           // [K+1][n_members][6] boundary factors
    const long long* unit_start;  // bulk-copy adjoint: row-unit prefix
    int* ctl_err;                 // error word of the step control
    float w0, wxy, wz;            // equilibrium weights (register adjoint; the
                                  // bulk-copy adjoint has the D3Q7 ones built in)
};
// run: consecutive tiles per block (the block keeps its gradient partials over them)
cudaError_t launch_adjoint(const AdjointArgs& a, long long n_tiles, int block, int spt, int run, cudaStream_t st);
// Sums gacc slots [tile_start[m]*per, tile_start[m+1]*per) per member.
cudaError_t launch_reduce_grad(const double* gacc, const long long* tile_start, int per, int n_members, double* out,
                               cudaStream_t st);
// bulk-copy adjoint (adjoint_tma.cu)
int adj_tma_slots_per_unit();
int adj_tma_max_sites(int shape);
cudaError_t adj_tma_prepare(int cap, int nst, int shape, int* ctas_per_sm);
cudaError_t launch_adjoint_tma(const AdjointArgs& a, long long n_units, int cap, int nst, int shape, int grid,
                               cudaStream_t st);

}  // namespace lbmbt
