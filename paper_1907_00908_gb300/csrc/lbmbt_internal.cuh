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

// Outer-boundary handling of one axis for one member.
enum BcMode : int {
    BC_PER = 0,       // modified periodic (Sec. 2.4.3): wrap with exp(+-i phi)
    BC_MIR = 1,       // mirror, G parallel to the face: hat g_i(x_m) = hat g_ibar(x_n)
    BC_MIR_CONJ = 2   // mirror, G normal to the face: conjugate + rewind (Sec. 2.4.4)
};

struct MemberDesc {
    float2* state;        // n_slots time levels, each 7 planes
    float2* adj;          // adjoint sweep: 2 levels of 7 planes (or nullptr)
    float2* field;        // M(x) output (complex64 [N]) or nullptr
    const uint8_t* mask;  // per-site membrane bits 0..5 + phase bits 6..7
    long long N;          // sites
    long long plane;      // plane stride in sites
    long long tile0;      // first work-list tile of this member
    int nx, ny, nz;
    int bc[3];            // BcMode per axis
    double gG[3];         // gamma*G0, rad/(um ms)
    double dx;            // um
    float ctheta[3];      // -gG_a*dx*dt: reaction angle = f_k * sum_a ctheta_a * n_a
    float omega[4];       // 1/tau_p (Eq. tau_def)
    float eps[4];         // 1 - exp(-dt/T2_p), from expm1 in FP64
    float s_share;        // 1/(1+P): crossing share of a membrane link (Eq. B5)
    float pad_;
};

// Step control word in device memory.  The sweep reads k here; the last block
// of every sweep launch advances it, so a captured graph of sweeps can be
// replayed from any step.  No kernel ever waits on it.
struct StepCtl {
    int k;              // step index the next sweep performs
    unsigned done;      // blocks finished in the current sweep
    int sig_step;       // step whose end signal is reduced (-1: none)
    int field_step;     // step whose end field is written (-1: none)
    int slot_base;      // src slot = (k - slot_base) % slot_mod
    int slot_mod;       // dst slot = (k + 1 - slot_base) % slot_mod
    int series;         // 1: reduce the signal after every step
    int err;            // device-side error bits
};

struct SweepArgs {
    const MemberDesc* members;
    const long long* tile_start;  // n_members + 1 prefix of tiles
    int n_members;
    StepCtl* ctl;
    const float* f;               // waveform per step
    const double* F;              // F_k = sum_{m<k} f_m dt, per step
    double2* partial;             // per-tile (sum Re M, sum Im M)
};

// ---- launchers (sweep.cu) ------------------------------------------------
cudaError_t launch_build_mask(const int32_t* labels, const uint8_t* phase_of_label, int n_labels,
                              int nx, int ny, int nz, const int bc[3], uint8_t* mask, int* err,
                              cudaStream_t st);
cudaError_t launch_set_ctl(StepCtl* ctl, const StepCtl& v, cudaStream_t st);
cudaError_t launch_init(const SweepArgs& a, long long n_tiles, int block, int spt, int slot,
                        cudaStream_t st);
cudaError_t launch_sweep(const SweepArgs& a, long long n_tiles, int block, int spt, cudaStream_t st);
cudaError_t launch_reduce(const double2* partial, const long long* tile_start, int n_members,
                          double2* out, double2* series, long long series_stride,
                          const StepCtl* ctl, cudaStream_t st);

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
    double Fprev;                 // F_(k-1)
    double* gacc;                 // per tile NGACC doubles, accumulated
};
cudaError_t launch_adjoint(const AdjointArgs& a, double Fk, long long n_tiles, int block, int spt, cudaStream_t st);
cudaError_t launch_reduce_grad(const double* gacc, const long long* tile_start, int n_members, double* out,
                               cudaStream_t st);

}  // namespace lbmbt
