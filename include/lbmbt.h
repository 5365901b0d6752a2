/*
 * lbmbt.h -- C ABI of the GB300 (sm_103a) hybrid lattice-Boltzmann
 * Bloch-Torrey library (Naughton, Tennyson & Georgiadis, arXiv 1907.00908).
 *
 * The library advances the complex transverse magnetisation M(x, t) of the
 * Bloch-Torrey equation (Sec. 2.1, Eq. LBM-B-Teq) with the paper's hybrid
 * lattice Boltzmann scheme (Sec. 2.3, Eq. LBM_process_list_2) on a D3Q7
 * lattice and returns the diffusion-MRI signal at the echo.  Every time step
 * is one fused pass over the lattice: streaming with the outer boundary
 * conditions (Sec. 2.4.3 modified periodic, Sec. 2.4.4 mirroring) and the
 * half-link permeable-membrane rule (Sec. 2.4.2, Eqs. B5 and P_def), the
 * reaction (Eq. reaction_LBM: gradient phase and T2 decay) and the BGK
 * collision (Eq. collision_LBM) with a relaxation time per phase
 * (Eq. tau_def).  Arithmetic is FP32; the signal is summed in FP64.
 *
 * Conventions (all entry points):
 *  - Units: um, ms.  b in s/mm^2 (as in the paper); gamma*G0 in rad/(um ms);
 *    D in um^2/ms; T2 in ms (INFINITY = no decay); kappa in um/ms
 *    (0 = impermeable, INFINITY = no membrane).
 *  - Volumes are [nz][ny][nx], x fastest; node n of an axis sits at n*dx.
 *    A periodic axis of n nodes has period n*dx.
 *  - D3Q7 weights: eps_D = 1/4, omega_0 = 1/4, omega_1..6 = 1/8.
 *  - Every call returns an int status: LBMBT_OK (0) or a negative code.
 *    lbmbt_last_error(ctx) gives a message for the last failed call on ctx.
 *    No call aborts the process; device-side checks report LBMBT_EDEVICE.
 *  - Ownership: the caller owns every buffer it passes; the library copies
 *    what it keeps.  Device pointers must be on the context's device; work
 *    is issued on the stream given to lbmbt_create, and each call returns
 *    after that stream has finished the call's work.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef LBMBT_H
#define LBMBT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LBMBT_OK = 0,
    LBMBT_EINVAL = -1,       /* invalid argument                                */
    LBMBT_ENOMEM = -2,       /* device or host allocation failed                */
    LBMBT_ECUDA = -3,        /* CUDA runtime error (message has the CUDA text)  */
    LBMBT_EUNSTABLE = -4,    /* tau <= 1/2 (Eq. tau_def); < 0.75 with angles     */
    LBMBT_EUNSUPPORTED = -5, /* mirror face with a gradient neither normal nor
                                parallel to it (Sec. 2.4.4)                     */
    LBMBT_EDEVICE = -6,      /* a device-side check failed (e.g. bad label)     */
    LBMBT_ESTATE = -7        /* call order: geometry/phases/sequence missing    */
};

enum { LBMBT_BC_PERIODIC = 0, LBMBT_BC_MIRROR = 1 };

typedef struct lbmbt_ctx lbmbt_ctx;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out is NULL on error. */
int lbmbt_create(lbmbt_ctx** out, int device, void* cuda_stream);

/* Free the context and every device buffer it holds.  NULL is accepted. */
int lbmbt_destroy(lbmbt_ctx* ctx);

/* Message of the last failed call on ctx ("" if none).  Valid until the next
 * call on ctx.  ctx == NULL gives the message of the last failed create. */
const char* lbmbt_last_error(const lbmbt_ctx* ctx);

/* Library version string. */
const char* lbmbt_version(void);

/*
 * Geometry (Sec. 2.1 phases; Sec. 2.4.2 membranes; Secs. 2.4.3-2.4.4 outer
 * boundaries).  labels: int32 compartment id per node, [nz][ny][nx], host or
 * device memory (labels_on_device != 0 means device).  phase_of_label[n_labels]
 * (host): phase id (0..3) of each label.  bc[3]: per axis x, y, z,
 * LBMBT_BC_PERIODIC or LBMBT_BC_MIRROR.  Every link between two nodes with
 * different labels carries a membrane at its midpoint (Delta_m = 1/2,
 * theta = 0); a mirror face never does.  The library builds, on the device,
 * one byte per node: bit (i-1), i = 1..6, set iff the link to the neighbour
 * across +e_i (D3Q7 order +x,-x,+y,-y,+z,-z) is a membrane; bits 6-7 hold the
 * phase id.
 *
 * lbmbt_set_geometry replaces all geometries by this one (index 0);
 * lbmbt_add_geometry appends one and returns its index in *index_out (for
 * batched runs over several geometries).  Errors: EINVAL for bad sizes, a
 * label outside [0, n_labels) (reported by the device check as EDEVICE), or
 * a phase id > 3.
 */
int lbmbt_set_geometry(lbmbt_ctx* ctx, int nx, int ny, int nz, double dx_um,
                       const int32_t* labels, int labels_on_device, int n_labels,
                       const uint8_t* phase_of_label, const int bc[3]);
int lbmbt_add_geometry(lbmbt_ctx* ctx, int nx, int ny, int nz, double dx_um,
                       const int32_t* labels, int labels_on_device, int n_labels,
                       const uint8_t* phase_of_label, const int bc[3], int* index_out);

/*
 * Slab of a larger grid (the paper's strip decomposition, Sec. 2.5, cut along
 * z here): the context's only geometry becomes planes z0 .. z0+nz-1 of a grid
 * of nz_global planes, so a grid can be split over several contexts (one per
 * GPU, or several on one GPU) that exchange one plane of one population per
 * face and time step.  labels_ext: int32 [nz + 2][ny][nx], host or device:
 * the plane below the slab, the slab's nz planes, the plane above (labels of
 * the neighbouring slabs, so the face links get their membrane bits; at a
 * global periodic face the wrapped plane).  lo_kind / hi_kind say what lies
 * across the low / high z face:
 *   LBMBT_FACE_OWN        the global face, a mirror (bc[2] = LBMBT_BC_MIRROR);
 *   LBMBT_FACE_HALO       another slab;
 *   LBMBT_FACE_HALO_WRAP  another slab across the periodic global face (the
 *                         halo value takes the wrap factor exp(+-i gamma
 *                         L_z G_z F_k) of Sec. 2.4.3, L_z = nz_global dx).
 * A face is OWN or wraps iff the slab touches the global face.  Node
 * coordinates (reaction phase, mirror and wrap factors) are global.  nx must
 * be even.  A slab is stepped with lbmbt_prepare and lbmbt_advance(ctx, 1,
 * ...); between steps the caller moves each member's faces to its
 * neighbours' halos (lbmbt_slab_faces -> lbmbt_slab_set_halos).  The halos
 * start at the initial state (M = 1).  lbmbt_run, lbmbt_run_batch and
 * lbmbt_advance with more than one step return ESTATE / EINVAL on a slab;
 * the adjoint returns EUNSUPPORTED.  The signal of a slab is its part of Z:
 * the caller sums Z over the slabs.
 */
enum { LBMBT_FACE_OWN = 0, LBMBT_FACE_HALO = 1, LBMBT_FACE_HALO_WRAP = 2 };
int lbmbt_set_geometry_slab(lbmbt_ctx* ctx, int nx, int ny, int nz, double dx_um,
                            const int32_t* labels_ext, int labels_on_device, int n_labels,
                            const uint8_t* phase_of_label, const int bc[3], int z0, int nz_global,
                            int lo_kind, int hi_kind);

/* Faces of member `member` of a prepared slab run at the current step, before
 * the next lbmbt_advance: lo_out receives hat g_6 (the population moving to
 * -z) of the slab's first plane, for the slab below; hi_out hat g_5 (moving
 * to +z) of its last plane, for the slab above.  Each is nx*ny complex64
 * values [ny][nx], host or device memory (NULL: skip).  The copies are issued
 * on the context's stream and the call returns without waiting for them. */
int lbmbt_slab_faces(lbmbt_ctx* ctx, int member, void* lo_out, void* hi_out);

/* Halo planes of member `member` for the next lbmbt_advance: lo_in = hat g_5
 * of the plane below the slab (the lower neighbour's hi_out), hi_in = hat g_6
 * of the plane above (the upper neighbour's lo_out); nx*ny complex64 each,
 * host or device (NULL: leave unchanged, e.g. at an OWN face).  Issued on the
 * context's stream; the call returns without waiting. */
int lbmbt_slab_set_halos(lbmbt_ctx* ctx, int member, const void* lo_in, const void* hi_in);

/*
 * Membrane positions on the lattice links of geometry `index`, for the
 * membrane rule of a straight membrane normal to the link (theta = 0) at a
 * distance Delta_m dx from the node (Sec. 2.4.2, Eqs. B4a-B4c with the
 * coefficients of Eqs. c_n and c_d), instead of the half-link rule (Eq. B5,
 * Delta_m = 1/2).  delta: float32 [6][nz][ny][nx], host or device memory
 * (delta_on_device != 0 means device); entry j-1 at a node is Delta_m of its
 * link to the neighbour across +e_j (D3Q7 order +x, -x, +y, -y, +z, -z),
 * read only on membrane links, 0 < Delta_m < 1 (host input is checked:
 * EINVAL), and a consistent input gives the two ends of a link Delta_m and
 * 1 - Delta_m.  The rule uses the node behind each end (the second
 * neighbours x_ii, x_ee of Eqs. B2a/B2b); where one of them lies in another
 * compartment, and for kappa = INFINITY, the link keeps the half-link rule.
 * delta = NULL removes the positions.  Runs with positions use the register
 * sweep (LBMBT_OPT_KERNEL = 2 fails with EINVAL); the adjoint and slabs
 * return EUNSUPPORTED.
 */
int lbmbt_set_link_distances(lbmbt_ctx* ctx, int index, const float* delta, int delta_on_device);

/*
 * Membrane angles on the links of a one-plane (2-D) geometry `index`, for
 * the general-angle membrane rule (Appendix B: the Dirichlet and Neumann
 * relations of Eqs. dirichlet_1-neumann_2, the flux relations phi_1 and
 * phi_2, Eqs. B1 and B1.5; coefficients as Eqs. B3a-B3c).  theta: float32
 * [6][1][ny][nx], host or device (theta_on_device != 0 means device); entry
 * j-1 at a node is the signed angle between the membrane normal, pointing
 * from the node's compartment to the neighbour's, and its link to the
 * neighbour across +e_j: normal = cos(theta) e_j + sin(theta) e_perp, e_perp
 * = +y for x links and +x for y links; |theta| < pi/2 (host input is
 * checked: EINVAL); a consistent input gives the two ends of a link opposite
 * angles.  The values at the membrane point and one lattice step to either
 * side along the perpendicular direction are extrapolated quadratically along
 * the link from the three nearest nodes of the same compartment; where such
 * a node lies in another compartment or beyond a mirror face, or an axis is
 * shorter than 4 nodes, the link keeps the theta = 0 rule.  Requires the
 * positions (lbmbt_set_link_distances, else EINVAL), a geometry of one z
 * plane (else EINVAL) and the D2Q5 lattice (LBMBT_OPT_LATTICE = 1; a run
 * on D3Q7 returns EUNSUPPORTED).  The extrapolation is unstable for tau near
 * 1/2: a run needs tau >= 0.75 in every phase (else EUNSTABLE).  Removing
 * the positions removes the angles; theta = NULL removes the angles only.
 * The paper gives this rule in 2-D only; there is no 3-D form here.
 */
int lbmbt_set_link_angles(lbmbt_ctx* ctx, int index, const float* theta, int theta_on_device);

/* Copy the per-node mask byte of geometry `index` (encoding above) to host
 * memory mask_out[nz*ny*nx]. */
int lbmbt_get_mask(lbmbt_ctx* ctx, int index, uint8_t* mask_out);

/* Piecewise-uniform diffusivity and T2 per phase (Sec. 2.1), n_phases 1..4.
 * tau_p = 1/2 + dt D_p / (eps_D dx^2) (Eq. tau_def) is checked at run time:
 * tau <= 1/2 gives EUNSTABLE. */
int lbmbt_set_phases(lbmbt_ctx* ctx, int n_phases, const double* D_um2_ms, const double* T2_ms);

/* Membrane permeability kappa (Eq. permeability_flux) for plain runs and the
 * default of batched members.  The link rule uses P = eps_D dx/(2 kappa dt)
 * (Eq. P_def): a share s = 1/(1+P) crosses, r = P/(1+P) is reflected
 * (Eq. B5). */
int lbmbt_set_permeability(lbmbt_ctx* ctx, double kappa_um_ms);

/* Gradient sequence G(t) = G0 f(t) (Sec. 2.1).  f[k] (host, n_steps values) is
 * the waveform used during step k (Eq. reaction_LBM at t^k = k dt); the
 * periodic boundary phase uses F_k = sum_{m<k} f[m] dt (Eq. periodic_phi).
 * gamma_G0[3] = gamma*G0 in rad/(um ms).  The run ends at t = n_steps*dt. */
int lbmbt_set_sequence(lbmbt_ctx* ctx, double dt_ms, int64_t n_steps, const double* f,
                       const double gamma_G0[3]);

/* Sequence with reaction sub-steps (Sec. 2.3: dt = k dt', one diffusion step
 * then k reaction steps): f_fine (host, n_steps * substeps values) samples
 * the waveform on the dt' = dt / substeps grid.  The k reaction factors of a
 * site commute, so the library applies one reaction per step with the mean
 * of the step's k samples (and the same F_k); substeps = 1 is
 * lbmbt_set_sequence.  Errors as lbmbt_set_sequence, EINVAL for substeps < 1. */
int lbmbt_set_sequence_substeps(lbmbt_ctx* ctx, double dt_ms, int64_t n_steps, int substeps,
                                const double* f_fine, const double gamma_G0[3]);

/* PGSE helper (Sec. 2.1, Fig. 2): from b (s/mm^2), delta, Delta, dt and a
 * direction, gamma_G0_out = sqrt(b/(delta^2 (Delta - delta/3))) * unit(dir)
 * and the effective waveform sampled at t^k = k dt: +1 on [0, delta), -1 on
 * [Delta, Delta + delta), 0 elsewhere, ending at TE = Delta + delta.
 * *n_steps_out = (Delta + delta)/dt; f_out (host, may be NULL to query the
 * length) receives n_steps values.  delta/dt and Delta/dt must be integers
 * (within 1e-9) else EINVAL. */
int lbmbt_pgse(double b_s_mm2, double delta_ms, double Delta_ms, double dt_ms,
               const double dir[3], double gamma_G0_out[3], int64_t* n_steps_out, double* f_out);

/*
 * Plain run from M = 1 (Sec. 2.1) over the set sequence on geometry 0.
 * signal_out[3] (host) = {Re Z, Im Z, |Z|/N} with Z = sum_x M(x, t_end)
 * (FP64 sum).  field_out_dev: device complex64 [N] receiving M(x, t_end), or
 * NULL.  series_out: host [n_steps][2] receiving Z after every step, or NULL.
 */
int lbmbt_run(lbmbt_ctx* ctx, double* signal_out, void* field_out_dev, double* series_out);

/* One member of a batched run: its gradient (direction x amplitude), the
 * geometry it runs on (index from set/add_geometry) and its permeability. */
typedef struct {
    double gamma_G0[3];
    int geometry;
    double kappa_um_ms;
} lbmbt_member;

/*
 * Batched run: n_members independent runs that share the set waveform f, dt
 * and phases, advanced together by one launch per time step over a work list
 * of (member, tile) (captured in a CUDA graph when enabled).  Members on the
 * same geometry share its mask.  signal_out (host) [n_members][3] as in
 * lbmbt_run; series_out (host) [n_members][n_steps][2] or NULL.
 */
int lbmbt_run_batch(lbmbt_ctx* ctx, int n_members, const lbmbt_member* members,
                    double* signal_out, double* series_out);

/* One member of lbmbt_run_batch_ex: lbmbt_member plus the member's own
 * gradient waveform and field output.  The dMRI protocols the method serves
 * (Sec. 2.1, Fig. 2) mix diffusion times (delta, Delta), so a batch can mix
 * waveforms:
 *   f        host, the member's waveform f[0 .. n_steps-1] sampled as in
 *            lbmbt_set_sequence (same dt), or NULL for the set waveform;
 *   n_steps  length of f, 1 .. the set sequence's n_steps (ignored when f is
 *            NULL): the member's signal and field are those at t = n_steps*dt
 *            (its echo); the batch runs to the longest, and a shorter member
 *            keeps stepping with f = 0 after its end, unobserved;
 *   field_dev device complex64 [N of its geometry] receiving M(x) at the
 *            member's end, or NULL. */
typedef struct {
    double gamma_G0[3];
    int geometry;
    double kappa_um_ms;
    const double* f;
    int64_t n_steps;
    void* field_dev;
} lbmbt_member_ex;

/*
 * lbmbt_run_batch with per-member waveforms and field outputs (one launch
 * per time step, as lbmbt_run_batch).  signal_out[n_members][3] as in
 * lbmbt_run, each member's at its own end; series_out [n_members][n_steps][2]
 * or NULL (entries past a member's end are of its continued, unobserved run).
 * The waveforms and fields are used by this call only.  Errors: EINVAL for a
 * waveform longer than the set sequence, empty, or not finite.
 */
int lbmbt_run_batch_ex(lbmbt_ctx* ctx, int n_members, const lbmbt_member_ex* members,
                       double* signal_out, double* series_out);

/*
 * Gradient of S = |Z|/N at t_end with respect to the per-phase D_p and T2_p
 * and the permeability kappa, for the plain run (geometry 0, set gradient),
 * by a hand-written adjoint (reverse-time) sweep: the forward states are
 * checkpointed every `checkpoint_every` steps (<= 0: 64) and recomputed
 * segment by segment.  signal_out[3] as in lbmbt_run; dS_dD[n_phases],
 * dS_dT2[n_phases] (host; T2 = INFINITY gives 0), dS_dkappa[1] (host).
 */
int lbmbt_grad(lbmbt_ctx* ctx, int checkpoint_every, double* signal_out,
               double* dS_dD, double* dS_dT2, double* dS_dkappa);

/* Batched form of lbmbt_grad: per member signal_out[n][3], dS_dD[n][n_phases],
 * dS_dT2[n][n_phases], dS_dkappa[n]. */
int lbmbt_grad_batch(lbmbt_ctx* ctx, int n_members, const lbmbt_member* members,
                     int checkpoint_every, double* signal_out, double* dS_dD,
                     double* dS_dT2, double* dS_dkappa);

/* Options. */
enum {
    LBMBT_OPT_GRAPH = 1,     /* 1 (default): replay step loops as CUDA graphs   */
    LBMBT_OPT_AUTOTUNE = 2,  /* 1: time launch shapes on first use (default 0)  */
    LBMBT_OPT_BLOCK = 3,     /* threads per block of the register sweep: a
                                multiple of 32 in 64..512                      */
    LBMBT_OPT_SPT = 4,       /* sites per thread of the sweep (1, 2 or 4)       */
    LBMBT_OPT_KERNEL = 5,    /* 0 (default) auto, 1 register sweep, 2 bulk-copy
                                (TMA) sweep; auto takes the bulk-copy sweep when
                                every member has nx % 16 == 0 and nx <= 1024  */
    LBMBT_OPT_KERNEL_USED = 6, /* read-only: 1 or 2 for the prepared run, else 0 */
    LBMBT_OPT_STAGES = 7,    /* shared-memory stages of the bulk-copy sweep, 2..6
                                as far as they fit (3 of 1024-site units); more
                                than fit give EINVAL                          */
    LBMBT_OPT_TMA_SHAPE = 8, /* bulk-copy consumers x sites per thread per unit:
                                0 = 512 x 2, 1 = 384 x 3, 2 = 256 x 4,
                                3 = 352 x 3 (default)                         */
    LBMBT_OPT_ADJOINT_KERNEL = 9, /* 0 (default) auto, 1 register adjoint sweep,
                                2 bulk-copy adjoint sweep (nx % 16 == 0, nx <= 512) */
    LBMBT_OPT_ADJOINT_SHAPE = 10, /* bulk-copy adjoint consumers x sites per thread:
                                0 = 256 x 2, 1 = 512 x 1, 2 = 480 x 1 (default;
                                units of <= 480 sites, so a run with an
                                nx > 480 takes shape 1)                        */
    LBMBT_OPT_LATTICE = 11,  /* 0 (default) D3Q7; 1 the 2-D D2Q5 lattice of
                                Sec. 2.3 (eps_D = 1/3, omega_0 = 1/3,
                                omega_1..4 = 1/6; tau, P and the membrane
                                coefficients use eps_D = 1/3) on geometries of
                                one z plane, register sweep and register
                                adjoint only (a forced bulk-copy adjoint
                                returns EUNSUPPORTED)                          */
    LBMBT_OPT_STAGE_OWN_Z = 12, /* bulk-copy sweep, geometries with membranes:
                                where the own-site values of the z populations
                                come from.  0 (default) auto: when some member
                                with membranes has a plane of >= 2^17 sites,
                                z-marching if the grid gives at least 32
                                columns per SM of >= 8 planes (a column length
                                that divides every member's nz), else staged;
                                otherwise prefetched.  1 always prefetched into
                                registers; 2 always staged with the unit (2 more
                                rows per stage slot); 3 always z-marching: each
                                CTA walks columns of units (the same rows of
                                consecutive planes) in z order and carries the
                                z values from unit to unit                     */
    LBMBT_OPT_STAGE_OWN_Z_USED = 13, /* read-only: 1 prefetched, 2 staged or 3
                                z-marching for a prepared bulk-copy run, else 0 */
    LBMBT_OPT_SCHEME = 14,   /* 0 (default) the hybrid scheme (Eq.
                                LBM_process_list_2); 1 the paper's comparison
                                scheme, the classical LBM with the reaction as
                                a source term in the collision (Appendix A,
                                Eqs. A2 and A12): hat g_i = g_i - (g_i -
                                omega_i M)/tau + dt omega_i R M, R = -i gamma
                                x.G0 f(t^k) - 1/T2, no reaction step; the
                                outer faces then take the waveform integral
                                after the step, F_(k+1) = sum_{m<=k} f_m dt.
                                Both sweeps (bit-identical fields), half-link
                                membranes only
                                (positions: EUNSUPPORTED), no reaction
                                sub-steps (EINVAL), no slabs and no adjoint
                                (EUNSUPPORTED); both lattices              */
    LBMBT_OPT_GRAD_GROUPS = 15, /* read-only: the number of groups the last
                                lbmbt_grad_batch split its members into so
                                that one group's checkpoints fit in the free
                                device memory (0 before any)              */
    LBMBT_OPT_TEST_WAIT_NS = 16 /* tests of the timeout path only; 0 (default)
                                off.  1 .. 1e9: every consumer warp of the
                                bulk-copy sweep first waits, with this limit
                                in ns, on a shared-memory barrier that nothing
                                completes; the wait runs out as a wait for a
                                lost copy would (every wait of the sweep is
                                bounded by 2 s), the CTA sets the step
                                control's error word after its producer has
                                waited (bounded) for its own copies in
                                flight, and the call returns LBMBT_EDEVICE.
                                The context stays usable                  */,
    LBMBT_OPT_COLUMN_PLANES = 17, /* bulk-copy sweep, z-marching form: planes
                                per column.  0 (default) auto: the longest
                                power of two <= 32 that divides every
                                member's nz and leaves >= 32 columns per SM
                                (for a forced z-marching run without one,
                                the longest that divides them).  1, 2, 4,
                                .., 64: that length; the run fails with
                                LBMBT_EINVAL when it does not divide every
                                member's nz                                  */
};
int lbmbt_set_option(lbmbt_ctx* ctx, int option, int64_t value);
int lbmbt_get_option(lbmbt_ctx* ctx, int option, int64_t* value);

/*
 * Low-level timing hook: advance the set-up plain or batched work by
 * `n_steps` sweeps from its current state without re-initialising (the first
 * call after lbmbt_prepare starts from M = 1).  Used by benchmarks to time the
 * steady-state sweep; lbmbt_prepare allocates and initialises.
 * n_members/members as in lbmbt_run_batch (n_members = 0: the plain run).
 * Signal partials are reduced on the last of the steps when want_signal != 0
 * and written to signal_out[n][3] (host) if not NULL.
 */
int lbmbt_prepare(lbmbt_ctx* ctx, int n_members, const lbmbt_member* members);
int lbmbt_advance(lbmbt_ctx* ctx, int64_t n_steps, int want_signal, double* signal_out);

/* Field output of the next lbmbt_prepare: device complex64 [N] receiving
 * M(x, t_end) of the (single) member when lbmbt_advance performs the last
 * step of the sequence; NULL (default) for none.  The buffer must stay valid
 * until that step; lbmbt_prepare with more than one member then fails. */
int lbmbt_set_field(lbmbt_ctx* ctx, void* field_dev);

/* Number of kernel launches the library issued on ctx since creation. */
int lbmbt_launch_count(lbmbt_ctx* ctx, int64_t* count_out);

/*
 * Plain sweep that allocates no device memory.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc (device
 * memory owned by another allocator, loops that must not enter the driver's
 * allocator, embeddings that forbid allocation after start-up).  It needs no
 * context and runs the same kernels as lbmbt_run on buffers the caller owns:
 *   mask_dev   device, one byte per node in the encoding of lbmbt_set_geometry
 *              (e.g. copied from lbmbt_get_mask);
 *   state_dev  device, 2 x 7 x plane complex64 values, plane = N rounded up
 *              to a multiple of 64 (N = nx*ny*nz); with init != 0 (and k0 = 0)
 *              level 0 is set to M = 1 at equilibrium first.  After the call
 *              the state of step k0 + n_steps is in level (k0 + n_steps) % 2,
 *              so calls can be chained with increasing k0;
 *   f[n_total_steps] (host) the whole waveform, as in lbmbt_set_sequence; the
 *              call performs steps k0 .. k0 + n_steps - 1 of it;
 *   signal_out[3] (host) = {Re Z, Im Z, |Z|/N} at the end of the last step.
 * Its working data (descriptor, step word, waveform and boundary-factor
 * tables, per-tile signal partials) lives in one fixed file-scope device
 * array of 2,754,304 bytes (2.63 MiB) that every GPU which loads the library
 * holds until the process exits.  Limits: N <= 16,777,216 sites and n_total_steps <= 32,768; larger
 * inputs are rejected with LBMBT_EINVAL and a message in errbuf (errbuf may
 * be NULL).  Every phase id in the mask (bits 6-7) must be < n_phases, else
 * LBMBT_ESTATE before the state is touched.  The library cannot see the
 * sizes of the caller's buffers: they must hold what is stated above.
 * The first call on a device looks up the array's device address (once per
 * device, cached for the life of the process, so it is stale after a
 * cudaDeviceReset); make that first call before any stream capture.  Every
 * call copies the waveform from host memory and waits for its stream.  All
 * calls share the one array and every call overwrites what it needs of it:
 * calls that overlap on the GPU (different streams or host threads without
 * ordering) race and give wrong results.  Work is issued on cuda_stream
 * (NULL = legacy default stream) and the call returns after it finished.
 */
int lbmbt_sweep_noalloc(int nx, int ny, int nz, double dx_um, const uint8_t* mask_dev, const int bc[3],
                        int n_phases, const double* D_um2_ms, const double* T2_ms, double kappa_um_ms,
                        double dt_ms, int64_t n_total_steps, const double* f, const double gamma_G0[3],
                        void* state_dev, int64_t k0, int64_t n_steps, int init, double* signal_out,
                        void* cuda_stream, char* errbuf, size_t errlen);

#ifdef __cplusplus
}
#endif

#endif /* LBMBT_H */
