/*
 * lbm_oracle.c -- plain, slow FP64 CPU reference of the hybrid lattice
 * Boltzmann Bloch-Torrey scheme (Naughton, Tennyson & Georgiadis,
 * arXiv 1907.00908).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA path is checked
 * against.  It shares no code, header, table or helper with the library under
 * paper_1907_00908_gb300/; only tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It is deliberately unoptimised: every step of one
 * time step is a separate sweep over the lattice, in the order the paper gives
 * (Eq. LBM_process_list_2): collision -> boundary/buffer layers -> streaming
 * (with the half-link membrane rule) -> reaction.
 *
 * The paper's comparison scheme, the classical LBM with the reaction as a
 * source term in the collision (Appendix A, Eq. A12), is the same loop with
 * the source added in the collision and no reaction step
 * (lbm_oracle_run_scheme).
 *
 * Lattice: D3Q7, directions 0=(0,0,0), 1=+x, 2=-x, 3=+y, 4=-y, 5=+z, 6=-z.
 * Weights: the paper gives D2Q5 only (Sec. 2.3: omega_0 = eps_D, omega_i =
 * eps_D/2, eps_D = 1/3).  For D3Q7 the same pattern with the isotropy
 * condition sum_i omega_i e_ia e_ib = eps_D delta_ab gives eps_D = 1/4,
 * omega_0 = 1/4, omega_1..6 = 1/8; this reproduces the tau = 0.58 the paper
 * quotes for its 3-D code (Sec. 3.5: D = 2.0, dt = 0.010, dx = 1.0).
 *
 * Grid: nx*ny*nz unique nodes, x fastest; node n sits at x_n = n*dx.
 * A periodic axis of N nodes has period L = N*dx (the paper's node N, which
 * duplicates node 0, is dropped).  Buffer layers at n = -2, -1 and n = N,
 * N+1 are held explicitly in a padded copy of the post-collision state (the
 * second layer serves the second-neighbour terms of the link-distance
 * membrane rule, Eqs. B4a-B4c).
 *
 * Units: um, ms.  gG[a] = gamma*G0_a in rad/(um*ms); D in um^2/ms; T2 in ms
 * (INFINITY allowed); kappa in um/ms (0 = impermeable, INFINITY = no membrane).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { Q = 7 };
static const int EX[Q] = {0, 1, -1, 0, 0, 0, 0};
static const int EY[Q] = {0, 0, 0, 1, -1, 0, 0};
static const int EZ[Q] = {0, 0, 0, 0, 0, 1, -1};
static const int OPP[Q] = {0, 2, 1, 4, 3, 6, 5};
/* D3Q7: eps_D = 1/4, omega_0 = eps_D, omega_i = eps_D / 2 (Sec. 2.3 weights) */
static const double EPS_D = 0.25;
static const double W[Q] = {0.25, 0.125, 0.125, 0.125, 0.125, 0.125, 0.125};
/* D2Q5 (Sec. 2.3, Eq. omega_i): directions 0, +x, -x, +y, -y (the first five
 * above), eps_D = 1/3, omega_0 = eps_D, omega_1..4 = eps_D / 2; the grid has
 * one z plane and the z populations are not used. */
static const double EPS_D2 = 1.0 / 3.0;
static const double W2[Q] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 0.0, 0.0};

enum { BC_PERIODIC = 0, BC_MIRROR = 1 };

/* Reflection of a lattice direction across a face normal to axis a: the axis-a
 * component flips, the others are unchanged.  For the direction that crosses
 * the face this is the opposite direction i-bar (Sec. 2.4.4). */
static int reflect_dir(int i, int axis)
{
    int e[3] = {EX[i], EY[i], EZ[i]};
    e[axis] = -e[axis];
    for (int j = 0; j < Q; ++j)
        if (EX[j] == e[0] && EY[j] == e[1] && EZ[j] == e[2]) return j;
    return -1;
}

/* Padded layout: (nx+4) x (ny+4) x (nz+4) nodes, coordinate -2..N+1 on each
 * axis; Q complex populations per node. */
enum { PAD = 2 };
typedef struct {
    int nx, ny, nz;
    int px, py, pz;
} grid_t;

static size_t pidx(const grid_t* g, int x, int y, int z)
{
    return ((size_t)(z + PAD) * g->py + (size_t)(y + PAD)) * g->px + (size_t)(x + PAD);
}

static size_t sidx(const grid_t* g, int x, int y, int z)
{
    return ((size_t)z * g->ny + (size_t)y) * g->nx + (size_t)x;
}

/* Eq. tau_def: tau = 1/2 + dt*D / (eps_D dx^2). */
static double tau_of(double D, double dt, double dx, double eps)
{
    return 0.5 + dt * D / (eps * dx * dx);
}

/* Eqs. P_def and B5: P = eps_D dx / (2 kappa dt); reflected share r = P/(1+P),
 * transmitted share s = 1/(1+P).  kappa = 0 -> P = inf (bounce-back);
 * kappa = inf -> P = 0 (plain streaming). */
static void membrane_shares(double kappa, double dt, double dx, double eps, double* r, double* s)
{
    if (kappa == 0.0) { *r = 1.0; *s = 0.0; return; }
    if (isinf(kappa)) { *r = 0.0; *s = 1.0; return; }
    double P = eps * dx / (2.0 * kappa * dt);
    *r = P / (1.0 + P);
    *s = 1.0 / (1.0 + P);
}

/* Coefficients of the link-distance membrane rule for a straight membrane
 * normal to the link (theta = 0), Eqs. B4a-B4c, from the Neumann (Eq. c_n)
 * and Dirichlet (Eq. c_d) coefficients of the node's fraction dl = Delta_m
 * and of the far node's fraction 1 - dl:
 *   A_j = (c_d4 c*_d4 c_nj eps_D dx + (c*_d4 c_n4 c_dj + c*_n4 c_d4 c_nj) kappa dt) / F
 *   B_j = c_d4 c_n4 (c*_nj - c*_dj) kappa dt / F
 *   F   = c_d4 c*_d4 eps_D dx + (c_d4 c*_n4 + c_n4 c*_d4) kappa dt.
 * A[0..2] multiply (own population towards the membrane, the same population
 * one node further back, own population away from it); B[0..2] multiply
 * (population arriving from the far node, the same population one node
 * beyond it, far node's population towards the membrane). */
static void coef_n(double d, double c[4])
{
    c[0] = 1.0;
    c[1] = -(2.0 * d - 1.0) / (2.0 * d + 1.0);
    c[2] = (2.0 * d - 1.0) / (2.0 * d + 1.0);
    c[3] = 2.0 / (2.0 * d + 1.0);
}

static void coef_d(double d, double c[4])
{
    c[0] = 2.0 * (d - 1.0);
    c[1] = -(2.0 * d - 1.0) * (2.0 * d - 1.0) / (2.0 * d + 1.0);
    c[2] = 2.0 * (2.0 * d - 1.0) / (2.0 * d + 1.0);
    c[3] = (3.0 - 2.0 * d) / (2.0 * d + 1.0);
}

static void link_coefficients(double dl, double kappa, double dt, double dx, double eps, double* A, double* B)
{
    double cn[4], cd[4], cns[4], cds[4];
    coef_n(dl, cn);
    coef_d(dl, cd);
    coef_n(1.0 - dl, cns);
    coef_d(1.0 - dl, cds);
    const double ex = eps * dx, kd = kappa * dt;
    const double F = cd[3] * cds[3] * ex + (cd[3] * cns[3] + cn[3] * cds[3]) * kd;
    for (int j = 0; j < 3; ++j) {
        A[j] = (cd[3] * cds[3] * cn[j] * ex + (cds[3] * cn[3] * cd[j] + cns[3] * cd[3] * cn[j]) * kd) / F;
        B[j] = cd[3] * cn[3] * (cns[j] - cds[j]) * kd / F;
    }
}

void lbm_oracle_link_coefficients(double dl, double kappa, double dt, double dx, double* A, double* B)
{
    link_coefficients(dl, kappa, dt, dx, EPS_D, A, B);
}

/*
 * General-angle membrane rule in 2-D (Appendix B: Eqs. dirichlet_1-neumann_2
 * for the link, Eqs. phi_1 and phi_2 for the lattice-direction fluxes, Eqs.
 * B1 and B1.5 for the membrane), for the population X = g'_abar(x_i)
 * arriving at the node x_i from the membrane on its link to x_e, alpha
 * pointing from x_i towards the membrane.  theta is the angle between the
 * membrane normal and the link; beta is the perpendicular lattice direction
 * with a positive component along the normal from x_i's side to x_e's.
 * Inputs (post-collision values):
 *   a = (hat g_alpha(x_i), hat g_alpha(x_ii), hat g_abar(x_i))
 *   b = (hat g_abar(x_e), hat g_abar(x_ee), hat g_alpha(x_e))
 *   p = (hat g_beta(x'_i), hat g_beta(x'_ii), hat g_bbar(x'_i))
 *   q = (hat g_bbar(x'_e), hat g_bbar(x'_ee), hat g_beta(x'_e))
 * The unknowns X, Y = g'_alpha(x_e) and V = (dt/dx) Phi_n,in satisfy three
 * linear equations (each relation written out below), solved by Cramer's
 * rule.  c' are the coefficients of Eqs. c_n, c_d at Delta_m = 0, c* at
 * 1 - Delta_m.  kappa = 0 gives the impermeable wall.
 */
static cplx angled_link(double dl, double th, double kappa, double dt, double dx, double eps,
                        const cplx a[3], const cplx b[3], const cplx p[3], const cplx q[3])
{
    double cn[4], cd[4], cns[4], cds[4], cnp[4], cdp[4];
    coef_n(dl, cn);
    coef_d(dl, cd);
    coef_n(1.0 - dl, cns);
    coef_d(1.0 - dl, cds);
    coef_n(0.0, cnp);
    coef_d(0.0, cdp);
    const double st = fabs(sin(th)), ct = cos(th);
    const double rho = kappa * dt / (eps * dx);
    /* the three-term sums of the Dirichlet and Neumann relations on each side
     * (Eqs. dirichlet_1, neumann_1 with a; dirichlet_2, neumann_2 with b) and
     * the Neumann-minus-Dirichlet sums along beta (Eqs. phi_1, phi_2) */
    cplx Sd = 0, Sn = 0, Sds = 0, Sns = 0, Tp = 0, Tq = 0;
    for (int j = 0; j < 3; ++j) {
        Sd += cd[j] * a[j];
        Sn += cn[j] * a[j];
        Sds += cds[j] * b[j];
        Sns += cns[j] * b[j];
        Tp += (cnp[j] - cdp[j]) * p[j];
        Tq += (cnp[j] - cdp[j]) * q[j];
    }
    const double rp = cnp[3] / cdp[3];
    const double Ki = cn[3] / cd[3] * st + rp * ct, Ke = cns[3] / cds[3] * st + rp * ct;
    /* Eq. neumann_1: (dt/dx) Phi_nabar = (X - Sn) / c_n4; Eq. phi_1 then reads
     *   (X - Sn)/c_n4 * Ki = Tp st / c'_d4 - (Sn - Sd) st / c_d4 + rp V        (row 0)
     * Eq. neumann_2 and Eq. phi_2 with Phi_n,ex = -Phi_n,in (Eq. B1.5):
     *   (Y - Sns)/c*_n4 * Ke = Tq st / c'_d4 - (Sns - Sds) st / c*_d4 - rp V   (row 1)
     * Eq. B1 with Eqs. dirichlet_1/2 (eps_D Phi_d = (X - Sd)/c_d4 ...):
     *   V = rho ((Y - Sds)/c*_d4 - (X - Sd)/c_d4)                              (row 2) */
    const double M[3][3] = {{Ki / cn[3], 0.0, -rp},
                            {0.0, Ke / cns[3], rp},
                            {rho / cd[3], -rho / cds[3], 1.0}};
    const cplx R[3] = {Tp * st / cdp[3] - (Sn - Sd) * st / cd[3] + Ki * Sn / cn[3],
                       Tq * st / cdp[3] - (Sns - Sds) * st / cds[3] + Ke * Sns / cns[3],
                       rho * (Sd / cd[3] - Sds / cds[3])};
    const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                       M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                       M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    /* X by Cramer's rule: column 0 replaced by R */
    const cplx detX = R[0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                      M[0][1] * (R[1] * M[2][2] - M[1][2] * R[2]) +
                      M[0][2] * (R[1] * M[2][1] - M[1][1] * R[2]);
    return detX / det;
}

/* Coefficients of the general-angle rule by linearity: X for each unit input
 * in turn; A, B, C, D multiply a, b, p, q (the paper's A^i_j, B^i_j, C^i_j,
 * D^i_j of Eq. B3a).  d2q5 != 0 takes eps_D = 1/3, else 1/4. */
void lbm_oracle_angled_coefficients(double dl, double th, double kappa, double dt, double dx, int d2q5,
                                    double* A, double* B, double* C, double* D)
{
    double* out[4] = {A, B, C, D};
    for (int v = 0; v < 4; ++v)
        for (int j = 0; j < 3; ++j) {
            cplx in[4][3] = {{0}};
            in[v][j] = 1.0;
            out[v][j] = creal(angled_link(dl, th, kappa, dt, dx, d2q5 ? EPS_D2 : EPS_D, in[0], in[1], in[2], in[3]));
        }
}

/* Value of hat g_p at node (x, y, z) of the padded state, the node possibly
 * beyond periodic faces on several axes (a corner of the buffer layers):
 * the wrapped node times the wrap factor of each face crossed (Sec. 2.4.3).
 * Returns 0 if the node lies beyond a mirror face (not covered here). */
static int ghat_periodic(const cplx* gh, const grid_t* g, const int* bc, const cplx* wrap_lo, const cplx* wrap_hi,
                         int x, int y, int z, int p, cplx* out)
{
    int c[3] = {x, y, z};
    const int dims[3] = {g->nx, g->ny, g->nz};
    cplx f = 1.0;
    for (int a = 0; a < 3; ++a) {
        if (c[a] >= 0 && c[a] < dims[a]) continue;
        if (bc[a] != BC_PERIODIC) return 0;
        f *= c[a] < 0 ? wrap_lo[a] : wrap_hi[a];
        c[a] = (c[a] % dims[a] + dims[a]) % dims[a];
    }
    *out = f * gh[pidx(g, c[0], c[1], c[2]) * Q + p];
    return 1;
}

static int32_t label_periodic(const int32_t* labels, const grid_t* g, int x, int y, int z)
{
    int c[3] = {x, y, z};
    const int dims[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; ++a) c[a] = (c[a] % dims[a] + dims[a]) % dims[a];
    return labels[sidx(g, c[0], c[1], c[2])];
}

/* Scalar parameters as the oracle derives them: out = {tau, r, s}. */
void lbm_oracle_params(double D, double dt, double dx, double kappa, double* out)
{
    out[0] = tau_of(D, dt, dx, EPS_D);
    membrane_shares(kappa, dt, dx, EPS_D, &out[1], &out[2]);
}

/*
 * Membrane/phase mask, the oracle's own builder.  Encoding (shared contract
 * with the library, each side written independently):
 *   bit (i-1), i = 1..6: the link from x to its neighbour x + e_i is a
 *     membrane, i.e. that neighbour exists (a periodic wrap counts; a mirror
 *     face has no neighbour) and its compartment label differs from x's
 *     (half-link membranes on every label change, Sec. 2.4.2 with
 *     Delta_m = 0.5, theta = 0);
 *   bits 6-7: phase id phase_of_label[label[x]] (0..3).
 */
int lbm_oracle_mask(int nx, int ny, int nz, const int32_t* labels, int n_labels,
                    const uint8_t* phase_of_label, const int* bc, uint8_t* mask_out)
{
    grid_t g = {nx, ny, nz, nx + 2 * PAD, ny + 2 * PAD, nz + 2 * PAD};
    int dims[3] = {nx, ny, nz};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t s = sidx(&g, x, y, z);
                int32_t L = labels[s];
                if (L < 0 || L >= n_labels) return -1;
                if (phase_of_label[L] > 3) return -1;
                unsigned m = (unsigned)phase_of_label[L] << 6;
                for (int i = 1; i < Q; ++i) {
                    int c[3] = {x + EX[i], y + EY[i], z + EZ[i]};
                    int inside = 1;
                    for (int a = 0; a < 3; ++a) {
                        if (c[a] < 0 || c[a] >= dims[a]) {
                            if (bc[a] == BC_PERIODIC)
                                c[a] = (c[a] + dims[a]) % dims[a];
                            else
                                inside = 0;
                        }
                    }
                    if (!inside) continue;
                    if (labels[sidx(&g, c[0], c[1], c[2])] != L) m |= 1u << (i - 1);
                }
                mask_out[s] = (uint8_t)m;
            }
    return 0;
}

/*
 * Population i arriving at node x = (x, y, z) across the membrane on its
 * link to y = x - e_i by the general-angle rule (2-D): theta[x][ibar] gives
 * the membrane normal from x's compartment to y's as cos(theta) e_ibar +
 * sin(theta) e_perp, e_perp = +y for a link along x and +x for a link along y;
 * beta = sign(theta) e_perp.  The values at the membrane point x'_i = x'_e =
 * x_m = x + Delta_m e_ibar and at x'_ii = x_m - e_beta, x'_ee = x_m + e_beta
 * are extrapolated along the link, quadratically, from the three nearest
 * nodes of the same compartment: x, x + e_i, x + 2 e_i (shifted by -e_beta
 * for x'_ii) on x's side; y, y - e_i, y - 2 e_i (shifted by +e_beta for
 * x'_ee) on y's side.  Returns 0 (the caller keeps the theta = 0 rule) when
 * one of those nodes lies in another compartment or beyond a mirror face,
 * or an axis is shorter than 4 nodes.
 */
static int angled_arrival(const cplx* gh, const grid_t* g, const int* bc, const int32_t* labels,
                          const cplx* wlo, const cplx* whi, int x, int y, int z, int i, double dl, double th,
                          double kappa, double dt, double dx, double eps, cplx* out)
{
    if (g->nx < 4 || g->ny < 4) return 0;
    const int ib = OPP[i];
    const int ex = EX[i], ey = EY[i];
    int bet;                                      /* beta */
    if (ex != 0) bet = th > 0 ? 3 : 4;            /* link along x: beta = +-y */
    else bet = th > 0 ? 1 : 2;                    /* link along y: beta = +-x */
    const int bbar = OPP[bet];
    const int bx = EX[bet], by = EY[bet];
    const int32_t Lx = label_periodic(labels, g, x, y, z);
    const int32_t Le = label_periodic(labels, g, x - ex, y - ey, z);

    /* a: alpha = ibar at x and x_ii = x + e_i, abar = i at x;
     * b: abar = i at x_e = y and x_ee = y - e_i, alpha = ibar at y */
    const int na[6][3] = {{0, 0, ib}, {ex, ey, ib}, {0, 0, i}, {-ex, -ey, i}, {-2 * ex, -2 * ey, i}, {-ex, -ey, ib}};
    cplx v[6];
    for (int k = 0; k < 6; ++k)
        if (!ghat_periodic(gh, g, bc, wlo, whi, x + na[k][0], y + na[k][1], z, na[k][2], &v[k])) return 0;
    const cplx a3[3] = {v[0], v[1], v[2]}, b3[3] = {v[3], v[4], v[5]};

    /* Lagrange weights of the nodes at 0, 1, 2 steps for the point t steps
     * the other way: t = dl on x's side, 1 - dl on y's side */
    double wi[3], we[3];
    const double ti = dl, te = 1.0 - dl;
    wi[0] = (1.0 + ti) * (2.0 + ti) / 2.0; wi[1] = -ti * (2.0 + ti); wi[2] = ti * (1.0 + ti) / 2.0;
    we[0] = (1.0 + te) * (2.0 + te) / 2.0; we[1] = -te * (2.0 + te); we[2] = te * (1.0 + te) / 2.0;
    /* the six extrapolated values: {side (0 = x, 1 = y), shift along beta,
     * population}: p = (g_beta(x'_i), g_beta(x'_ii), g_bbar(x'_i)),
     * q = (g_bbar(x'_e), g_bbar(x'_ee), g_beta(x'_e)) */
    const int pts[6][3] = {{0, 0, bet}, {0, -1, bet}, {0, 0, bbar}, {1, 0, bbar}, {1, 1, bbar}, {1, 0, bet}};
    cplx pq[6];
    for (int k = 0; k < 6; ++k) {
        const int side = pts[k][0], sh = pts[k][1], pop = pts[k][2];
        cplx acc = 0;
        for (int m = 0; m < 3; ++m) {
            /* x side: x + m e_i; y side: y - m e_i = x - (1 + m) e_i */
            const int step = side ? -(1 + m) : m;
            const int nx_ = x + step * ex + sh * bx, ny_ = y + step * ey + sh * by;
            if (label_periodic(labels, g, nx_, ny_, z) != (side ? Le : Lx)) return 0;
            cplx u;
            if (!ghat_periodic(gh, g, bc, wlo, whi, nx_, ny_, z, pop, &u)) return 0;
            acc += (side ? we[m] : wi[m]) * u;
        }
        pq[k] = acc;
    }
    const cplx p3[3] = {pq[0], pq[1], pq[2]}, q3[3] = {pq[3], pq[4], pq[5]};
    *out = angled_link(dl, th, kappa, dt, dx, eps, a3, b3, p3, q3);
    return 1;
}

/*
 * One complete run from the initial condition M = 1 + 0i (Sec. 2.1) to
 * t = n_steps * dt.
 *
 * f[k] is the waveform sample used during step k (G(t^k) = G0 f(t^k),
 * Eq. reaction_LBM); the periodic phase uses F_k = sum_{m<k} f[m] dt
 * (Eq. periodic_phi).
 *
 * Outputs (each may be NULL):
 *   Z_out[2]          : sum over sites of M(x, t^K), K = n_steps (Re, Im);
 *   field_out[2N]     : M(x, t^K) per site (Re, Im interleaved);
 *   series_out[2K]    : sum over sites of M(x, t^{k+1}) after each step;
 *   state_out[2*7*N]  : g_i(x, t^K) per site, direction-major within a site.
 * Returns 0, or -1 on invalid input.
 */
static int run_impl(int nx, int ny, int nz, double dx,
                    const int32_t* labels, int n_labels, const uint8_t* phase_of_label,
                    const int* bc, int n_phases, const double* D, const double* T2,
                    double kappa, double dt, long n_steps, const double* f,
                    const double* gG, int n_threads, const double* delta, const double* theta, int substeps,
                    int d2q5, int classical, double* Z_out, double* field_out, double* series_out,
                    double* state_out)
{
    if (nx < 1 || ny < 1 || nz < 1 || dx <= 0 || dt <= 0 || n_steps < 0 || substeps < 1) return -1;
    if (classical && substeps != 1) return -1;   /* no reaction split to sub-step */
    if (d2q5 && nz != 1) return -1;
    if (theta && (!delta || !d2q5)) return -1;   /* the angle rule is the paper's 2-D one */
    const int nq = d2q5 ? 5 : Q;                  /* populations in use */
    const double eps = d2q5 ? EPS_D2 : EPS_D;
    const double* w = d2q5 ? W2 : W;
    if (n_phases < 1 || n_phases > 4) return -1;
    for (int a = 0; a < 3; ++a)
        if (bc[a] != BC_PERIODIC && bc[a] != BC_MIRROR) return -1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    grid_t g = {nx, ny, nz, nx + 2 * PAD, ny + 2 * PAD, nz + 2 * PAD};
    const int dims[3] = {nx, ny, nz};
    const size_t N = (size_t)nx * ny * nz;
    const size_t NP = (size_t)g.px * g.py * g.pz;

    for (size_t s = 0; s < N; ++s) {
        if (labels[s] < 0 || labels[s] >= n_labels) return -1;
        if (phase_of_label[labels[s]] >= n_phases) return -1;
    }

    /* Mirror BC with a gradient that is neither normal nor parallel to the
     * face is not covered by the paper (Sec. 2.4.4). */
    int mirror_conj[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        if (bc[a] != BC_MIRROR || gG[a] == 0.0) continue;
        for (int b = 0; b < 3; ++b)
            if (b != a && gG[b] != 0.0) return -1;
        mirror_conj[a] = 1;
    }

    double tau[4], decay[4];
    for (int p = 0; p < n_phases; ++p) {
        if (!(D[p] > 0.0)) return -1;
        tau[p] = tau_of(D[p], dt, dx, eps);
        decay[p] = exp(-dt / substeps / T2[p]); /* per reaction sub-step; T2 = inf -> 1 */
    }
    double r, s;
    membrane_shares(kappa, dt, dx, eps, &r, &s);
    if (delta)
        for (size_t i = 0; i < 6 * N; ++i)
            if (!(delta[i] > 0.0 && delta[i] < 1.0)) return -1;
    if (theta)
        for (size_t i = 0; i < 6 * N; ++i)
            if (!(fabs(theta[i]) < 1.5707963267948966)) return -1;

    cplx* gs = malloc(sizeof(cplx) * Q * N);     /* g_i(x, t^k)             */
    cplx* gh = malloc(sizeof(cplx) * Q * NP);    /* hat g_i with buffers    */
    int32_t* lab = malloc(sizeof(int32_t) * NP); /* labels with buffers     */
    uint8_t* ph = malloc(N);
    if (!gs || !gh || !lab || !ph) { free(gs); free(gh); free(lab); free(ph); return -1; }

    /* Labels of the buffer nodes (layers d = 0, 1 beyond each face):
     * periodic -> the wrapped node; mirror -> the node mirrored in the face
     * (Sec. 2.4.4: node -1-d mirrors node d, node N+d mirrors node N-1-d), so
     * a mirror face is never a membrane.  A layer deeper than the axis
     * (N = 1) repeats the mirrored/wrapped index modulo N. */
    for (size_t i = 0; i < NP; ++i) lab[i] = -1;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                lab[pidx(&g, x, y, z)] = labels[sidx(&g, x, y, z)];
                ph[sidx(&g, x, y, z)] = phase_of_label[labels[sidx(&g, x, y, z)]];
            }
    for (int a = 0; a < 3; ++a) {
        int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
        for (int d = 0; d < PAD; ++d)
            for (int u = 0; u < dims[o2]; ++u)
                for (int v = 0; v < dims[o1]; ++v) {
                    int lo[3], hi[3], slo[3], shi[3];
                    lo[a] = -1 - d; hi[a] = dims[a] + d;
                    lo[o1] = hi[o1] = slo[o1] = shi[o1] = v;
                    lo[o2] = hi[o2] = slo[o2] = shi[o2] = u;
                    if (bc[a] == BC_PERIODIC) {
                        slo[a] = ((dims[a] - 1 - d) % dims[a] + dims[a]) % dims[a];
                        shi[a] = d % dims[a];
                    } else {
                        slo[a] = d % dims[a];
                        shi[a] = ((dims[a] - 1 - d) % dims[a] + dims[a]) % dims[a];
                    }
                    lab[pidx(&g, lo[0], lo[1], lo[2])] = labels[sidx(&g, slo[0], slo[1], slo[2])];
                    lab[pidx(&g, hi[0], hi[1], hi[2])] = labels[sidx(&g, shi[0], shi[1], shi[2])];
                }
    }

    /* Initial condition M = 1 + 0i at equilibrium: g_i = omega_i M (Eq. g_eq). */
    for (size_t x = 0; x < N; ++x)
        for (int i = 0; i < Q; ++i) gs[x * Q + i] = w[i];   /* D2Q5: the z populations stay 0 */

    double F = 0.0; /* F_k = sum_{m<k} f_m dt */
    for (long k = 0; k < n_steps; ++k) {
        /* 1. Collision (Eq. collision_LBM), M = sum_i g_i (Eq. M'summation).
         *    Classical scheme (Eq. A12): plus the source dt omega_i R M with
         *    R = -i gamma x.G0 f(t^k) - 1/T2 (Eq. A2), x = n dx. */
#pragma omp parallel for
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t si = sidx(&g, x, y, z), pi = pidx(&g, x, y, z);
                    cplx M = 0;
                    for (int i = 0; i < nq; ++i) M += gs[si * Q + i];
                    double t = tau[ph[si]];
                    cplx R = 0;
                    if (classical) {
                        double xdotG = (x * dx) * gG[0] + (y * dx) * gG[1] + (z * dx) * gG[2];
                        R = -I * xdotG * f[k] - 1.0 / T2[ph[si]];   /* T2 = inf -> 0 */
                    }
                    for (int i = 0; i < nq; ++i) {
                        cplx gi = gs[si * Q + i];
                        gh[pi * Q + i] = gi - (gi - w[i] * M) / t;
                        if (classical) gh[pi * Q + i] += dt * w[i] * R * M;
                    }
                }

        /* Phase of the outer faces for this step's streaming.  Hybrid: the
         * streamed populations precede this step's reaction, F_k.  Classical:
         * the source of step k is already in them (they stand for t^(k+1)),
         * so F_(k+1) = F_k + f_k dt. */
        const double Fb = classical ? F + f[k] * dt : F;

        /* 2. Buffer layers (Sec. 2.4.3 Eq. collision_BC; Sec. 2.4.4). */
        for (int a = 0; a < 3; ++a) {
            int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
            double L = dims[a] * dx;
            double phi = gG[a] * L * Fb; /* Eq. periodic_phi, per axis */
            cplx wrap_lo = cexp(I * phi), wrap_hi = cexp(-I * phi);
            /* mirror, G normal to the face: hat g_i(x_m) =
             * conj( hat g_ibar(x_n) exp(i gamma (x_n + x_m - 2 x_o).G0 F) ),
             * origin x_o = 0 (where G0.x = 0). */
            double xlo = (0 + (-1)) * dx, xhi = ((dims[a] - 1) + dims[a]) * dx;
            cplx rot_lo = cexp(I * gG[a] * xlo * Fb), rot_hi = cexp(I * gG[a] * xhi * Fb);
            for (int d = 0; d < PAD; ++d)
            for (int u = 0; u < dims[o2]; ++u)
                for (int v = 0; v < dims[o1]; ++v) {
                    /* layer d: node -1-d and node N+d.  Periodic: images of
                     * nodes N-1-d and d.  Mirror: reflections of nodes d and
                     * N-1-d, whose x_n + x_m is -dx and (2N-1) dx for every d. */
                    int lo[3], hi[3], c0[3], cN[3];
                    lo[a] = -1 - d; hi[a] = dims[a] + d;
                    c0[a] = d % dims[a];
                    cN[a] = ((dims[a] - 1 - d) % dims[a] + dims[a]) % dims[a];
                    lo[o1] = hi[o1] = c0[o1] = cN[o1] = v;
                    lo[o2] = hi[o2] = c0[o2] = cN[o2] = u;
                    size_t plo = pidx(&g, lo[0], lo[1], lo[2]), phi_ = pidx(&g, hi[0], hi[1], hi[2]);
                    size_t p0 = pidx(&g, c0[0], c0[1], c0[2]), pN = pidx(&g, cN[0], cN[1], cN[2]);
                    for (int i = 0; i < nq; ++i) {
                        if (bc[a] == BC_PERIODIC) {
                            gh[plo * Q + i] = wrap_lo * gh[pN * Q + i];
                            gh[phi_ * Q + i] = wrap_hi * gh[p0 * Q + i];
                        } else {
                            int ri = reflect_dir(i, a);
                            if (mirror_conj[a]) {
                                gh[plo * Q + i] = conj(gh[p0 * Q + ri] * rot_lo);
                                gh[phi_ * Q + i] = conj(gh[pN * Q + ri] * rot_hi);
                            } else {
                                gh[plo * Q + i] = gh[p0 * Q + ri];
                                gh[phi_ * Q + i] = gh[pN * Q + ri];
                            }
                        }
                    }
                }
        }

        /* wrap factors of this step per axis (for the corner nodes of the
         * general-angle rule) */
        cplx wlo[3], whi[3];
        for (int a = 0; a < 3; ++a) {
            wlo[a] = cexp(I * gG[a] * dims[a] * dx * Fb);
            whi[a] = cexp(-I * gG[a] * dims[a] * dx * Fb);
        }

        /* 3. Streaming (Eq. streaming_LBM), with the half-link membrane rule
         *    on links whose end nodes carry different labels (Eqs. B2a_text,
         *    B2b_text with the B5 coefficients): the population arriving at x
         *    in direction i is s * (what streams in) + r * (what x sent out
         *    towards the membrane, reflected). */
        /* 4. Reaction (Eq. reaction_LBM), x_n = n dx, as `substeps` reaction
         *    steps of dt' = dt / substeps after the one diffusion step
         *    (Sec. 2.3: dt = k dt'), waveform sampled at the start of each. */
        const double dts = dt / substeps;
#pragma omp parallel for
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t si = sidx(&g, x, y, z), pi = pidx(&g, x, y, z);
                    int Lx = lab[pi];
                    cplx gbar[Q];
                    gbar[0] = gh[pi * Q + 0];
                    for (int i = 1; i < nq; ++i) {
                        size_t py_ = pidx(&g, x - EX[i], y - EY[i], z - EZ[i]);
                        if (lab[py_] == Lx) {
                            gbar[i] = gh[py_ * Q + i];
                            continue;
                        }
                        const int ib = OPP[i];   /* from x towards the membrane */
                        /* link-distance rule (Eqs. B4a-B4c): needs the node
                         * behind x (x + e_i) in x's compartment and the node
                         * beyond the far node (x - 2 e_i) in the far node's;
                         * otherwise, and for kappa = inf (no membrane), the
                         * half-link rule of Eq. B5 */
                        size_t pb = pidx(&g, x + EX[i], y + EY[i], z + EZ[i]);
                        size_t pe = pidx(&g, x - 2 * EX[i], y - 2 * EY[i], z - 2 * EZ[i]);
                        if (delta && !isinf(kappa) && lab[pb] == Lx && lab[pe] == lab[py_]) {
                            const double dl = delta[si * 6 + (ib - 1)];
                            const double th = theta ? theta[si * 6 + (ib - 1)] : 0.0;
                            if (th != 0.0 && angled_arrival(gh, &g, bc, labels, wlo, whi, x, y, z, i, dl, th, kappa,
                                                            dt, dx, eps, &gbar[i]))
                                continue;
                            double A[3], B[3];
                            link_coefficients(dl, kappa, dt, dx, eps, A, B);
                            gbar[i] = A[0] * gh[pi * Q + ib] + A[1] * gh[pb * Q + ib] + A[2] * gh[pi * Q + i] +
                                      B[0] * gh[py_ * Q + i] + B[1] * gh[pe * Q + i] + B[2] * gh[py_ * Q + ib];
                        } else {
                            gbar[i] = s * gh[py_ * Q + i] + r * gh[pi * Q + ib];
                        }
                    }
                    double xdotG = (x * dx) * gG[0] + (y * dx) * gG[1] + (z * dx) * gG[2];
                    for (int j = 0; j < substeps && !classical; ++j) {   /* 4. (hybrid only) */
                        cplx fac = cexp(-I * xdotG * f[k * substeps + j] * dts) * decay[ph[si]];
                        for (int i = 0; i < nq; ++i) gbar[i] = fac * gbar[i];
                    }
                    for (int i = 0; i < nq; ++i) gs[si * Q + i] = gbar[i];
                }
        for (int j = 0; j < substeps; ++j) F += f[k * substeps + j] * dts;

        if (series_out) {
            cplx Z = 0;
            for (size_t x = 0; x < N; ++x)
                for (int i = 0; i < Q; ++i) Z += gs[x * Q + i];
            series_out[2 * k] = creal(Z);
            series_out[2 * k + 1] = cimag(Z);
        }
    }

    /* 5. Signal: Z = sum_x M(x, t^K) (Sec. 2.1: S from the summed M). */
    cplx Z = 0;
    for (size_t x = 0; x < N; ++x) {
        cplx M = 0;
        for (int i = 0; i < Q; ++i) M += gs[x * Q + i];
        Z += M;
        if (field_out) { field_out[2 * x] = creal(M); field_out[2 * x + 1] = cimag(M); }
        if (state_out)
            for (int i = 0; i < Q; ++i) {
                state_out[2 * (x * Q + i)] = creal(gs[x * Q + i]);
                state_out[2 * (x * Q + i) + 1] = cimag(gs[x * Q + i]);
            }
    }
    if (Z_out) { Z_out[0] = creal(Z); Z_out[1] = cimag(Z); }
    free(gs); free(gh); free(lab); free(ph);
    return 0;
}

int lbm_oracle_run(int nx, int ny, int nz, double dx,
                   const int32_t* labels, int n_labels, const uint8_t* phase_of_label,
                   const int* bc, int n_phases, const double* D, const double* T2,
                   double kappa, double dt, long n_steps, const double* f,
                   const double* gG, int n_threads,
                   double* Z_out, double* field_out, double* series_out, double* state_out)
{
    return run_impl(nx, ny, nz, dx, labels, n_labels, phase_of_label, bc, n_phases, D, T2, kappa, dt, n_steps, f,
                    gG, n_threads, NULL, NULL, 1, 0, 0, Z_out, field_out, series_out, state_out);
}

/*
 * The same run with membranes at given positions on their links (theta = 0,
 * Eqs. B4a-B4c): delta[6*s + (j-1)], j = 1..6, is the distance, in units of
 * dx, from node s to the membrane on its link to the neighbour s + e_j
 * (0 < delta < 1; read only on membrane links).  A consistent input has
 * delta[s][j] = 1 - delta[s + e_j][jbar].
 */
int lbm_oracle_run_links(int nx, int ny, int nz, double dx,
                         const int32_t* labels, int n_labels, const uint8_t* phase_of_label,
                         const int* bc, int n_phases, const double* D, const double* T2,
                         double kappa, double dt, long n_steps, const double* f,
                         const double* gG, int n_threads, const double* delta,
                         double* Z_out, double* field_out, double* series_out, double* state_out)
{
    if (!delta) return -1;
    return run_impl(nx, ny, nz, dx, labels, n_labels, phase_of_label, bc, n_phases, D, T2, kappa, dt, n_steps, f,
                    gG, n_threads, delta, NULL, 1, 0, 0, Z_out, field_out, series_out, state_out);
}

/*
 * General form: optional membrane positions (as lbm_oracle_run_links, or
 * NULL), `substeps` >= 1 reaction steps of dt / substeps after each
 * diffusion step (Sec. 2.3, dt = k dt'; f then holds n_steps * substeps
 * samples on the dt' grid), d2q5 != 0 for the 2-D D2Q5 lattice of
 * Sec. 2.3 (nz = 1), and with it optional membrane angles theta[6*s + (j-1)]
 * (radians, |theta| < pi/2, read on membrane links with a position) for
 * the general-angle rule (angled_arrival); a consistent input has
 * theta[s][j] = -theta[s + e_j][jbar].
 */
int lbm_oracle_run_ex(int nx, int ny, int nz, double dx,
                      const int32_t* labels, int n_labels, const uint8_t* phase_of_label,
                      const int* bc, int n_phases, const double* D, const double* T2,
                      double kappa, double dt, long n_steps, const double* f,
                      const double* gG, int n_threads, const double* delta, const double* theta, int substeps,
                      int d2q5, double* Z_out, double* field_out, double* series_out, double* state_out)
{
    return run_impl(nx, ny, nz, dx, labels, n_labels, phase_of_label, bc, n_phases, D, T2, kappa, dt, n_steps, f,
                    gG, n_threads, delta, theta, substeps, d2q5, 0, Z_out, field_out, series_out, state_out);
}

/*
 * As lbm_oracle_run_ex, with `classical` != 0 selecting the classical LBM
 * of Appendix A (Eq. A12): the reaction enters the collision as the source
 * dt omega_i R M, R = -i gamma x.G0 f(t^k) - 1/T2, and there is no reaction
 * step (substeps must be 1).  The outer faces take F_(k+1) = sum_{m<=k} f_m dt
 * (see run_impl).
 */
int lbm_oracle_run_scheme(int nx, int ny, int nz, double dx,
                          const int32_t* labels, int n_labels, const uint8_t* phase_of_label,
                          const int* bc, int n_phases, const double* D, const double* T2,
                          double kappa, double dt, long n_steps, const double* f,
                          const double* gG, int n_threads, const double* delta, const double* theta, int substeps,
                          int d2q5, int classical, double* Z_out, double* field_out, double* series_out,
                          double* state_out)
{
    return run_impl(nx, ny, nz, dx, labels, n_labels, phase_of_label, bc, n_phases, D, T2, kappa, dt, n_steps, f,
                    gG, n_threads, delta, theta, substeps, d2q5, classical, Z_out, field_out, series_out,
                    state_out);
}
