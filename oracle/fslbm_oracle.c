/*
 * FP64 CPU oracle for one time step of the coupled free-surface lattice
 * Boltzmann / discrete-element method of Schwarzmeier et al., "Particle-
 * resolved simulation of antidunes in free-surface flows" (Section 2).
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. The GPU product path
 * never calls it and shares no code, header, table or helper with it.
 *
 * Design: plain and slow on purpose. Two PDF arrays (pull streaming), cell-
 * major storage f[cell*27+q], FP64 everywhere, no AA pattern, no worklists,
 * no fusion. Each function names the passage of the paper it follows; the
 * paper names the methods but prints none of their formulas, so every detail
 * it leaves open follows a stated reading (tags [R-n], listed in the design
 * notes of the repository).
 *
 * Step order (reading R-0; the state between steps is the post-collision
 * PDF field f*, the cell types, the interface mass m and fill level phi, the
 * interface normals, the particles and the FP64 mass pool):
 *   S1  stream with boundary conditions: halfway bounce-back at walls
 *       (Section 2.1), moving bounce-back + momentum exchange at particle
 *       links (Section 2.2), free-surface reconstruction at interface cells
 *       (Section 2.1: gas pressure boundary condition)
 *   S2  interface mass exchange
 *   S3  cumulant collision with gravity forcing (Section 2.1)
 *   S4  interface normals of the new fill levels (for S8 weights)
 *   S5  conversion candidates, S6 conflict rule, S7 fill/empty neighbours
 *   S8  excess-mass redistribution, S9 finalise cell types
 *   S10 hydrodynamic force averaging + DEM sub-steps (Section 2.2)
 *   S11 particle re-mapping: covered/uncovered cells (Section 2.2)
 *   S12 spread the mass pool over all interface cells
 *   S13 normals of the final fill levels (used by S1 of the next step)
 *
 * Parity status: the collision, streaming, free-surface boundary, mass
 * exchange, normals and DEM contact law are pinned by tests against closed
 * forms and invariants. The heuristic parts of the conversion (S5-S9) and
 * the re-mapping (S11) are pinned by the mass-conservation and
 * order-independence invariants and by hand-computed cases: the excess
 * shares, the new-interface and uncovered-cell states (orc_excess_shares,
 * orc_new_interface_mean, orc_uncovered_state on hand-built blocks) and
 * whole steps on flat layers at rest whose outcome is worked out by hand.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NQ 27

/* cell types (public convention of the exported type field) */
enum { T_GAS = 0, T_LIQ = 1, T_IFC = 2, T_SOL = 3 };
/* conversion marks (S5-S7) */
enum { CV_NONE = 0, CV_TO_LIQ = 1, CV_TO_GAS = 2 };
enum { MK_NONE = 0, MK_NEW = 1, MK_EMPTIED = 2 };

typedef struct {
    int nx, ny, nz;
    int periodic[3];          /* 1: periodic axis, 0: no-slip walls on both faces */
    double omega;             /* shear relaxation rate, nu = (1/omega - 1/2)/3 */
    double g[3];              /* body acceleration (gravity incl. slope forcing) */
    double rho_gas;           /* gas pressure p_g = rho_gas / 3 */
    double liquid_height;     /* initial free-surface height (cells) */
    double eps_conv;          /* conversion hysteresis epsilon (R-7) */
    double eps_normal;        /* n.c margin for normal-based reconstruction (R-5) */
    int reconstruct_normal;   /* 1: also rebuild directions with n.c < -eps_normal */
    double rho_p;             /* particle density (liquid reference density 1) */
    double restitution;       /* DEM coefficient of restitution e */
    double friction;          /* Coulomb friction coefficient mu */
    double poisson;           /* Poisson ratio nu_p */
    double collision_time;    /* DEM collision time T_c */
    int dem_substeps;         /* DEM sub-steps per LBM step */
    int link_mass_correction; /* 1: net moving-bounce-back injection into liquid
                                 cells is taken from the pool (R-12a) */
    double sigma;             /* surface tension: the gas-side reconstruction
                                 density is rho_gas + 6 sigma kappa (R-21) */
    int excess_even;          /* 1: excess mass split evenly over the receivers
                                 instead of by the normal weights (R-8 variant) */
    int lubrication;          /* 1: lubrication corrections below the resolved gap (R-23) */
    int galilean_correction;  /* 1: Galilean-invariance correction of the second-order
                                 rates (R-3 variant) */
} orc_params;

typedef struct {
    int partner;              /* particle index (>i) or -1-wall */
    double xi[3];             /* tangential spring displacement */
    int used;
} orc_hist;

#define MAX_HIST 48

typedef struct orc {
    orc_params p;
    long n;
    double *f, *ft;           /* post-collision state, scratch */
    uint8_t *type;
    double *mass, *rho, *u, *phi, *nrm;
    double *curv;             /* interface curvature of the learned model, 0 elsewhere */
    int *owner;
    double pool;
    long step;
    long invariant_violations;
    /* particles */
    int np;
    double *X, *U, *W, *R, *M, *I;
    uint8_t *fixed;
    double *Fh, *Th, *Fp, *Tp;
    int have_prev;
    orc_hist *hist;           /* np * MAX_HIST */
    double *fixmetric;        /* map of the fixed particles alone (static) */
    int *fixowner;
    double *mlp;              /* learned-normal parameters, NULL: Parker-Youngs */
    int mlp_bf16;             /* round products' operands to bfloat16 */
    int mlp_mirror;           /* average the network over the x and y mirror images */
} orc;

/* ---------------------------------------------------------------- tables */

static int CX[NQ], CY[NQ], CZ[NQ], OPP[NQ];
static double WQ[NQ];
static double MINV[NQ][NQ];   /* inverse of the raw-moment matrix at u = 0 */
static int tables_ready = 0;

static void build_tables(void)
{
    if (tables_ready) return;
    /* D3Q27 (Section 2.1): c in {-1,0,1}^3, index q = (cx+1)+3(cy+1)+9(cz+1).
     * Weights 8/27 (rest), 2/27 (faces), 1/54 (edges), 1/216 (corners). */
    for (int q = 0; q < NQ; ++q) {
        CX[q] = q % 3 - 1;
        CY[q] = (q / 3) % 3 - 1;
        CZ[q] = q / 9 - 1;
        int k = abs(CX[q]) + abs(CY[q]) + abs(CZ[q]);
        WQ[q] = k == 0 ? 8.0 / 27.0 : k == 1 ? 2.0 / 27.0 : k == 2 ? 1.0 / 54.0 : 1.0 / 216.0;
    }
    for (int q = 0; q < NQ; ++q)
        for (int r = 0; r < NQ; ++r)
            if (CX[r] == -CX[q] && CY[r] == -CY[q] && CZ[r] == -CZ[q]) OPP[q] = r;
    /* raw-moment matrix M[r][q] = cx^a cy^b cz^c, r = a + 3b + 9c; invert by
     * Gauss-Jordan elimination with partial pivoting. */
    double A[NQ][2 * NQ];
    for (int r = 0; r < NQ; ++r) {
        int a = r % 3, b = (r / 3) % 3, c = r / 9;
        for (int q = 0; q < NQ; ++q)
            A[r][q] = pow(CX[q], a) * pow(CY[q], b) * pow(CZ[q], c);
        for (int q = 0; q < NQ; ++q) A[r][NQ + q] = (r == q) ? 1.0 : 0.0;
    }
    for (int col = 0; col < NQ; ++col) {
        int piv = col;
        for (int r = col + 1; r < NQ; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int k = 0; k < 2 * NQ; ++k) {
                double t = A[col][k]; A[col][k] = A[piv][k]; A[piv][k] = t;
            }
        double d = A[col][col];
        for (int k = 0; k < 2 * NQ; ++k) A[col][k] /= d;
        for (int r = 0; r < NQ; ++r) {
            if (r == col) continue;
            double fac = A[r][col];
            if (fac == 0.0) continue;
            for (int k = 0; k < 2 * NQ; ++k) A[r][k] -= fac * A[col][k];
        }
    }
    for (int r = 0; r < NQ; ++r)
        for (int q = 0; q < NQ; ++q) MINV[r][q] = A[r][NQ + q];
    tables_ready = 1;
}

/* ------------------------------------------------------- local operators */

/* Second-order equilibrium w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2),
 * used by the free-surface reconstruction and by cell initialisation. */
void orc_feq(double rho, const double u[3], double feq[NQ])
{
    build_tables();
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int q = 0; q < NQ; ++q) {
        double cu = CX[q] * u[0] + CY[q] * u[1] + CZ[q] * u[2];
        feq[q] = WQ[q] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

static double ipow(double x, int k) { return k == 0 ? 1.0 : k == 1 ? x : x * x; }
static const double BINOM[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 2, 1}};

/* D3Q27 cumulant collision with all relaxation rates 1 except the shear rate
 * omega (Section 2.1, Geier et al. 2015 named there), with the body force
 * F = rho g applied by the half-shifted velocity and the sign flip of the
 * first-order central moments (R-2). Readings R-1/R-3: second-order shear
 * parts relax with omega, the trace relaxes with rate 1 to rho; all
 * cumulants of order >= 3 relax with rate 1 to zero, so the post-collision
 * central moments of orders 3..6 are those of rho * N(0, S), S = k2* / rho.
 * Moments are formed by direct summation and inverted through the raw-moment
 * matrix, without any per-axis (chimera) factorisation.
 *
 * With gal set, the Galilean-invariance correction of Geier et al. (2015) for
 * the second-order relaxation (reading R-3, off by default): the velocity
 * gradients follow from the non-equilibrium second-order moments,
 *   d_x u_x = -omega/(2 rho) (2 k_xx - k_yy - k_zz) - 1/(2 rho) (k_xx + k_yy + k_zz - rho),
 *   d_y u_y = d_x u_x + 3 omega/(2 rho) (k_xx - k_yy),
 *   d_z u_z = d_x u_x + 3 omega/(2 rho) (k_xx - k_zz),
 * (bulk rate 1), and the relaxed normal-stress differences and trace lose
 * 3 rho (1 - omega/2) (u_x^2 d_x u_x - u_y^2 d_y u_y), the same with z, and
 * 3 rho (1 - 1/2) (u_x^2 d_x u_x + u_y^2 d_y u_y + u_z^2 d_z u_z): the terms
 * of third order in u that the D3Q27 lattice (c^3 = c) puts into the
 * viscous stress. */
void orc_collide_gal(const double f[NQ], const double g[3], double omega, int gal, double out[NQ])
{
    build_tables();
    double rho = 0.0, j[3] = {0, 0, 0};
    for (int q = 0; q < NQ; ++q) {
        rho += f[q];
        j[0] += f[q] * CX[q];
        j[1] += f[q] * CY[q];
        j[2] += f[q] * CZ[q];
    }
    double F[3] = {rho * g[0], rho * g[1], rho * g[2]};
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / rho;

    double k[3][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int q = 0; q < NQ; ++q)
                    s += f[q] * ipow(CX[q] - u[0], a) * ipow(CY[q] - u[1], b) * ipow(CZ[q] - u[2], c);
                k[a][b][c] = s;
            }

    double kp[3][3][3];
    memset(kp, 0, sizeof(kp));
    kp[0][0][0] = rho;
    kp[1][0][0] = 0.5 * F[0];
    kp[0][1][0] = 0.5 * F[1];
    kp[0][0][1] = 0.5 * F[2];
    /* second order */
    double Dxy = k[2][0][0] - k[0][2][0];
    double Dxz = k[2][0][0] - k[0][0][2];
    double Dxy_s = (1.0 - omega) * Dxy;
    double Dxz_s = (1.0 - omega) * Dxz;
    double T_s = rho;
    if (gal) {
        double kxx = k[2][0][0], kyy = k[0][2][0], kzz = k[0][0][2];
        double dxu = -omega / (2.0 * rho) * (2.0 * kxx - kyy - kzz) - 1.0 / (2.0 * rho) * (kxx + kyy + kzz - rho);
        double dyv = dxu + 3.0 * omega / (2.0 * rho) * (kxx - kyy);
        double dzw = dxu + 3.0 * omega / (2.0 * rho) * (kxx - kzz);
        double ax = u[0] * u[0] * dxu, ay = u[1] * u[1] * dyv, az = u[2] * u[2] * dzw;
        Dxy_s -= 3.0 * rho * (1.0 - 0.5 * omega) * (ax - ay);
        Dxz_s -= 3.0 * rho * (1.0 - 0.5 * omega) * (ax - az);
        T_s -= 3.0 * rho * 0.5 * (ax + ay + az);
    }
    kp[2][0][0] = (Dxy_s + Dxz_s + T_s) / 3.0;
    kp[0][2][0] = (Dxz_s - 2.0 * Dxy_s + T_s) / 3.0;
    kp[0][0][2] = (Dxy_s - 2.0 * Dxz_s + T_s) / 3.0;
    kp[1][1][0] = (1.0 - omega) * k[1][1][0];
    kp[1][0][1] = (1.0 - omega) * k[1][0][1];
    kp[0][1][1] = (1.0 - omega) * k[0][1][1];
    /* Gaussian closure of orders 3..6 (odd orders vanish) */
    double Sxx = kp[2][0][0] / rho, Syy = kp[0][2][0] / rho, Szz = kp[0][0][2] / rho;
    double Sxy = kp[1][1][0] / rho, Sxz = kp[1][0][1] / rho, Syz = kp[0][1][1] / rho;
    kp[2][2][0] = rho * (Sxx * Syy + 2.0 * Sxy * Sxy);
    kp[2][0][2] = rho * (Sxx * Szz + 2.0 * Sxz * Sxz);
    kp[0][2][2] = rho * (Syy * Szz + 2.0 * Syz * Syz);
    kp[2][1][1] = rho * (Sxx * Syz + 2.0 * Sxy * Sxz);
    kp[1][2][1] = rho * (Syy * Sxz + 2.0 * Sxy * Syz);
    kp[1][1][2] = rho * (Szz * Sxy + 2.0 * Sxz * Syz);
    kp[2][2][2] = rho * (Sxx * Syy * Szz
                         + 2.0 * (Sxx * Syz * Syz + Syy * Sxz * Sxz + Szz * Sxy * Sxy)
                         + 8.0 * Sxy * Sxz * Syz);

    /* central -> raw moments (binomial theorem), raw moments -> PDFs */
    double m[NQ];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int pa = 0; pa <= a; ++pa)
                    for (int pb = 0; pb <= b; ++pb)
                        for (int pc = 0; pc <= c; ++pc)
                            s += BINOM[a][pa] * BINOM[b][pb] * BINOM[c][pc]
                                 * ipow(u[0], a - pa) * ipow(u[1], b - pb) * ipow(u[2], c - pc)
                                 * kp[pa][pb][pc];
                m[a + 3 * b + 9 * c] = s;
            }
    for (int q = 0; q < NQ; ++q) {
        double s = 0.0;
        for (int r = 0; r < NQ; ++r) s += MINV[q][r] * m[r];
        out[q] = s;
    }
}

void orc_collide(const double f[NQ], const double g[3], double omega, double out[NQ])
{
    orc_collide_gal(f, g, omega, 0, out);
}

/* ------------------------------------------------------------ geometry */

static long cidx(const orc* o, int x, int y, int z)
{
    return (long)x + (long)o->p.nx * ((long)y + (long)o->p.ny * (long)z);
}

/* Neighbour of (x,y,z) at offset d: returns the cell index, or -1 when the
 * neighbour lies beyond a wall face (non-periodic axis). */
static long nbr(const orc* o, int x, int y, int z, int dx, int dy, int dz)
{
    int c[3] = {x + dx, y + dy, z + dz};
    int L[3] = {o->p.nx, o->p.ny, o->p.nz};
    for (int a = 0; a < 3; ++a) {
        if (c[a] < 0 || c[a] >= L[a]) {
            if (!o->p.periodic[a]) return -1;
            c[a] = (c[a] + L[a]) % L[a];
        }
    }
    return cidx(o, c[0], c[1], c[2]);
}

static void coords(const orc* o, long i, int* x, int* y, int* z)
{
    *x = (int)(i % o->p.nx);
    *y = (int)((i / o->p.nx) % o->p.ny);
    *z = (int)(i / ((long)o->p.nx * o->p.ny));
}

static int is_fluid(int t) { return t == T_LIQ || t == T_IFC; }

/* minimal-image component of a displacement along axis a */
static double min_image(const orc* o, int a, double d)
{
    int L[3] = {o->p.nx, o->p.ny, o->p.nz};
    if (o->p.periodic[a]) d -= L[a] * floor(d / L[a] + 0.5);
    return d;
}

/* velocity of the cell's most recent collision, recovered from its post-
 * collision PDFs: u = (sum c f* - rho g / 2) / rho  (R-4) */
static void post_velocity(const orc* o, const double* fs, double* rho_out, double u[3])
{
    double r = 0, j[3] = {0, 0, 0};
    for (int q = 0; q < NQ; ++q) {
        r += fs[q];
        j[0] += CX[q] * fs[q];
        j[1] += CY[q] * fs[q];
        j[2] += CZ[q] * fs[q];
    }
    for (int a = 0; a < 3; ++a) u[a] = (j[a] - 0.5 * r * o->p.g[a]) / r;
    *rho_out = r;
}

/* surface velocity of particle p at point x (minimal image) */
static void particle_velocity_at(const orc* o, int p, const double x[3], double ub[3])
{
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = min_image(o, a, x[a] - o->X[3 * p + a]);
    const double* w = &o->W[3 * p];
    ub[0] = o->U[3 * p + 0] + (w[1] * d[2] - w[2] * d[1]);
    ub[1] = o->U[3 * p + 1] + (w[2] * d[0] - w[0] * d[2]);
    ub[2] = o->U[3 * p + 2] + (w[0] * d[1] - w[1] * d[0]);
}

/* ------------------------------------------ conversion heuristics (R-7, R-8, R-11)
 * Each works on the 3x3x3 block around one cell, index q = (cx+1) +
 * 3(cy+1) + 9(cz+1) (13 is the cell itself), with the cell types of the
 * snapshot taken before the conversion; NB_WALL marks a block position
 * beyond a wall face. one_step calls them; the tests call them on blocks
 * built by hand. */
#define NB_WALL 255

/* Excess mass of an interface cell that converts (Section 2.1, R-8): ex is
 * shared among the receivers (recv[q] != 0, q != 13) with weights
 * max(0, s n.c_q), s = +1 for a cell turning liquid and -1 for one turning
 * gas, n the cell's normal toward the gas; evenly over the receivers when
 * every weight vanishes or `even` is set. share[q] gets each part (0 for
 * the others). Returns 1, with every share 0, when there is no receiver:
 * the excess then belongs to the global pool. */
int orc_excess_shares(int to_liquid, double ex, const double n[3], const uint8_t recv[NQ], int even,
                      double share[NQ])
{
    build_tables();
    double sgn = to_liquid ? 1.0 : -1.0;
    double w[NQ], wsum = 0.0;
    int nrec = 0;
    for (int q = 0; q < NQ; ++q) {
        share[q] = 0.0;
        w[q] = 0.0;
        if (q == 13 || !recv[q]) continue;
        double v = sgn * (n[0] * CX[q] + n[1] * CY[q] + n[2] * CZ[q]);
        if (v < 0.0) v = 0.0;
        w[q] = v;
        wsum += v;
        nrec++;
    }
    if (nrec == 0) return 1;
    for (int q = 0; q < NQ; ++q) {
        if (q == 13 || !recv[q]) continue;
        share[q] = (wsum > 0.0 && !even) ? ex * w[q] / wsum : ex / nrec;
    }
    return 0;
}

/* Start of a gas cell that turns interface next to a filled cell (Section
 * 2.1, R-7): the mean density and velocity over the block's liquid and
 * interface cells (q != 13; type[q] from the snapshot, u[3q..3q+2]). The new
 * cell then holds f_eq(rho_bar, u_bar) and mass 0. Returns the number of
 * cells averaged; with none, nothing is written. */
int orc_new_interface_mean(const uint8_t type[NQ], const double rho[NQ], const double u[3 * NQ], double* rb,
                           double ub[3])
{
    double rs = 0, us[3] = {0, 0, 0};
    int cnt = 0;
    for (int q = 0; q < NQ; ++q) {
        if (q == 13 || !is_fluid(type[q])) continue;
        rs += rho[q];
        for (int a = 0; a < 3; ++a) us[a] += u[3 * q + a];
        cnt++;
    }
    if (cnt == 0) return 0;
    *rb = rs / cnt;
    for (int a = 0; a < 3; ++a) ub[a] = us[a] / cnt;
    return cnt;
}

/* State of a cell that a particle uncovers (Section 2.2, R-11), from the
 * snapshot of its block: without a liquid or interface neighbour it turns
 * gas (returns T_GAS, nothing else written); otherwise it takes
 * f_eq(rho_bar, u_b), rho_bar the mean density of those neighbours and u_b
 * = U_p + Omega_p x d the particle's surface velocity at the cell centre
 * (d = x_c - X_p, minimal image), and becomes interface with mass 0 if a
 * neighbour is gas, liquid with mass rho_bar otherwise. The mass it holds is
 * taken from the pool by the caller. */
int orc_uncovered_state(const uint8_t type[NQ], const double rho[NQ], const double Up[3], const double Wp[3],
                        const double d[3], double f[NQ], double* rb, double ub[3], double* mass)
{
    double rs = 0.0;
    int cnt = 0, gas = 0;
    for (int q = 0; q < NQ; ++q) {
        if (q == 13 || type[q] == NB_WALL) continue;
        if (is_fluid(type[q])) { rs += rho[q]; cnt++; }
        if (type[q] == T_GAS) gas = 1;
    }
    if (cnt == 0) return T_GAS;
    *rb = rs / cnt;
    ub[0] = Up[0] + (Wp[1] * d[2] - Wp[2] * d[1]);
    ub[1] = Up[1] + (Wp[2] * d[0] - Wp[0] * d[2]);
    ub[2] = Up[2] + (Wp[0] * d[1] - Wp[1] * d[0]);
    orc_feq(*rb, ub, f);
    *mass = gas ? 0.0 : *rb;
    return gas ? T_IFC : T_LIQ;
}

/* Parker-Youngs normal (R-10): gradient sum_c w(c) c phi(x+c), weights 4
 * (face), 2 (edge), 1 (corner); wall and solid neighbours take the centre
 * value. Returns n = -grad/|grad| (pointing toward the gas), zero if the
 * gradient vanishes. */
static void pyn_normal(const orc* o, long cell, const double* phi, double n[3])
{
    int x, y, z;
    coords(o, cell, &x, &y, &z);
    double g[3] = {0, 0, 0};
    double c0 = phi[cell];
    for (int q = 0; q < NQ; ++q) {
        int k = abs(CX[q]) + abs(CY[q]) + abs(CZ[q]);
        if (k == 0) continue;
        double w = k == 1 ? 4.0 : k == 2 ? 2.0 : 1.0;
        long nb = nbr(o, x, y, z, CX[q], CY[q], CZ[q]);
        double v = (nb < 0 || o->type[nb] == T_SOL) ? c0 : phi[nb];
        g[0] += w * CX[q] * v;
        g[1] += w * CY[q] * v;
        g[2] += w * CZ[q] * v;
    }
    double len = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (len > 0.0) {
        n[0] = -g[0] / len; n[1] = -g[1] / len; n[2] = -g[2] / len;
    } else {
        n[0] = n[1] = n[2] = 0.0;
    }
}

/* Learned normal (R-17): a 27-64-64-4 perceptron with ReLU maps the fill
 * levels of the 3x3x3 block (clamped to [0,1]) to a raw normal and the
 * curvature. Parameter layout: W1 (64x27), b1, W2 (64x64), b2, W3 (4x64),
 * b3, matrices row-major (out, in). The finite-difference normal stands in
 * when a wall or solid cell lies in the block, when the raw normal's length
 * is outside [1/2, 2], or when the two normals are more than 30 degrees
 * apart. With mlp_bf16 the operands of every product (weights, inputs,
 * hidden activations) are rounded to bfloat16 first, as on tensor cores,
 * so that the fallback decisions are taken on the same values; sums and
 * biases stay FP64. */
#define MLP_NPARAM 6212
static double bf16_round(double a)
{
    if (a == 0.0 || !isfinite(a)) return a;
    int e;
    double m = frexp(a, &e);               /* a = m 2^e, |m| in [1/2, 1) */
    return ldexp(nearbyint(ldexp(m, 8)), e - 8);
}

/* Raw network output (n_x, n_y, n_z, curvature) of one stencil of operand
 * values */
static void mlp_raw(const orc* o, const double in[NQ], double out[4])
{
    const double *W1 = o->mlp, *b1 = W1 + 64 * 27, *W2 = b1 + 64, *b2 = W2 + 64 * 64, *W3 = b2 + 64,
                 *b3 = W3 + 4 * 64;
    const int r = o->mlp_bf16;
    double h1[64], h2[64];
    for (int j = 0; j < 64; ++j) {
        double a = b1[j];
        for (int i = 0; i < NQ; ++i) a += W1[j * 27 + i] * in[i];
        h1[j] = a > 0.0 ? (r ? bf16_round(a) : a) : 0.0;
    }
    for (int j = 0; j < 64; ++j) {
        double a = b2[j];
        for (int i = 0; i < 64; ++i) a += W2[j * 64 + i] * h1[i];
        h2[j] = a > 0.0 ? (r ? bf16_round(a) : a) : 0.0;
    }
    for (int k = 0; k < 4; ++k) {
        double a = b3[k];
        for (int i = 0; i < 64; ++i) a += W3[k * 64 + i] * h2[i];
        out[k] = a;
    }
}

/* Stencil index q = (cx+1) + 3(cy+1) + 9(cz+1) under the mirror images of
 * R-17g: bit 0 of m reverses x, bit 1 reverses y */
static int mirror_q(int q, int m)
{
    int a = q % 3, b = (q / 3) % 3, c = q / 9;
    if (m & 1) a = 2 - a;
    if (m & 2) b = 2 - b;
    return a + 3 * b + 9 * c;
}

static void mlp_normal(const orc* o, long cell, const double* phi, double n[3], double* kappa)
{
    int x, y, z;
    coords(o, cell, &x, &y, &z);
    double in[NQ];
    int bad = 0;
    for (int q = 0; q < NQ; ++q) {
        long nb = nbr(o, x, y, z, CX[q], CY[q], CZ[q]);
        if (nb < 0 || o->type[nb] == T_SOL) { bad = 1; in[q] = 0.0; continue; }
        double v = phi[nb];
        in[q] = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
    }
    double fd[3];
    pyn_normal(o, cell, phi, fd);
    n[0] = fd[0]; n[1] = fd[1]; n[2] = fd[2];
    if (bad) return;
    /* o->mlp already holds the operand values (weights rounded at set-up
     * when mlp_bf16); inputs and hidden activations are rounded here */
    if (o->mlp_bf16)
        for (int i = 0; i < NQ; ++i) in[i] = bf16_round(in[i]);
    double out[4];
    mlp_raw(o, in, out);
    if (o->mlp_mirror) {
        /* R-17g: the network on the stencil mirrored in x, in y and in both
         * (value at q taken from the mirrored index), each output mapped
         * back (the mirrored components change sign), and the four averaged */
        for (int m = 1; m < 4; ++m) {
            double im[NQ], ym[4];
            for (int q = 0; q < NQ; ++q) im[q] = in[mirror_q(q, m)];
            mlp_raw(o, im, ym);
            out[0] += (m & 1) ? -ym[0] : ym[0];
            out[1] += (m & 2) ? -ym[1] : ym[1];
            out[2] += ym[2];
            out[3] += ym[3];
        }
        for (int k = 0; k < 4; ++k) out[k] *= 0.25;
    }
    double len = sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
    if (!(len >= 0.5 && len <= 2.0)) return;
    double m[3] = {out[0] / len, out[1] / len, out[2] / len};
    if (m[0] * fd[0] + m[1] * fd[1] + m[2] * fd[2] < 0.8660254037844386) return;   /* cos 30 deg */
    n[0] = m[0]; n[1] = m[1]; n[2] = m[2];
    if (kappa) *kappa = out[3];
}

/* Interface normal, and (kappa not NULL) the curvature: the learned model's
 * where its normal is taken, 0 where the finite-difference normal stands */
static void normal_at(const orc* o, long cell, const double* phi, double n[3], double* kappa)
{
    if (kappa) *kappa = 0.0;
    if (o->mlp) mlp_normal(o, cell, phi, n, kappa);
    else pyn_normal(o, cell, phi, n);
}

/* Parker-Youngs normal of a bare 3x3x3 fill stencil (index q as above), used
 * by tests; all 27 values are taken as given. */
void orc_normal_stencil(const double phi27[NQ], double n[3])
{
    build_tables();
    double g[3] = {0, 0, 0};
    for (int q = 0; q < NQ; ++q) {
        int k = abs(CX[q]) + abs(CY[q]) + abs(CZ[q]);
        if (k == 0) continue;
        double w = k == 1 ? 4.0 : k == 2 ? 2.0 : 1.0;
        g[0] += w * CX[q] * phi27[q];
        g[1] += w * CY[q] * phi27[q];
        g[2] += w * CZ[q] * phi27[q];
    }
    double len = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (len > 0.0) { n[0] = -g[0] / len; n[1] = -g[1] / len; n[2] = -g[2] / len; }
    else n[0] = n[1] = n[2] = 0.0;
}

static void refresh_phi(orc* o, long i)
{
    switch (o->type[i]) {
    case T_LIQ: o->phi[i] = 1.0; break;
    case T_IFC: o->phi[i] = o->mass[i] / o->rho[i]; break;
    default: o->phi[i] = 0.0; break;
    }
}

/* ------------------------------------------------------ life cycle */

orc* orc_create(const orc_params* p)
{
    build_tables();
    orc* o = (orc*)calloc(1, sizeof(orc));
    o->p = *p;
    o->n = (long)p->nx * p->ny * p->nz;
    long n = o->n;
    o->f = (double*)calloc((size_t)n * NQ, sizeof(double));
    o->ft = (double*)calloc((size_t)n * NQ, sizeof(double));
    o->type = (uint8_t*)calloc((size_t)n, 1);
    o->mass = (double*)calloc((size_t)n, sizeof(double));
    o->rho = (double*)calloc((size_t)n, sizeof(double));
    o->u = (double*)calloc((size_t)n * 3, sizeof(double));
    o->phi = (double*)calloc((size_t)n, sizeof(double));
    o->nrm = (double*)calloc((size_t)n * 3, sizeof(double));
    o->curv = (double*)calloc((size_t)n, sizeof(double));
    o->owner = (int*)malloc((size_t)n * sizeof(int));
    for (long i = 0; i < n; ++i) o->owner[i] = -1;

    /* R-15: initial surface. fill(k) = clamp(H - k, 0, 1); gas where the
     * fill is 0, interface where 0 < fill < 1 or where a full cell has gas
     * directly above; hydrostatic density rho = rho_gas exp(3|g_z|(H - z_c))
     * so that the liquid pressure equals the gas pressure at the surface
     * (Section 3.1); velocity zero; f* = f_eq(rho, 0). */
    double H = p->liquid_height;
    for (long i = 0; i < n; ++i) {
        int x, y, z;
        coords(o, i, &x, &y, &z);
        double fk = H - z;
        fk = fk < 0 ? 0 : (fk > 1 ? 1 : fk);
        double fa = H - (z + 1);
        fa = fa < 0 ? 0 : (fa > 1 ? 1 : fa);
        int above_gas = (z + 1 < p->nz) ? (fa == 0.0) : (p->periodic[2] ? (H - 0 <= 0) : 0);
        uint8_t t;
        if (fk == 0.0) t = T_GAS;
        else if (fk < 1.0 || above_gas) t = T_IFC;
        else t = T_LIQ;
        o->type[i] = t;
        if (t != T_GAS) {
            double zc = z + 0.5;
            double r = p->rho_gas * exp(3.0 * fabs(p->g[2]) * (H - zc));
            if (p->g[2] == 0.0) r = p->rho_gas;
            double u0[3] = {0, 0, 0};
            orc_feq(r, u0, &o->f[i * NQ]);
            o->rho[i] = r;
            o->mass[i] = r * fk;
        }
        refresh_phi(o, i);
    }
    for (long i = 0; i < n; ++i)
        if (o->type[i] == T_IFC) normal_at(o, i, o->phi, &o->nrm[3 * i], &o->curv[i]);
    return o;
}

/* Re-initialises the fluid from a free-surface height per column, H[y*nx+x]
 * (R-15 applied column by column): fill(k) = clamp(H - k, 0, 1); gas where
 * the fill is 0; liquid where it is 1 and no 26-neighbour is gas; interface
 * otherwise; hydrostatic density from the column's own surface height. Solid
 * cells are left untouched. */
int orc_init_surface(orc* o, const double* H)
{
    const orc_params* p = &o->p;
    long n = o->n;
    double* fill = (double*)malloc(sizeof(double) * n);
    for (long i = 0; i < n; ++i) {
        int x, y, z;
        coords(o, i, &x, &y, &z);
        double fk = H[(long)y * p->nx + x] - z;
        fill[i] = fk < 0 ? 0 : (fk > 1 ? 1 : fk);
    }
    for (long i = 0; i < n; ++i) {
        if (o->type[i] == T_SOL) continue;
        int x, y, z;
        coords(o, i, &x, &y, &z);
        uint8_t t;
        if (fill[i] == 0.0) t = T_GAS;
        else {
            int gas_nb = 0;
            for (int q = 0; q < NQ; ++q) {
                if (q == 13) continue;
                long nb = nbr(o, x, y, z, CX[q], CY[q], CZ[q]);
                if (nb >= 0 && o->type[nb] != T_SOL && fill[nb] == 0.0) gas_nb = 1;
            }
            t = (fill[i] < 1.0 || gas_nb) ? T_IFC : T_LIQ;
        }
        o->type[i] = t;
        o->mass[i] = 0.0;
        if (t != T_GAS) {
            double r = p->rho_gas * exp(3.0 * fabs(p->g[2]) * (H[(long)y * p->nx + x] - (z + 0.5)));
            double u0[3] = {0, 0, 0};
            orc_feq(r, u0, &o->f[i * NQ]);
            o->rho[i] = r;
            o->u[3 * i] = o->u[3 * i + 1] = o->u[3 * i + 2] = 0.0;
            o->mass[i] = r * fill[i];
        }
        refresh_phi(o, i);
    }
    for (long i = 0; i < n; ++i) {
        if (o->type[i] == T_IFC) normal_at(o, i, o->phi, &o->nrm[3 * i], &o->curv[i]);
        else o->nrm[3 * i] = o->nrm[3 * i + 1] = o->nrm[3 * i + 2] = o->curv[i] = 0.0;
    }
    free(fill);
    return 0;
}

void orc_destroy(orc* o)
{
    if (!o) return;
    free(o->f); free(o->ft); free(o->type); free(o->mass); free(o->rho); free(o->u);
    free(o->phi); free(o->nrm); free(o->curv); free(o->owner);
    free(o->X); free(o->U); free(o->W); free(o->R); free(o->M); free(o->I); free(o->fixed);
    free(o->Fh); free(o->Th); free(o->Fp); free(o->Tp); free(o->hist);
    free(o->fixmetric); free(o->fixowner); free(o->mlp);
    free(o);
}

/* Selects the learned normal (theta: MLP_NPARAM values in the layout above;
 * NULL restores Parker-Youngs) and recomputes the interface normals. */
int orc_set_mlp(orc* o, const double* theta, int bf16)
{
    free(o->mlp);
    o->mlp = NULL;
    if (theta) {
        o->mlp = (double*)malloc(sizeof(double) * MLP_NPARAM);
        if (!o->mlp) return -1;
        memcpy(o->mlp, theta, sizeof(double) * MLP_NPARAM);
        if (bf16) {   /* weight matrices to their operand values; biases stay */
            for (int i = 0; i < MLP_NPARAM; ++i) {
                int is_bias = (i >= 64 * 27 && i < 64 * 27 + 64) ||
                              (i >= 64 * 27 + 64 + 64 * 64 && i < 64 * 27 + 64 + 64 * 64 + 64) || i >= 6208;
                if (!is_bias) o->mlp[i] = bf16_round(o->mlp[i]);
            }
        }
    }
    o->mlp_bf16 = bf16;
    for (long i = 0; i < o->n; ++i)
        if (o->type[i] == T_IFC) normal_at(o, i, o->phi, &o->nrm[3 * i], &o->curv[i]);
    return 0;
}

/* Mirror averaging of the learned normal (R-17g): on = 1 averages the
 * network over the stencil and its mirror images in x, y and both; the
 * interface normals are recomputed when a network is set. */
int orc_set_mlp_mirror(orc* o, int on)
{
    o->mlp_mirror = on != 0;
    if (o->mlp)
        for (long i = 0; i < o->n; ++i)
            if (o->type[i] == T_IFC) normal_at(o, i, o->phi, &o->nrm[3 * i], &o->curv[i]);
    return 0;
}

/* Map of the particles onto the grid (Section 2.2, R-11): a cell is solid
 * iff |x_c - X_p|^2 <= r_p^2 (minimal image, evaluated without fused
 * multiply-add); overlapping spheres: the smallest |x_c - X|^2 - r^2 wins,
 * ties go to the lowest index. Writes the new owner of every cell. */
static void map_particles(const orc* o, int want_fixed, double* best, int* newowner)
{
    int L[3] = {o->p.nx, o->p.ny, o->p.nz};
    for (int p = 0; p < o->np; ++p) {
        if ((o->fixed[p] != 0) != (want_fixed != 0)) continue;
        double r = o->R[p];
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            double X = o->X[3 * p + a];
            lo[a] = (int)floor(X - r - 0.5);
            hi[a] = (int)ceil(X + r - 0.5);
            if (!o->p.periodic[a]) {
                if (lo[a] < 0) lo[a] = 0;
                if (hi[a] > L[a] - 1) hi[a] = L[a] - 1;
            }
        }
        for (int kz = lo[2]; kz <= hi[2]; ++kz)
            for (int ky = lo[1]; ky <= hi[1]; ++ky)
                for (int kx = lo[0]; kx <= hi[0]; ++kx) {
                    double dx = (kx + 0.5) - o->X[3 * p + 0];
                    double dy = (ky + 0.5) - o->X[3 * p + 1];
                    double dz = (kz + 0.5) - o->X[3 * p + 2];
                    double metric = ((dx * dx + dy * dy) + dz * dz) - r * r;
                    if (metric > 0.0) continue;
                    int cx = ((kx % L[0]) + L[0]) % L[0];
                    int cy = ((ky % L[1]) + L[1]) % L[1];
                    int cz = ((kz % L[2]) + L[2]) % L[2];
                    long c = cidx(o, cx, cy, cz);
                    if (metric < best[c] || (metric == best[c] && p < newowner[c])) {
                        best[c] = metric;
                        newowner[c] = p;
                    }
                }
    }
}

/* Fixed particles never move, so their part of the map is computed once. */
static void compute_map(const orc* o, int* newowner)
{
    long n = o->n;
    double* best = (double*)malloc((size_t)n * sizeof(double));
    for (long i = 0; i < n; ++i) { best[i] = o->fixmetric[i]; newowner[i] = o->fixowner[i]; }
    map_particles(o, 0, best, newowner);
    free(best);
}

int orc_add_spheres(orc* o, int n, const double* xyz, const double* radius, const uint8_t* fixed)
{
    int np = o->np + n;
    o->X = (double*)realloc(o->X, sizeof(double) * 3 * np);
    o->U = (double*)realloc(o->U, sizeof(double) * 3 * np);
    o->W = (double*)realloc(o->W, sizeof(double) * 3 * np);
    o->Fh = (double*)realloc(o->Fh, sizeof(double) * 3 * np);
    o->Th = (double*)realloc(o->Th, sizeof(double) * 3 * np);
    o->Fp = (double*)realloc(o->Fp, sizeof(double) * 3 * np);
    o->Tp = (double*)realloc(o->Tp, sizeof(double) * 3 * np);
    o->R = (double*)realloc(o->R, sizeof(double) * np);
    o->M = (double*)realloc(o->M, sizeof(double) * np);
    o->I = (double*)realloc(o->I, sizeof(double) * np);
    o->fixed = (uint8_t*)realloc(o->fixed, np);
    o->hist = (orc_hist*)realloc(o->hist, sizeof(orc_hist) * MAX_HIST * np);
    for (int k = 0; k < n; ++k) {
        int p = o->np + k;
        for (int a = 0; a < 3; ++a) {
            o->X[3 * p + a] = xyz[3 * k + a];
            o->U[3 * p + a] = o->W[3 * p + a] = 0.0;
            o->Fh[3 * p + a] = o->Th[3 * p + a] = o->Fp[3 * p + a] = o->Tp[3 * p + a] = 0.0;
        }
        double r = radius[k];
        o->R[p] = r;
        o->M[p] = o->p.rho_p * (4.0 / 3.0) * M_PI * r * r * r;
        o->I[p] = 0.4 * o->M[p] * r * r;
        o->fixed[p] = fixed ? fixed[k] : 0;
        memset(&o->hist[(size_t)MAX_HIST * p], 0, sizeof(orc_hist) * MAX_HIST);
    }
    o->np = np;
    if (!o->fixmetric) {
        o->fixmetric = (double*)malloc(sizeof(double) * o->n);
        o->fixowner = (int*)malloc(sizeof(int) * o->n);
    }
    for (long i = 0; i < o->n; ++i) { o->fixmetric[i] = INFINITY; o->fixowner[i] = -1; }
    map_particles(o, 1, o->fixmetric, o->fixowner);
    int* own = (int*)malloc(sizeof(int) * o->n);
    compute_map(o, own);
    for (long i = 0; i < o->n; ++i) {
        if (own[i] >= 0) {
            o->type[i] = T_SOL;
            o->owner[i] = own[i];
            o->mass[i] = 0.0;
            o->phi[i] = 0.0;
        }
    }
    free(own);
    for (long i = 0; i < o->n; ++i)
        if (o->type[i] == T_IFC) normal_at(o, i, o->phi, &o->nrm[3 * i], &o->curv[i]);
    return 0;
}

/* ------------------------------------------------------------- DEM */

static orc_hist* hist_find(orc* o, int i, int partner, int create)
{
    orc_hist* h = &o->hist[(size_t)MAX_HIST * i];
    for (int s = 0; s < MAX_HIST; ++s)
        if (h[s].used && h[s].partner == partner) return &h[s];
    if (!create) return NULL;
    for (int s = 0; s < MAX_HIST; ++s)
        if (!h[s].used) {
            h[s].used = 1; h[s].partner = partner;
            h[s].xi[0] = h[s].xi[1] = h[s].xi[2] = 0.0;
            return &h[s];
        }
    return NULL;
}

static void cross(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Linear spring-dashpot contact (Section 2.2 parameterisation, R-13):
 * k_n = m_eff (pi^2 + ln^2 e)/T_c^2, d_n = -2 m_eff ln e / T_c, tangential
 * spring k_t = k_n 2(1-nu)/(2-nu) with history, d_t = d_n, Coulomb limit
 * mu |F_n|. n points from particle i to its partner, vrel is the velocity of
 * i's contact point relative to the partner's. Returns the force on i and
 * updates the history. */
static void contact_force(const orc* o, double meff, const double n[3], double delta,
                          const double vrel[3], double xi[3], double dtsub, double F[3], double Ft[3])
{
    double e = o->p.restitution, Tc = o->p.collision_time;
    double le = log(e);
    double kn = meff * (M_PI * M_PI + le * le) / (Tc * Tc);
    double dn = -2.0 * meff * le / Tc;
    double kt = kn * 2.0 * (1.0 - o->p.poisson) / (2.0 - o->p.poisson);
    double dt_ = dn;
    double vn = vrel[0] * n[0] + vrel[1] * n[1] + vrel[2] * n[2];
    double vt[3] = {vrel[0] - vn * n[0], vrel[1] - vn * n[1], vrel[2] - vn * n[2]};
    double fn = kn * delta + dn * vn;          /* force on i is -fn n */
    double xn = xi[0] * n[0] + xi[1] * n[1] + xi[2] * n[2];
    for (int a = 0; a < 3; ++a) xi[a] = xi[a] - xn * n[a] + vt[a] * dtsub;
    for (int a = 0; a < 3; ++a) Ft[a] = -kt * xi[a] - dt_ * vt[a];
    double ftl = sqrt(Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2]);
    double lim = o->p.friction * fabs(fn);
    if (ftl > lim && ftl > 0.0) {
        for (int a = 0; a < 3; ++a) {
            Ft[a] = lim * Ft[a] / ftl;
            xi[a] = -(Ft[a] + dt_ * vt[a]) / kt;
        }
    }
    for (int a = 0; a < 3; ++a) F[a] = -fn * n[a] + Ft[a];
}

/* Lubrication correction (Section 2.2, reading R-23): the paper adds normal
 * and tangential lubrication forces where a gap between two surfaces is too
 * small for the lattice to resolve, and gives no formula. Reading: the
 * asymptotic resistances of two nearly touching spheres with effective
 * radius R_eff = r_i r_j / (r_i + r_j) (a sphere at a wall: R_eff = r),
 *   normal      6 pi mu R_eff^2 / h
 *   tangential  6 pi mu R_eff (8/15) ln(1 / h)   (relative sliding)
 * each less its value at the gap h_c = 2/3 cell that the lattice still
 * resolves, so both vanish at h_c; the gap is clamped below at h_min = 1e-2
 * cell. mu = rho nu with the reference density 1. n points from the
 * particle to its partner (or the wall), vrel is the relative velocity of
 * the surfaces at the contact point; returns the force on the particle. */
#define LUB_HC (2.0 / 3.0)
#define LUB_HMIN 1e-2
static void lubrication_force(const orc* o, double Reff, const double n[3], double h, const double vrel[3],
                              double Fl[3], double Ft[3])
{
    double hh = h < LUB_HMIN ? LUB_HMIN : h;
    double mu = (1.0 / o->p.omega - 0.5) / 3.0;
    double vn = vrel[0] * n[0] + vrel[1] * n[1] + vrel[2] * n[2];
    double cn = 6.0 * M_PI * mu * Reff * Reff * (1.0 / hh - 1.0 / LUB_HC);
    double ct = 6.0 * M_PI * mu * Reff * (8.0 / 15.0) * log(LUB_HC / hh);
    for (int a = 0; a < 3; ++a) {
        double vt = vrel[a] - vn * n[a];
        Ft[a] = -ct * vt;
        Fl[a] = -cn * vn * n[a] + Ft[a];
    }
}

static void dem_substep(orc* o, const double* Fhyd, const double* Thyd, double dts)
{
    int np = o->np;
    double* F = (double*)calloc((size_t)3 * np, sizeof(double));
    double* T = (double*)calloc((size_t)3 * np, sizeof(double));
    int L[3] = {o->p.nx, o->p.ny, o->p.nz};
    for (int i = 0; i < np; ++i)
        for (int a = 0; a < 3; ++a) {
            F[3 * i + a] = Fhyd[3 * i + a] + o->M[i] * o->p.g[a];
            T[3 * i + a] = Thyd[3 * i + a];
        }
    /* particle-particle contacts (each pair once) */
    for (int i = 0; i < np; ++i) {
        for (int j = i + 1; j < np; ++j) {
            if (o->fixed[i] && o->fixed[j]) continue;
            double d[3];
            for (int a = 0; a < 3; ++a) d[a] = min_image(o, a, o->X[3 * j + a] - o->X[3 * i + a]);
            double dist2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double rs = o->R[i] + o->R[j];
            if (o->p.lubrication && dist2 < (rs + LUB_HC) * (rs + LUB_HC)) {
                double dist = sqrt(dist2);
                double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
                double wsum[3], wn[3], vrel[3], Fl[3], Ft[3], ti[3], tj[3];
                for (int a = 0; a < 3; ++a) wsum[a] = o->R[i] * o->W[3 * i + a] + o->R[j] * o->W[3 * j + a];
                cross(wsum, n, wn);
                for (int a = 0; a < 3; ++a) vrel[a] = o->U[3 * i + a] - o->U[3 * j + a] + wn[a];
                lubrication_force(o, o->R[i] * o->R[j] / rs, n, dist - rs, vrel, Fl, Ft);
                double ri_n[3] = {o->R[i] * n[0], o->R[i] * n[1], o->R[i] * n[2]};
                double rj_n[3] = {o->R[j] * n[0], o->R[j] * n[1], o->R[j] * n[2]};
                cross(ri_n, Ft, ti);
                cross(rj_n, Ft, tj);
                for (int a = 0; a < 3; ++a) {
                    F[3 * i + a] += Fl[a];
                    F[3 * j + a] -= Fl[a];
                    T[3 * i + a] += ti[a];
                    T[3 * j + a] += tj[a];
                }
            }
            if (dist2 >= rs * rs) {
                orc_hist* h = hist_find(o, i, j, 0);
                if (h) h->used = 0;
                continue;
            }
            double dist = sqrt(dist2);
            double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
            double delta = rs - dist;
            double wsum[3], wn[3];
            for (int a = 0; a < 3; ++a)
                wsum[a] = o->R[i] * o->W[3 * i + a] + o->R[j] * o->W[3 * j + a];
            cross(wsum, n, wn);
            double vrel[3];
            for (int a = 0; a < 3; ++a) vrel[a] = o->U[3 * i + a] - o->U[3 * j + a] + wn[a];
            double meff = o->M[i] * o->M[j] / (o->M[i] + o->M[j]);
            orc_hist* h = hist_find(o, i, j, 1);
            if (!h) continue;                  /* history table full */
            double Fc[3], Ft[3];
            contact_force(o, meff, n, delta, vrel, h->xi, dts, Fc, Ft);
            double ri_n[3] = {o->R[i] * n[0], o->R[i] * n[1], o->R[i] * n[2]};
            double rj_n[3] = {o->R[j] * n[0], o->R[j] * n[1], o->R[j] * n[2]};
            double ti[3], tj[3];
            cross(ri_n, Ft, ti);
            cross(rj_n, Ft, tj);         /* torque on j: (-r_j n) x (-Ft) */
            for (int a = 0; a < 3; ++a) {
                F[3 * i + a] += Fc[a];
                F[3 * j + a] -= Fc[a];
                T[3 * i + a] += ti[a];
                T[3 * j + a] += tj[a];
            }
        }
    }
    /* particle-wall contacts: wall planes at 0 and L on non-periodic axes,
     * walls have infinite mass and zero velocity */
    for (int i = 0; i < np; ++i) {
        if (o->fixed[i]) continue;
        for (int a = 0; a < 3; ++a) {
            if (o->p.periodic[a]) continue;
            for (int side = 0; side < 2; ++side) {
                int wid = -1 - (2 * a + side);
                double dist = side == 0 ? o->X[3 * i + a] : (L[a] - o->X[3 * i + a]);
                double delta = o->R[i] - dist;
                if (o->p.lubrication && -delta < LUB_HC) {
                    double n[3] = {0, 0, 0};
                    n[a] = side == 0 ? -1.0 : 1.0;
                    double rw[3] = {o->R[i] * o->W[3 * i + 0], o->R[i] * o->W[3 * i + 1], o->R[i] * o->W[3 * i + 2]};
                    double wn[3], vrel[3], Fl[3], Ft[3], ti[3];
                    cross(rw, n, wn);
                    for (int b = 0; b < 3; ++b) vrel[b] = o->U[3 * i + b] + wn[b];
                    lubrication_force(o, o->R[i], n, -delta, vrel, Fl, Ft);
                    double ri_n[3] = {o->R[i] * n[0], o->R[i] * n[1], o->R[i] * n[2]};
                    cross(ri_n, Ft, ti);
                    for (int b = 0; b < 3; ++b) { F[3 * i + b] += Fl[b]; T[3 * i + b] += ti[b]; }
                }
                if (delta <= 0.0) {
                    orc_hist* h = hist_find(o, i, wid, 0);
                    if (h) h->used = 0;
                    continue;
                }
                double n[3] = {0, 0, 0};
                n[a] = side == 0 ? -1.0 : 1.0;
                double rw[3] = {o->R[i] * o->W[3 * i + 0], o->R[i] * o->W[3 * i + 1], o->R[i] * o->W[3 * i + 2]};
                double wn[3];
                cross(rw, n, wn);
                double vrel[3];
                for (int b = 0; b < 3; ++b) vrel[b] = o->U[3 * i + b] + wn[b];
                orc_hist* h = hist_find(o, i, wid, 1);
                if (!h) continue;
                double Fc[3], Ft[3];
                contact_force(o, o->M[i], n, delta, vrel, h->xi, dts, Fc, Ft);
                double ri_n[3] = {o->R[i] * n[0], o->R[i] * n[1], o->R[i] * n[2]};
                double ti[3];
                cross(ri_n, Ft, ti);
                for (int b = 0; b < 3; ++b) { F[3 * i + b] += Fc[b]; T[3 * i + b] += ti[b]; }
            }
        }
    }
    /* semi-implicit Euler (R-14); fixed particles are not integrated: they
     * keep their position and their (normally zero) prescribed velocity */
    for (int i = 0; i < np; ++i) {
        if (o->fixed[i]) continue;
        for (int a = 0; a < 3; ++a) {
            o->U[3 * i + a] += dts * F[3 * i + a] / o->M[i];
            o->W[3 * i + a] += dts * T[3 * i + a] / o->I[i];
            double x = o->X[3 * i + a] + dts * o->U[3 * i + a];
            if (o->p.periodic[a]) x -= L[a] * floor(x / L[a]);
            o->X[3 * i + a] = x;
        }
    }
    free(F);
    free(T);
}

/* ------------------------------------------------------------ one step */

/* the 3x3x3 block around cell i: types (NB_WALL beyond a wall face) from
 * `types`, densities and velocities from the current state */
static void gather_block(const orc* o, long i, const uint8_t* types, uint8_t t27[NQ], double r27[NQ],
                         double u27[3 * NQ])
{
    int x, y, z;
    coords(o, i, &x, &y, &z);
    for (int q = 0; q < NQ; ++q) {
        long y_ = nbr(o, x, y, z, CX[q], CY[q], CZ[q]);
        if (y_ < 0) {
            t27[q] = NB_WALL;
            r27[q] = 0.0;
            u27[3 * q] = u27[3 * q + 1] = u27[3 * q + 2] = 0.0;
            continue;
        }
        t27[q] = types[y_];
        r27[q] = o->rho[y_];
        for (int a = 0; a < 3; ++a) u27[3 * q + a] = o->u[3 * y_ + a];
    }
}

static void one_step(orc* o)
{
    const orc_params* P = &o->p;
    long n = o->n;
    const double rho0 = 1.0;   /* reference density of Section 2.1 */

    /* S1-S3: stream, mass exchange, collide. Reads the state f*, writes ft. */
    double* mnew = (double*)malloc(sizeof(double) * n);
    double* rnew = (double*)malloc(sizeof(double) * n);
    double* unew = (double*)malloc(sizeof(double) * 3 * n);
    long viol = 0;
#pragma omp parallel for schedule(static) reduction(+ : viol)
    for (long i = 0; i < n; ++i) {
        mnew[i] = o->mass[i];
        rnew[i] = o->rho[i];
        unew[3 * i] = o->u[3 * i];
        unew[3 * i + 1] = o->u[3 * i + 1];
        unew[3 * i + 2] = o->u[3 * i + 2];
        int t = o->type[i];
        if (!is_fluid(t)) continue;
        int x, y, z;
        coords(o, i, &x, &y, &z);
        const double* fs = &o->f[i * NQ];
        double fin[NQ];
        double rr, ur[3], feqG[NQ];
        int have_rec = 0;
        for (int q = 0; q < NQ; ++q) {
            int qb = OPP[q];
            long s = nbr(o, x, y, z, -CX[q], -CY[q], -CZ[q]);
            if (s < 0) { fin[q] = fs[qb]; continue; }            /* wall */
            int ts = o->type[s];
            if (ts == T_SOL) {                                     /* moving wall */
                double xb[3] = {x + 0.5 - 0.5 * CX[q], y + 0.5 - 0.5 * CY[q], z + 0.5 - 0.5 * CZ[q]};
                double ub[3];
                particle_velocity_at(o, o->owner[s], xb, ub);
                double cu = CX[q] * ub[0] + CY[q] * ub[1] + CZ[q] * ub[2];
                fin[q] = fs[qb] + 6.0 * WQ[q] * rho0 * cu;
                continue;
            }
            int rebuild = (ts == T_GAS);
            if (!rebuild && t == T_IFC && P->reconstruct_normal) {
                const double* nn = &o->nrm[3 * i];
                double nc = nn[0] * CX[q] + nn[1] * CY[q] + nn[2] * CZ[q];
                if (nc < -P->eps_normal) rebuild = 1;
            }
            if (rebuild) {
                if (t != T_IFC) viol++;
                if (!have_rec) {
                    post_velocity(o, fs, &rr, ur);
                    /* gas pressure plus the Laplace pressure 2 sigma kappa (Section 2.1) */
                    orc_feq(P->rho_gas + 6.0 * P->sigma * o->curv[i], ur, feqG);
                    have_rec = 1;
                }
                fin[q] = feqG[q] + feqG[qb] - fs[qb];
                continue;
            }
            fin[q] = o->f[s * NQ + q];
        }
        /* S2: interface mass exchange with the post-collision PDFs (R-6):
         * m += sum_i s_i (f*_ibar(x+c_i) - f*_i(x)), s = 1 toward liquid,
         * (phi(x)+phi(y))/2 toward interface, 0 otherwise. */
        if (t == T_IFC) {
            double dm = 0.0;
            for (int q = 0; q < NQ; ++q) {
                if (q == 13) continue;
                long y_ = nbr(o, x, y, z, CX[q], CY[q], CZ[q]);
                if (y_ < 0) continue;
                int ty = o->type[y_];
                double s;
                if (ty == T_LIQ) s = 1.0;
                else if (ty == T_IFC) s = 0.5 * (o->phi[i] + o->phi[y_]);
                else continue;
                dm += s * (o->f[y_ * NQ + OPP[q]] - fs[q]);
            }
            mnew[i] = o->mass[i] + dm;
        }
        /* S3: collision */
        double rho = 0, j[3] = {0, 0, 0};
        for (int q = 0; q < NQ; ++q) {
            rho += fin[q];
            j[0] += fin[q] * CX[q];
            j[1] += fin[q] * CY[q];
            j[2] += fin[q] * CZ[q];
        }
        rnew[i] = rho;
        for (int a = 0; a < 3; ++a) unew[3 * i + a] = (j[a] + 0.5 * rho * P->g[a]) / rho;
        orc_collide_gal(fin, P->g, P->omega, P->galilean_correction, &o->ft[i * NQ]);
        if (t == T_LIQ) mnew[i] = rho;
    }
    o->invariant_violations += viol;

    /* S1 (continued): momentum exchange at particle links, serial, with the
     * state f* (Section 2.2; Wen et al. 2014 form, R-12). Force on the
     * particle per link: (c_ibar - u_b) f*_ibar(x) - (c_i - u_b) f_i(x), with
     * zero-centred PDFs (f - w), so the uniform reference pressure exerts no
     * force. Torque (x_b - X_p) x F. */
    for (int p = 0; p < o->np; ++p)
        for (int a = 0; a < 3; ++a) o->Fh[3 * p + a] = o->Th[3 * p + a] = 0.0;
    double injected = 0.0;   /* mass the moving bounce-back added to liquid cells */
    for (long i = 0; i < n; ++i) {
        if (!is_fluid(o->type[i])) continue;
        int x, y, z;
        coords(o, i, &x, &y, &z);
        const double* fs = &o->f[i * NQ];
        for (int q = 0; q < NQ; ++q) {
            long s = nbr(o, x, y, z, -CX[q], -CY[q], -CZ[q]);
            if (s < 0 || o->type[s] != T_SOL) continue;
            int p = o->owner[s];
            int qb = OPP[q];
            double xb[3] = {x + 0.5 - 0.5 * CX[q], y + 0.5 - 0.5 * CY[q], z + 0.5 - 0.5 * CZ[q]};
            double ub[3];
            particle_velocity_at(o, p, xb, ub);
            double cu = CX[q] * ub[0] + CY[q] * ub[1] + CZ[q] * ub[2];
            double fout = fs[qb] - WQ[qb];                       /* f*_ibar - w */
            double fback = fs[qb] + 6.0 * WQ[q] * rho0 * cu - WQ[q];  /* f_i - w */
            if (o->type[i] == T_LIQ) injected += 6.0 * WQ[q] * rho0 * cu;
            double c[3] = {CX[q], CY[q], CZ[q]};
            double Fl[3];
            for (int a = 0; a < 3; ++a) Fl[a] = -c[a] * (fout + fback) - ub[a] * (fout - fback);
            double r[3];
            for (int a = 0; a < 3; ++a) r[a] = min_image(o, a, xb[a] - o->X[3 * p + a]);
            double tq[3];
            cross(r, Fl, tq);
            for (int a = 0; a < 3; ++a) { o->Fh[3 * p + a] += Fl[a]; o->Th[3 * p + a] += tq[a]; }
        }
    }

    /* R-12a: over a closed voxel surface the injections cancel; where a
     * moving sphere touches a wall or another solid they do not, and the
     * remainder is taken from the pool so that the liquid mass is kept */
    if (P->link_mass_correction) o->pool -= injected;

    /* commit S1-S3 */
    double* tmp = o->f; o->f = o->ft; o->ft = tmp;
    free(o->mass); o->mass = mnew;
    free(o->rho); o->rho = rnew;
    free(o->u); o->u = unew;
    for (long i = 0; i < n; ++i) refresh_phi(o, i);

    /* S4: normals of the new fill levels */
    double* n1 = (double*)calloc((size_t)3 * n, sizeof(double));
    for (long i = 0; i < n; ++i)
        if (o->type[i] == T_IFC) normal_at(o, i, o->phi, &n1[3 * i], NULL);

    /* S5: conversion candidates (R-7), from a snapshot of the cell types */
    uint8_t* conv = (uint8_t*)calloc((size_t)n, 1);
    for (long i = 0; i < n; ++i) {
        if (o->type[i] != T_IFC) continue;
        int x, y, z;
        coords(o, i, &x, &y, &z);
        int has_gas = 0, has_liq = 0;
        for (int q = 0; q < NQ; ++q) {
            if (q == 13) continue;
            long y_ = nbr(o, x, y, z, CX[q], CY[q], CZ[q]);
            if (y_ < 0) continue;
            if (o->type[y_] == T_GAS) has_gas = 1;
            if (o->type[y_] == T_LIQ) has_liq = 1;
        }
        double ph = o->phi[i];
        if (ph > 1.0 + P->eps_conv) conv[i] = CV_TO_LIQ;
        else if (ph < -P->eps_conv) conv[i] = CV_TO_GAS;
        else if (!has_gas) conv[i] = CV_TO_LIQ;
        else if (!has_liq) conv[i] = CV_TO_GAS;
    }
    /* S6: filling wins: no to-gas cell next to a to-liquid cell */
    for (long i = 0; i < n; ++i) {
        if (conv[i] != CV_TO_GAS) continue;
        int x, y, z;
        coords(o, i, &x, &y, &z);
        for (int q = 0; q < NQ; ++q) {
            if (q == 13) continue;
            long y_ = nbr(o, x, y, z, CX[q], CY[q], CZ[q]);
            if (y_ >= 0 && conv[y_] == CV_TO_LIQ) { conv[i] = CV_NONE; break; }
        }
    }
    /* S7: gas neighbours of to-liquid cells become interface cells, liquid
     * neighbours of to-gas cells become interface cells (keep their PDFs). */
    uint8_t* mark = (uint8_t*)calloc((size_t)n, 1);
    for (long i = 0; i < n; ++i) {
        if (conv[i] == CV_NONE) continue;
        int x, y, z;
        coords(o, i, &x, &y, &z);
        for (int q = 0; q < NQ; ++q) {
            if (q == 13) continue;
            long y_ = nbr(o, x, y, z, CX[q], CY[q], CZ[q]);
            if (y_ < 0) continue;
            if (conv[i] == CV_TO_LIQ && o->type[y_] == T_GAS) mark[y_] = MK_NEW;
            if (conv[i] == CV_TO_GAS && o->type[y_] == T_LIQ) mark[y_] = MK_EMPTIED;
        }
    }
    for (long i = 0; i < n; ++i) {
        if (mark[i] == MK_NEW) {
            /* f* = f_eq(mean rho, mean u) of the liquid/interface neighbours
             * of the snapshot; m = 0 (a new cell always neighbours the
             * interface cell that filled) */
            uint8_t t27[NQ];
            double r27[NQ], u27[3 * NQ], rb = 0.0, ubar[3] = {0, 0, 0};
            gather_block(o, i, o->type, t27, r27, u27);
            orc_new_interface_mean(t27, r27, u27, &rb, ubar);
            orc_feq(rb, ubar, &o->f[i * NQ]);
            o->rho[i] = rb;
            for (int a = 0; a < 3; ++a) o->u[3 * i + a] = ubar[a];
            o->mass[i] = 0.0;
        } else if (mark[i] == MK_EMPTIED) {
            o->mass[i] = o->rho[i];
        }
    }
    /* S8: excess mass (R-8) */
    for (long i = 0; i < n; ++i) {
        if (conv[i] == CV_NONE) continue;
        double ex;
        if (conv[i] == CV_TO_LIQ) { ex = o->mass[i] - o->rho[i]; o->mass[i] = o->rho[i]; }
        else { ex = o->mass[i]; o->mass[i] = 0.0; }
        /* receivers: interface neighbours that do not convert, and the
         * cells that turn interface in this step */
        int x, y, z;
        coords(o, i, &x, &y, &z);
        uint8_t recv[NQ];
        long cell_of[NQ];
        for (int q = 0; q < NQ; ++q) {
            recv[q] = 0;
            cell_of[q] = -1;
            if (q == 13) continue;
            long y_ = nbr(o, x, y, z, CX[q], CY[q], CZ[q]);
            if (y_ < 0) continue;
            cell_of[q] = y_;
            recv[q] = (o->type[y_] == T_IFC && conv[y_] == CV_NONE) || mark[y_] != MK_NONE;
        }
        double share[NQ];
        if (orc_excess_shares(conv[i] == CV_TO_LIQ, ex, &n1[3 * i], recv, P->excess_even, share)) {
            o->pool += ex;
            continue;
        }
        for (int q = 0; q < NQ; ++q)
            if (recv[q]) o->mass[cell_of[q]] += share[q];
    }
    /* S9: finalise */
    for (long i = 0; i < n; ++i) {
        if (conv[i] == CV_TO_LIQ) o->type[i] = T_LIQ;
        else if (conv[i] == CV_TO_GAS) o->type[i] = T_GAS;
        if (mark[i] != MK_NONE) o->type[i] = T_IFC;
        if (o->type[i] == T_GAS) o->mass[i] = 0.0;
        refresh_phi(o, i);
    }
    free(conv);
    free(mark);
    free(n1);

    /* S10: particles. Hydrodynamic force held at the average of this and the
     * previous step (R-14), n_sub semi-implicit Euler sub-steps. */
    if (o->np > 0) {
        double* Fa = (double*)malloc(sizeof(double) * 3 * o->np);
        double* Ta = (double*)malloc(sizeof(double) * 3 * o->np);
        for (int k = 0; k < 3 * o->np; ++k) {
            Fa[k] = o->have_prev ? 0.5 * (o->Fh[k] + o->Fp[k]) : o->Fh[k];
            Ta[k] = o->have_prev ? 0.5 * (o->Th[k] + o->Tp[k]) : o->Th[k];
            o->Fp[k] = o->Fh[k];
            o->Tp[k] = o->Th[k];
        }
        o->have_prev = 1;
        int ns = P->dem_substeps > 0 ? P->dem_substeps : 1;
        for (int s = 0; s < ns; ++s) dem_substep(o, Fa, Ta, 1.0 / ns);
        free(Fa);
        free(Ta);

        /* S11: re-map (R-11) against a snapshot of the cell types */
        int* own = (int*)malloc(sizeof(int) * n);
        compute_map(o, own);
        uint8_t* snap = (uint8_t*)malloc((size_t)n);
        memcpy(snap, o->type, (size_t)n);
        uint8_t* uncovered_liq = (uint8_t*)calloc((size_t)n, 1);
        for (long i = 0; i < n; ++i) {
            int was = snap[i];
            if (own[i] >= 0) {
                if (is_fluid(was)) o->pool += o->mass[i];
                o->type[i] = T_SOL;
                o->owner[i] = own[i];
                o->mass[i] = 0.0;
                continue;
            }
            if (was != T_SOL) continue;
            /* uncovered */
            int x, y, z;
            coords(o, i, &x, &y, &z);
            int pold = o->owner[i];
            uint8_t t27[NQ];
            double r27[NQ], u27[3 * NQ];
            gather_block(o, i, snap, t27, r27, u27);
            double xc[3] = {x + 0.5, y + 0.5, z + 0.5}, d[3];
            for (int a = 0; a < 3; ++a) d[a] = min_image(o, a, xc[a] - o->X[3 * pold + a]);
            double rb = 0.0, ub[3] = {0, 0, 0}, m = 0.0;
            int t = orc_uncovered_state(t27, r27, &o->U[3 * pold], &o->W[3 * pold], d, &o->f[i * NQ], &rb, ub, &m);
            o->owner[i] = -1;
            o->type[i] = (uint8_t)t;
            if (t == T_GAS) { o->mass[i] = 0.0; continue; }
            o->rho[i] = rb;
            for (int a = 0; a < 3; ++a) o->u[3 * i + a] = ub[a];
            o->mass[i] = m;
            if (t == T_LIQ) uncovered_liq[i] = 1;
            o->pool -= o->mass[i];
        }
        /* uncovered liquid cells that ended next to a gas cell become
         * interface cells (the liquid/gas separation invariant) */
        for (long i = 0; i < n; ++i) {
            if (!uncovered_liq[i]) continue;
            int x, y, z;
            coords(o, i, &x, &y, &z);
            for (int q = 0; q < NQ; ++q) {
                if (q == 13) continue;
                long y_ = nbr(o, x, y, z, CX[q], CY[q], CZ[q]);
                if (y_ >= 0 && o->type[y_] == T_GAS) { o->type[i] = T_IFC; break; }
            }
        }
        for (long i = 0; i < n; ++i) refresh_phi(o, i);
        free(own);
        free(snap);
        free(uncovered_liq);
    }

    /* S12: spread the pool evenly over all interface cells */
    long nifc = 0;
    for (long i = 0; i < n; ++i) nifc += o->type[i] == T_IFC;
    if (nifc > 0 && o->pool != 0.0) {
        double share = o->pool / (double)nifc;
        for (long i = 0; i < n; ++i)
            if (o->type[i] == T_IFC) { o->mass[i] += share; refresh_phi(o, i); }
        o->pool = 0.0;
    }
    /* S13: normals for the next step's boundary condition */
    for (long i = 0; i < n; ++i) {
        if (o->type[i] == T_IFC) normal_at(o, i, o->phi, &o->nrm[3 * i], &o->curv[i]);
        else o->nrm[3 * i] = o->nrm[3 * i + 1] = o->nrm[3 * i + 2] = o->curv[i] = 0.0;
    }
    o->step++;
}

void orc_step(orc* o, int nsteps)
{
    for (int s = 0; s < nsteps; ++s) one_step(o);
}

/* --------------------------------------------------------- accessors */

enum {
    F_PDF = 0, F_TYPE = 1, F_MASS = 2, F_PHI = 3, F_RHO = 4, F_U = 5, F_NORMAL = 6, F_OWNER = 7, F_CURV = 8,
    P_X = 16, P_U = 17, P_W = 18, P_F = 19, P_T = 20, P_R = 21
};

/* Copies a field out. PDFs are exported direction-major: dst[q*n + cell]. */
int orc_get(const orc* o, int which, void* dst)
{
    long n = o->n;
    switch (which) {
    case F_PDF: {
        double* d = (double*)dst;
        for (int q = 0; q < NQ; ++q)
            for (long i = 0; i < n; ++i) d[q * n + i] = o->f[i * NQ + q];
        return 0;
    }
    case F_TYPE: memcpy(dst, o->type, (size_t)n); return 0;
    case F_MASS: memcpy(dst, o->mass, sizeof(double) * n); return 0;
    case F_PHI: memcpy(dst, o->phi, sizeof(double) * n); return 0;
    case F_RHO: memcpy(dst, o->rho, sizeof(double) * n); return 0;
    case F_U: {
        double* d = (double*)dst;
        for (int a = 0; a < 3; ++a)
            for (long i = 0; i < n; ++i) d[a * n + i] = o->u[3 * i + a];
        return 0;
    }
    case F_NORMAL: {
        double* d = (double*)dst;
        for (int a = 0; a < 3; ++a)
            for (long i = 0; i < n; ++i) d[a * n + i] = o->nrm[3 * i + a];
        return 0;
    }
    case F_OWNER: memcpy(dst, o->owner, sizeof(int) * n); return 0;
    case F_CURV: memcpy(dst, o->curv, sizeof(double) * n); return 0;
    case P_X: memcpy(dst, o->X, sizeof(double) * 3 * o->np); return 0;
    case P_U: memcpy(dst, o->U, sizeof(double) * 3 * o->np); return 0;
    case P_W: memcpy(dst, o->W, sizeof(double) * 3 * o->np); return 0;
    case P_F: memcpy(dst, o->Fh, sizeof(double) * 3 * o->np); return 0;
    case P_T: memcpy(dst, o->Th, sizeof(double) * 3 * o->np); return 0;
    case P_R: memcpy(dst, o->R, sizeof(double) * o->np); return 0;
    default: return -1;
    }
}

/* Overwrites a field (test set-up). PDFs direction-major as in orc_get;
 * after PDFs the cell densities and velocities are recomputed from them. */
int orc_set(orc* o, int which, const void* src)
{
    long n = o->n;
    switch (which) {
    case F_PDF: {
        const double* s = (const double*)src;
        for (int q = 0; q < NQ; ++q)
            for (long i = 0; i < n; ++i) o->f[i * NQ + q] = s[q * n + i];
        for (long i = 0; i < n; ++i) {
            if (!is_fluid(o->type[i])) continue;
            double r, u[3];
            post_velocity(o, &o->f[i * NQ], &r, u);
            o->rho[i] = r;
            for (int a = 0; a < 3; ++a) o->u[3 * i + a] = u[a];
            if (o->type[i] == T_LIQ) o->mass[i] = r;
            refresh_phi(o, i);
        }
        return 0;
    }
    case F_MASS:
        memcpy(o->mass, src, sizeof(double) * n);
        for (long i = 0; i < n; ++i) refresh_phi(o, i);
        for (long i = 0; i < n; ++i)
            if (o->type[i] == T_IFC) normal_at(o, i, o->phi, &o->nrm[3 * i], &o->curv[i]);
        return 0;
    case P_U: memcpy(o->U, src, sizeof(double) * 3 * o->np); return 0;
    case P_W: memcpy(o->W, src, sizeof(double) * 3 * o->np); return 0;
    case P_X: memcpy(o->X, src, sizeof(double) * 3 * o->np); return 0;
    default: return -1;
    }
}

#ifdef _OPENMP
#include <omp.h>
#endif
/* number of threads the parallel loops use */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

long orc_ncells(const orc* o) { return o->n; }
int orc_nparticles(const orc* o) { return o->np; }
long orc_violations(const orc* o) { return o->invariant_violations; }
double orc_pool(const orc* o) { return o->pool; }
/* test set-up: the FP64 mass pool that the next step spreads */
void orc_set_pool(orc* o, double pool) { o->pool = pool; }

/* Body-force acceleration (gravity) for the following steps: the fluid's
 * forcing and the particles' weight both read it. */
void orc_set_gravity(orc* o, double gx, double gy, double gz)
{
    o->p.g[0] = gx;
    o->p.g[1] = gy;
    o->p.g[2] = gz;
}

/* Diagnostics: [0] liquid mass sum_L rho + sum_I m + pool, [1..3] fluid
 * momentum sum rho u over liquid and interface cells, [4] fill-weighted bulk
 * velocity sum phi rho u_x / sum phi rho, [5] interface cell count,
 * [6] bedload rate of Eq. (1) sum u_x,p V_p / (L_x L_y), [7] pool. */
void orc_reduce(const orc* o, double out[8])
{
    double mass = 0, mom[3] = {0, 0, 0}, num = 0, den = 0, nifc = 0;
    for (long i = 0; i < o->n; ++i) {
        int t = o->type[i];
        if (!is_fluid(t)) continue;
        mass += o->mass[i];
        for (int a = 0; a < 3; ++a) mom[a] += o->rho[i] * o->u[3 * i + a];
        num += o->phi[i] * o->rho[i] * o->u[3 * i];
        den += o->phi[i] * o->rho[i];
        if (t == T_IFC) nifc += 1;
    }
    double qb = 0;
    for (int p = 0; p < o->np; ++p)
        qb += o->U[3 * p] * (4.0 / 3.0) * M_PI * o->R[p] * o->R[p] * o->R[p];
    qb /= (double)o->p.nx * (double)o->p.ny;
    out[0] = mass + o->pool;
    out[1] = mom[0]; out[2] = mom[1]; out[3] = mom[2];
    out[4] = den > 0 ? num / den : 0.0;
    out[5] = nifc;
    out[6] = qb;
    out[7] = o->pool;
}
