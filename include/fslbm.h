/*
 * fslbm.h - C ABI of the GB300 (sm_103a) implementation of one time step of
 * the coupled free-surface lattice Boltzmann / discrete-element method of
 * Schwarzmeier et al., "Particle-resolved simulation of antidunes in
 * free-surface flows" (Section 2).
 *
 * One time step (Section 2; step order as documented with fslbm_step):
 *   - D3Q27 cumulant collision, all rates 1 except the shear rate omega,
 *     nu = (1/omega - 1/2)/3, with gravity forcing (Section 2.1);
 *   - streaming with halfway bounce-back at no-slip walls (Section 2.1);
 *   - free-surface (volume-of-fluid) update: gas-pressure boundary condition
 *     at interface cells, interface mass exchange, cell conversion and excess
 *     mass redistribution (Section 2.1);
 *   - geometrically resolved spheres: moving bounce-back and momentum-exchange
 *     force/torque, explicit particle-to-grid mapping (Section 2.2);
 *   - DEM contact (restitution, collision time, Poisson ratio, friction) and
 *     Newton-Euler integration (Section 2.2).
 *
 * Conventions
 *   - Lattice units: cell size 1, time step 1, reference density 1
 *     (Section 2.1). Cell (x,y,z) has its centre at (x+1/2, y+1/2, z+1/2);
 *     linear index x + nx*(y + ny*z) (x fastest).
 *   - Directions q = (cx+1) + 3(cy+1) + 9(cz+1), c in {-1,0,1}^3.
 *   - Cell types: 0 gas, 1 liquid, 2 interface, 3 solid (particle).
 *   - Ownership: the library owns every device buffer it allocates; callers
 *     own what they pass in. Calls are ordered on the CUDA stream given to
 *     fslbm_create. fslbm_step only enqueues work; fslbm_get_fields,
 *     fslbm_set_fields, fslbm_reduce and fslbm_sync synchronise the stream.
 *   - Errors: every call returns 0 or a negative FSLBM_E* code; no exception
 *     or abort crosses the ABI. Errors detected on the device (capacity
 *     overflow, non-finite values, an exhausted wait) are recorded in a sticky
 *     device error word that the next synchronising call returns; once set it
 *     stays set until fslbm_destroy.
 *   - Thread safety: one handle must not be used from two threads at once.
 */
#ifndef FSLBM_H
#define FSLBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FSLBM_ABI_VERSION 1

#define FSLBM_OK 0
#define FSLBM_EINVAL (-1)      /* invalid argument or parameter */
#define FSLBM_ENOMEM (-2)      /* device allocation failed */
#define FSLBM_ECAPACITY (-3)   /* a fixed-capacity device list overflowed */
#define FSLBM_ENAN (-4)        /* non-finite value detected */
#define FSLBM_EDEVICE (-5)     /* CUDA runtime error */
#define FSLBM_ESTATE (-6)      /* call not valid in the current state */
#define FSLBM_EINVARIANT (-7)  /* a liquid cell touched a gas cell */
#define FSLBM_ETIMEOUT (-8)    /* a bounded device wait gave up */

/* boundary flags: a set bit makes the axis periodic, a clear bit puts no-slip
 * walls (halfway bounce-back, Section 2.1) on both of its faces */
#define FSLBM_PERIODIC_X 1u
#define FSLBM_PERIODIC_Y 2u
#define FSLBM_PERIODIC_Z 4u

/* PDF storage (all arithmetic is FP32; the stored value is f_i - w_i, in
 * FP16 multiplied by the exact factor 2^12 so that small deviations stay in
 * FP16's normal range; |f_i - w_i| above 16 overflows and is reported as
 * FSLBM_ENAN) */
#define FSLBM_STORE_FP32 0
#define FSLBM_STORE_FP16 1
#define FSLBM_STORE_BF16 2

#define FSLBM_GAS 0
#define FSLBM_LIQUID 1
#define FSLBM_INTERFACE 2
#define FSLBM_SOLID 3

typedef struct fslbm fslbm;

/* Parameters of the problem statement (Sections 2.1, 2.2, 3.1), lattice
 * units. Fill with fslbm_default_params, then override. */
typedef struct {
    uint32_t struct_size;        /* sizeof(fslbm_params), ABI check */
    int32_t nx, ny, nz;          /* lattice size, each >= 1 */
    uint32_t bc_flags;           /* FSLBM_PERIODIC_* bits */
    double omega;                /* shear relaxation rate, 0 < omega < 2 */
    double g[3];                 /* body acceleration (gravity incl. slope forcing) */
    double rho_gas;              /* gas pressure p_g = rho_gas / 3 */
    double sigma;                /* surface tension sigma >= 0 (Section 2.1): the
                                    gas-side reconstruction density is
                                    rho_gas + 6 sigma kappa, kappa the
                                    curvature of the learned normal model (0
                                    where the finite-difference normal is
                                    taken, which carries none) */
    double liquid_height;        /* initial flat free surface height (cells) */
    int32_t init_profile;        /* 0: fluid at rest */
    int32_t storage;             /* FSLBM_STORE_* */
    int32_t normal_model;        /* 0: finite-difference (Parker-Youngs) normal;
                                    1: learned normal (weights must be set with
                                    fslbm_set_normal_model before fslbm_step) */
    int32_t reconstruct_normal;  /* 1: also rebuild PDFs with n.c_i < -eps_normal */
    double eps_conv;             /* conversion hysteresis on the fill level */
    double eps_normal;           /* margin of the normal-based reconstruction */
    double rho_p;                /* particle density (liquid reference 1) */
    double restitution;          /* DEM coefficient of restitution, 0 < e <= 1 */
    double friction;             /* Coulomb friction coefficient */
    double poisson;              /* Poisson ratio of the particle material */
    double collision_time;       /* DEM collision time T_c (time steps) */
    int32_t dem_substeps;        /* DEM sub-steps per LBM step, >= 1 */
    int32_t link_mass_correction; /* 1: the net mass the moving bounce-back injects
                                    into liquid cells is taken from the mass pool */
    int64_t capacity_particles;  /* maximum number of spheres (0: 65536) */
    int64_t capacity_interface;  /* maximum interface cells (0: ncells/4 + 4096) */
    int32_t excess_even;         /* 1: the excess mass of a converting cell is split
                                    evenly over its receivers instead of along the
                                    normal (a variant of the free-surface method) */
    int32_t lubrication;         /* 1: lubrication corrections of the DEM where a gap
                                    between two particles, or a particle and a wall,
                                    is below the 2/3 cell the lattice resolves
                                    (Section 2.2): normal 6 pi mu R^2 (1/h - 1/h_c),
                                    tangential 6 pi mu R (8/15) ln(h_c / h), R the
                                    effective radius, h clamped at 1e-2 */
    int32_t galilean_correction; /* 1: Galilean-invariance correction of the second-
                                    order relaxation (Geier et al. 2015): the normal-
                                    stress differences and the trace lose their terms
                                    of third order in u; the liquid cells then run in
                                    the one-cell kernel. Default 0 (the paper's runs,
                                    read as without it) */
    int32_t link_mode;           /* where the moving bounce-back and the momentum
                                    exchange at particle links (Section 2.2) are taken:
                                    0 (default) the library's choice, at present 1;
                                    1 a separate pass over the solid cells before the
                                    liquid cells; 2 the fluid side, inside the kernels
                                    of the liquid and interface cells, where the lattice
                                    allows it (x extent a multiple of 32, 32-bit element
                                    indices, no Galilean correction; else 1). Both give
                                    the same values up to rounding */
} fslbm_params;

/* Fills *p with defaults: periodic x, walls in y and z, omega = 1/0.51,
 * g = 0, rho_gas = 1, eps_conv = eps_normal = 1e-2, reconstruct_normal = 1,
 * rho_p = 2.55, e = 0.88, mu = 0.5, nu_p = 0.22, T_c = 24, 10 sub-steps,
 * lubrication on, Galilean correction off. */
void fslbm_default_params(fslbm_params* p);

/* Creates a simulation on the current CUDA device. `cuda_stream` is a
 * cudaStream_t (NULL: the legacy default stream); every later call is
 * ordered on it. The fluid starts flat at rest (Section 3.1): cells below
 * liquid_height liquid, the layer holding or touching the surface interface
 * with its fill level, gas above; hydrostatic density rho_gas
 * exp(3 |g_z| (H - z)). Returns FSLBM_EINVAL for bad parameters (including
 * a negative or non-finite sigma and normal_model outside {0, 1}), FSLBM_ENOMEM if the device buffers do
 * not fit. On success *out owns every device buffer of the run. */
int fslbm_create(const fslbm_params* p, void* cuda_stream, fslbm** out);

/* Adds n spheres (Section 2.2): centres xyz[3n], radii radius[n] (> 0 and
 * < half of every periodic extent), fixed[n] (1: never integrated, velocity
 * kept as set; NULL: all mobile). Pointers are host memory unless on_device
 * is 1. Cells whose centre lies inside a sphere become solid; their fluid is
 * removed. Must be called before the first fslbm_step; may be called once. */
int fslbm_add_spheres(fslbm* s, int64_t n, const double* xyz, const double* radius,
                      const uint8_t* fixed, int on_device);

/* Re-initialises the liquid from a free-surface height per column,
 * height_xy[y*nx + x] (host or device per on_device), with the rule of
 * fslbm_create applied column by column; solid cells are kept. Valid before
 * the first fslbm_step only. */
int fslbm_init_surface(fslbm* s, const double* height_xy, int on_device);

/* Advances n_steps time steps. Each step (Section 2):
 *   1 stream with boundary conditions, momentum exchange, interface mass
 *     exchange, cumulant collision;
 *   2 interface normals; conversion candidates (fill level beyond
 *     1 + eps_conv or below -eps_conv, or no gas / no liquid neighbour);
 *     filling wins over emptying; gas neighbours of filled cells and liquid
 *     neighbours of emptied cells become interface cells; excess mass is
 *     spread over interface neighbours along the normal;
 *   3 hydrodynamic force averaged over two steps, DEM sub-steps;
 *   4 particle re-mapping (covered cells give their mass to a pool,
 *     uncovered cells are refilled from it);
 *   5 the pool is spread over all interface cells; normals for the next step.
 * Asynchronous on the stream; returns the sticky error word as of the call
 * (a device error raised by these steps is returned by a later call).
 * From the third step on, each step is replayed from a CUDA graph captured
 * once per parity (the same kernels with the same arguments, so the results
 * are bitwise those of direct launches), unless the stream given to
 * fslbm_create is the legacy default stream (NULL), which cannot be captured,
 * the caller is itself capturing the stream (the launches then go into the
 * caller's graph), or the flow-rate control is on. The graphs are captured
 * again after a call that changes a launch argument (body force, flow
 * control, wait limit, normal model, spheres). */
int fslbm_step(fslbm* s, int64_t n_steps);

/* Field selection bits for fslbm_get_fields / fslbm_set_fields. dst[k] /
 * src[k] is the buffer of the k-th selected field in increasing bit order.
 * Layouts (N = nx*ny*nz, np = number of spheres):
 *   PDF     double [27][N]   post-collision PDFs f*_q, 0 outside liquid/interface
 *   TYPE    uint8  [N]       cell type
 *   MASS    double [N]       liquid: rho, interface: m, else 0
 *   PHI     double [N]       fill level (liquid 1, interface m/rho, else 0)
 *   RHO     double [N]       density of liquid/interface cells, else 0
 *   U       double [3][N]    velocity of the last collision (liquid/interface)
 *   NORMAL  double [3][N]    interface normal (toward the gas), else 0
 *   OWNER   int32  [N]       owning sphere of solid cells, else -1
 *   P_X, P_U, P_OMEGA, P_F, P_T  double [np][3]  centre, velocity, angular
 *            velocity, hydrodynamic force and torque of the last step
 *   P_R     double [np]      radius                                       */
#define FSLBM_FIELD_PDF (1u << 0)
#define FSLBM_FIELD_TYPE (1u << 1)
#define FSLBM_FIELD_MASS (1u << 2)
#define FSLBM_FIELD_PHI (1u << 3)
#define FSLBM_FIELD_RHO (1u << 4)
#define FSLBM_FIELD_U (1u << 5)
#define FSLBM_FIELD_NORMAL (1u << 6)
#define FSLBM_FIELD_OWNER (1u << 7)
#define FSLBM_FIELD_P_X (1u << 16)
#define FSLBM_FIELD_P_U (1u << 17)
#define FSLBM_FIELD_P_OMEGA (1u << 18)
#define FSLBM_FIELD_P_F (1u << 19)
#define FSLBM_FIELD_P_T (1u << 20)
#define FSLBM_FIELD_P_R (1u << 21)

/* Copies the selected fields into dst (device pointers if dst_on_device,
 * else host). Synchronises the stream; returns the sticky error word. */
int fslbm_get_fields(fslbm* s, uint32_t field_mask, void* const* dst, int dst_on_device);

/* Overwrites the selected fields from src (host unless src_on_device).
 * Supported: PDF (densities, velocities and liquid masses follow from it),
 * MASS (interface masses; fill levels and normals are recomputed), P_U,
 * P_OMEGA. Synchronises the stream. */
int fslbm_set_fields(fslbm* s, uint32_t field_mask, const void* const* src, int src_on_device);

/* FP64 diagnostics (Section 3.2): out[0] liquid mass (sum over liquid rho +
 * sum over interface m + mass pool), out[1..3] fluid momentum, out[4]
 * fill-weighted bulk velocity sum phi rho u_x / sum phi rho, out[5] number of
 * interface cells, out[6] bedload rate of Eq. (1) sum u_x,p V_p / (L_x L_y),
 * out[7] mass pool. Synchronises the stream. */
int fslbm_reduce(fslbm* s, double out[8]);

/* Body-force acceleration g (lattice units): drives the fluid (Section 2.1
 * forcing) and weighs the particles, from the next step on. Each component
 * must be finite and within [-1, 1]; else FSLBM_EINVAL. No synchronisation. */
int fslbm_set_body_force(fslbm* s, const double g[3]);
int fslbm_get_body_force(const fslbm* s, double g[3]);

/* Flow-rate control (Section 3.1: the streamwise body force is adjusted
 * during the run to hold the bulk flow rate). The paper gives no control
 * law; this one is an integral controller: after every `interval` completed
 * steps of fslbm_step, with U the fill-weighted bulk velocity of the state
 * reached (fslbm_reduce out[4]), g_x <- g_x + gain (target_u - U). Each
 * update costs one reduction over the lattice and a synchronisation of the
 * stream. In a steady laminar film of depth H it settles at
 * g_x = 3 nu target_u / H^2. The updated g_x is clamped to [-1, 1], the range
 * fslbm_set_body_force accepts; a non-finite update sets FSLBM_ENAN.
 *   target_u  finite
 *   interval  steps between updates; 0 switches the control off
 *   gain      finite, >= 0, in acceleration per unit of velocity error
 * Invalid arguments: FSLBM_EINVAL. */
int fslbm_set_flow_control(fslbm* s, double target_u, double gain, int64_t interval);

/* Bed topography (Section 3.2): phi_b(x, z), the fraction of the cells of
 * the column (x, ., z) covered by a particle (y-averaged solid fraction), and
 * the bed height h_b(x), the z at which phi_b crosses phi_b_level (the paper
 * uses 0.3), linearly interpolated between cell centres (cell k at
 * z = k + 1/2). The topmost crossing counts; above the lattice phi_b is 0,
 * and below it the bottom wall counts as solid (phi_b = 1 at z = -1/2). A
 * bed whose top solid layer is H - 1 therefore gives H - 1/2 + (1 - level).
 *   phi_b_level  threshold in (0, 1]; other values: FSLBM_EINVAL
 *   h            double [nx] out, x-fastest (device if on_device, else host)
 *   phi          optional double [nz][nx] out (NULL: not copied), same memory
 *                kind as h
 * The first call allocates (nz + 1) nx doubles of device scratch, kept until
 * fslbm_destroy. Synchronises the stream; returns the sticky error word. */
int fslbm_bed_height(fslbm* s, double phi_b_level, double* h, double* phi, int on_device);

/* Transport and flow numbers of the current state (Section 4.2, Table 2):
 *   out[0] mean water depth h_bar: the free-surface elevation of each column
 *          (its liquid and solid volume: 1 per liquid or solid cell, the fill
 *          level per interface cell), averaged over y, less the bed height
 *          h_b(x) at phi_b = 0.3 (fslbm_bed_height), averaged over x
 *   out[1] tan(psi) = g_x / |g_z|, the slope of the imposed body force
 *   out[2] Shields number h_bar tan(psi) / (d50 (rho_p - 1)), with the
 *          hydraulic radius taken as h_bar (periodic spanwise boundaries)
 *   out[3] bedload rate q_b of Eq. (1) (fslbm_reduce out[6])
 *   out[4] Einstein number q_b / sqrt((rho_p - 1) |g| d50^3), |g| the
 *          magnitude of the body acceleration
 *   out[5] mean bed height
 * rho_p is the particle density of the run (liquid reference density 1);
 * out[2] and out[4] are 0 where rho_p = 1 or g = 0. d50 > 0 (lattice units).
 * The first call allocates nx (nz + ny + 1) + 2 doubles of device scratch,
 * kept until fslbm_destroy. Synchronises the stream. */
int fslbm_transport_numbers(fslbm* s, double d50, double out[6]);

/* Power spectral density of a bed-height series (Section 4.1) and its
 * dominant bedform. h: device, double [nt][nx], h_b(x) sampled every dt
 * steps on cells of size dx (for example rows of fslbm_bed_height results);
 * psd: device, double [nt][nx], written with |H(l, j)|^2 / (nt nx), H the
 * two-dimensional discrete Fourier transform over t and x (kernel
 * exp(-2 pi i (j x / nx + l t / nt))) of h less its mean. peak: host,
 * double [4], the largest value at wavenumbers 1 <= j <= nx / 2 (ties: the
 * lowest l, then j) as wavelength nx dx / j, period nt dt / |l| (l taken in
 * (-nt/2, nt/2]; infinity for l = 0), celerity wavelength / period, positive
 * toward +x, and amplitude 2 sqrt(psd / (nt nx)) (exact for a single
 * travelling sine on the grid's frequencies). 2 <= nt <= 65535,
 * 2 <= nx <= 2^20, dx, dt > 0, else FSLBM_EINVAL. Needs no handle;
 * allocates 16 (nx + nt + nt nx) + 32 bytes of device scratch for the call
 * (FSLBM_ENOMEM if that fails) and synchronises cuda_stream (NULL: the
 * legacy default stream). FSLBM_EDEVICE on a CUDA error. */
int fslbm_bed_spectrum(const double* h, int64_t nt, int64_t nx, double dx, double dt, double* psd, double peak[4],
                       void* cuda_stream);

/* Waits for the stream; returns the sticky error word. */
int fslbm_sync(fslbm* s);

/* Number of completed steps and of spheres. */
int64_t fslbm_steps_done(const fslbm* s);
int64_t fslbm_num_spheres(const fslbm* s);

/* Checks the liquid/gas separation that the conversion rules maintain: adds
 * the number of liquid cells that have a gas neighbour now to a running
 * count and returns that count (0 while the separation holds). Synchronises
 * the stream. */
int64_t fslbm_invariant_violations(fslbm* s);

/* Measurement hooks for the benchmark. fslbm_timing(s, 1) clears and starts
 * recording a pair of CUDA events around every stream-collide sweep (the
 * dominant kernel pair: bulk-cell and boundary-cell kernels) that fslbm_step
 * enqueues, and counting the kernel launches it enqueues; fslbm_timing(s, 0)
 * stops recording. fslbm_timing_read waits for the stream and returns the
 * summed sweep time in milliseconds, the number of sweeps and the number of
 * kernel launches since the last start. */
int fslbm_timing(fslbm* s, int on);
int fslbm_timing_read(fslbm* s, double* sweep_ms, int64_t* sweeps, int64_t* kernel_launches);

/* Test hook of the device error path. Every wait of a kernel on an
 * asynchronous copy (the bulk copies of the staged stream-collide sweep) is
 * bounded: after `polls` unsuccessful polls it gives up, sets the sticky
 * error FSLBM_ETIMEOUT, and its kernel returns early (still waiting, with the
 * default bound, for the copies it has issued, so that none lands after the
 * block has left). The default, and the maximum, is 4194304 polls; 0 makes
 * every such wait give up at once, which lets a test check that a wait that
 * runs out reaches the caller as FSLBM_ETIMEOUT with the context still
 * usable. Takes effect from the next fslbm_step. FSLBM_EINVAL outside
 * [0, 4194304]. */
int fslbm_set_wait_limit(fslbm* s, int64_t polls);

/* Number of cells of each type (gas, liquid, interface, solid) in
 * counts[0..3]. Synchronises the stream. */
int fslbm_cell_counts(fslbm* s, int64_t counts[4]);

/* Allocation-free FP64 reduction of lattice fields the caller already holds
 * on the device. The paper has no counterpart; this is a service for callers
 * that cannot call cudaMalloc, such as code running inside a memory pool that
 * another framework owns, or code allowed to touch only the memory it is
 * handed. It needs no fslbm handle and allocates nothing: its scratch is a
 * fixed 128 KiB array in the library's device image, present on every device
 * that loads the library until the process exits.
 *   pdf    device, double [27][ncells]: PDFs in the layout of
 *          FSLBM_FIELD_PDF (what fslbm_get_fields exports)
 *   type   device, uint8 [ncells]: cell types (FSLBM_FIELD_TYPE)
 *   mass   device, double [ncells]: interface masses (FSLBM_FIELD_MASS)
 *   g      host, double [3]: the body acceleration of the run
 *   out    device, double [4]: written with the liquid mass (sum over liquid
 *          rho + sum over interface m) and the fluid momentum (x, y, z), the
 *          quantities of fslbm_reduce out[0] - out[7] and out[1..3]
 *   cuda_stream  cudaStream_t the work is ordered on (NULL: legacy default)
 * Returns FSLBM_EINVAL for NULL pointers or ncells <= 0, FSLBM_ECAPACITY for
 * ncells above 4096 * 65536 (the scratch holds 4096 blocks of partial sums),
 * FSLBM_EDEVICE if the scratch address cannot be obtained or a launch fails.
 * The call only enqueues work; read out after synchronising the stream. The
 * first call on a device loads the library's device code there, if nothing
 * has yet, to find the scratch array's address (make that first call before
 * any stream capture); every call looks the address up again, which is a
 * host-side query, so a device reset between calls does no harm. Pending
 * launch errors of earlier, unrelated work are cleared at entry and not
 * reported by this call. Every call shares the one scratch array, which
 * keeps the last call's partial sums: calls whose kernels overlap on the GPU
 * (different streams without ordering) race on it. Each call overwrites every
 * partial sum it reads, so nothing needs clearing between calls, and the sums
 * are added in a fixed order: two calls on the same fields give identical
 * results. */
int fslbm_reduce_fields_noalloc(const double* pdf, const uint8_t* type, const double* mass, int64_t ncells,
                                const double g[3], double* out, void* cuda_stream);

/* ---------------------------------------------------------------- learned normal
 * The interface normal used by the free-surface boundary condition (the
 * choice of reconstructed directions) and by the excess-mass weights
 * (Section 2.1 cites the free-surface LBM; the paper names no normal
 * scheme) can come from a 27-64-64-4 perceptron with ReLU instead of the
 * finite-difference (Parker-Youngs) gradient. Its input is the fill levels
 * of the 3x3x3 block around an interface cell (liquid 1, gas 0, interface
 * phi clamped to [0,1]; block index q = (cx+1) + 3(cy+1) + 9(cz+1)); its
 * outputs are a raw normal toward the gas and the curvature. Parameters,
 * 6212 values: W1 (64x27), b1 (64), W2 (64x64), b2 (64), W3 (4x64), b3 (4),
 * matrices row-major (out, in). The finite-difference normal is kept where a
 * wall or solid cell lies in the block, where the raw normal's length is
 * outside [1/2, 2], and where the two normals are more than 30 degrees
 * apart. Products run on tensor cores: BF16 operands, FP32 accumulation. */

/* Selects the learned normal for the run and recomputes the interface
 * normals of the current state. w: host memory, n_params = 6212 BF16 bit
 * patterns in the parameter layout (copied; the caller keeps ownership).
 * w = NULL with n_params = 0 returns to the finite-difference normal.
 * Stream-ordered; synchronises the stream. FSLBM_EINVAL for another size. */
int fslbm_set_normal_model(fslbm* s, const uint16_t* w, int64_t n_params);

/* Mirror averaging of the learned normal (a reading for the normal the
 * free-surface condition of Section 2.1 uses; the paper has no learned
 * normal): on = 1 evaluates the network on the block and on its mirror
 * images in x, in y and in both (block index q takes the value of the
 * mirrored index), negates the mirrored components of each output, and
 * averages the four raw outputs before the length and angle rules above.
 * The normal is then exactly equivariant under those mirrors: a block that
 * is its own mirror image gets no component along the mirrored axis (a flat
 * horizontal surface keeps a vertical normal), where the plain network can
 * tilt it by a fraction of a degree. The products remain BF16 operands with
 * FP32 sums; the averaging is FP32. on = 0 (the default) is the plain
 * network. Recomputes the interface normals of the current state when a
 * network is set. Synchronises the stream. FSLBM_EINVAL for another value
 * of on or a missing handle. */
int fslbm_set_normal_mirror(fslbm* s, int32_t on);

/* Learned-normal counters since the last fslbm_set_normal_model:
 * out[0] normals evaluated, out[1] normals taken from the network (the rest
 * fell back). Zeros under the finite-difference normal. Synchronises. */
int fslbm_normal_stats(fslbm* s, uint64_t out[2]);

/* Interface stencils of the current state, labelled by the height-function
 * method: training and test data of the learned normal taken from the
 * method's own runs (the paper has no learned normal). For every interface
 * cell whose 3x3x3 block holds no wall or
 * solid cell: the network's input (fill levels of the block, liquid 1,
 * interface phi clamped to [0, 1], gas 0, stencil index
 * (dx+1) + 3(dy+1) + 9(dz+1)) and, where the height function is defined, a
 * label. The height function takes the axis a of the largest component of
 * the Parker-Youngs normal, sums the fill levels of the 3x3 columns of seven
 * cells along a centred on the cell's row (a column counts only if its end
 * cell on the liquid side is liquid and on the gas side gas), and forms the
 * normal toward the gas and the mean curvature (positive for a convex liquid
 * body) from the central differences of the heights.
 *   capacity  stencils the buffers hold; the first `capacity` found are
 *             written, in no fixed order
 *   fill      device float [capacity][27] out
 *   target    device float [capacity][4] out: label (n_x, n_y, n_z, kappa)
 *   fd        optional (NULL) device float [capacity][4] out: the
 *             Parker-Youngs normal of the same block, 0
 *   cells     optional (NULL) device int32 [capacity] out: cell index
 *   found     host out: the number of labelled stencils (may exceed capacity)
 * Stream-ordered; synchronises the stream. FSLBM_EINVAL for a NULL handle or
 * found, capacity < 0, or capacity > 0 with fill or target NULL. */
int fslbm_log_stencils(fslbm* s, int64_t capacity, float* fill, float* target, float* fd, int32_t* cells,
                       int64_t* found);

/* Training data of the learned normal. params: device, n rows of 12 doubles
 * describing analytic surfaces through P = s n0 (kind 0 plane, 1 liquid
 * sphere of radius r centred at P - r n0, 2 gas sphere centred at P + r n0,
 * 3 sine wave w <= A (sin(k u + phase) - sin(phase)) with u = (x-P).e1,
 * w = (x-P).n0); row layout: kind, n0[3], s, r, A, k, phase, e1[3]. Writes,
 * on the device, fill[n][27] (liquid volume fraction of each cell of the
 * block around the origin: exact for planes, exact x-chords of 64x64 rows
 * for spheres, 64^3 midpoint samples for sine waves) and target[n][4]
 * (unit normal toward the gas at P, mean curvature, positive for a convex
 * liquid body). Synchronises. */
int fslbm_mlp_stencils(const double* params, int64_t n, float* fill, float* target, void* cuda_stream);

/* Loss and gradient of the learned normal over n stencils (device
 * pointers): theta[6212] FP32 parameters, fill[n][27], target[n][4];
 * loss = mean of 1 - cos(n, n_true) + lam (k - k_true)^2 + mu (|n| - 1)^2,
 * written to loss[1]; its gradient to grad[6212]. n <= 2^24.
 * Synchronises. */
int fslbm_mlp_gradient(const float* theta, const float* fill, const float* target, int64_t n, double lam,
                       double mu, float* grad, float* loss, void* cuda_stream);

/* Adam (beta 0.9, 0.999, eps 1e-8, bias-corrected, moments starting at
 * zero) for `steps` batches of `batch` stencils drawn from the n in
 * fill/target: slot j of step t takes SplitMix64 output t*batch + j of
 * `seed`, v, stencil v mod n and, with augment, cube symmetry
 * (v >> 32) mod 48 (permutation (v>>32 mod 48)/8 of the axes in
 * lexicographic order, sign flips from its low 3 bits). The step size of
 * step k is lr (lr_end / lr)^(k / (steps - 1)), constant when lr_end is 0.
 * theta (device,
 * FP32) is updated in place; loss_curve (device, `steps` floats, or NULL)
 * receives each step's loss before its update. Synchronises. */
int fslbm_mlp_train(float* theta, const float* fill, const float* target, int64_t n, int64_t steps, int batch,
                    double lr, double lr_end, double lam, double mu, uint64_t seed, int augment, float* loss_curve,
                    void* cuda_stream);

/* Raw network outputs (n_x, n_y, n_z, curvature) of n stencils: theta[6212]
 * FP32, fill[n][27], out[n][4], all device memory. Synchronises. */
int fslbm_mlp_infer(const float* theta, const float* fill, int64_t n, float* out, void* cuda_stream);

/* Releases every device buffer of the run. NULL is ignored. */
void fslbm_destroy(fslbm* s);

/* Static description of an error code. */
const char* fslbm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* FSLBM_H */
