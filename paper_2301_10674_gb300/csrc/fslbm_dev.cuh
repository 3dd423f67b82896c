// Device-side definitions shared by the CUDA translation units of the
// free-surface LBM / DEM step: lattice constants, the state handed to every
// kernel, PDF storage formats, AA-pattern slot arithmetic and the cumulant
// collision (Section 2.1 of Schwarzmeier et al., "Particle-resolved simulation
// of antidunes in free-surface flows").
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fslbm.h"

namespace fsl {

constexpr int Q = 27;

// direction q = (cx+1) + 3(cy+1) + 9(cz+1)
__host__ __device__ constexpr int cx(int q) { return q % 3 - 1; }
__host__ __device__ constexpr int cy(int q) { return (q / 3) % 3 - 1; }
__host__ __device__ constexpr int cz(int q) { return q / 9 - 1; }
__host__ __device__ constexpr int opp(int q) { return 26 - q; }
__host__ __device__ constexpr int nnz(int q) {
    return (cx(q) != 0) + (cy(q) != 0) + (cz(q) != 0);
}
// D3Q27 weights: 8/27 rest, 2/27 faces, 1/54 edges, 1/216 corners
__host__ __device__ constexpr float wq(int q) {
    return nnz(q) == 0 ? 8.f / 27.f : nnz(q) == 1 ? 2.f / 27.f : nnz(q) == 2 ? 1.f / 54.f : 1.f / 216.f;
}
__host__ __device__ constexpr double wqd(int q) {
    return nnz(q) == 0 ? 8.0 / 27.0 : nnz(q) == 1 ? 2.0 / 27.0 : nnz(q) == 2 ? 1.0 / 54.0 : 1.0 / 216.0;
}

// cell flag byte
enum : uint8_t {
    T_GAS = 0, T_LIQ = 1, T_IFC = 2, T_SOL = 3, TYPE_MASK = 3,
    F_NEW = 8,       // gas cell becoming interface (filling)
    F_EMPTIED = 16,  // liquid cell becoming interface (emptying)
};
// conversion codes
enum : uint8_t { CV_TO_LIQ = 1, CV_TO_GAS = 2, CV_EVEN = 4 };

// error bits of the sticky device word (mapped to FSLBM_E* on the host)
enum : int { ERR_CAPACITY = 1, ERR_NAN = 2, ERR_INVARIANT = 4, ERR_HISTORY = 8, ERR_DISPLACEMENT = 16, ERR_TIMEOUT = 32 };

constexpr int SP_TILE = 256;     // cells per x-tile of the staged even step
constexpr int BED_SEG = 256;     // cells per x-segment of the bed kernel (one block of 128 pairs)
constexpr int WAIT_LIMIT_DEFAULT = 1 << 22;   // polls of a bounded device wait

constexpr int REDUCE_TAIL_BLOCKS = 64;   // blocks of the reduction's second level
constexpr int REDUCE_MAX_BY = 1024;   // row blocks of the lattice reduction (several rows per thread)
constexpr int HIST_SLOTS = 16;   // tangential-spring history slots per particle
constexpr int NB_SLOTS = 32;     // DEM neighbour-list slots per particle

struct Dev {
    // lattice
    int nx, ny, nz;
    int per_x, per_y, per_z;
    long long n;
    // LBM parameters
    float omega, gx, gy, gz;
    float rho_gas, eps_conv, eps_normal;
    float sigma;       // surface tension: reconstruction density rho_gas + 6 sigma kappa
    int recon_normal;
    int excess_even;   // excess mass split evenly over the receivers
    int galilean;      // Galilean-invariance correction of the second-order relaxation
    int storage;
    int link_corr;     // net moving-bounce-back injection into liquid cells taken from the pool
    int idx32;         // 27 n < 2^32: PDF element indices fit 32 bits
    int wait_limit;    // polls before a bounded device wait gives up
    // element offsets of an odd step for interior cells: the pull of
    // direction q reads f[cell + pull_off[q]], the push writes
    // f[cell + push_off[q]] (constant per launch, held in the parameter bank)
    long long pull_off[27];
    long long push_off[27];
    // PDFs (f - w), AA pattern, direction-major [27][n]; side buffer of the
    // interface cells' own post-collision PDFs (same format)
    void* f;
    void* fs;
    uint8_t* flags;
    float* mass;       // interface mass m
    float* phi;        // interface fill level
    float4* ru;        // (rho, ux, uy, uz) of the last collision, interface cells
    float4* nrm;       // interface normal used by the next step's boundary condition
    float4* nrm1;      // normal of the converting cells at the current fill levels (excess weights)
    int* owner;        // owning particle of solid cells
    uint8_t* conv;     // conversion code of interface cells (0 outside a step)
    float* exscale;    // excess mass per unit weight of converting cells
    // 16-bit storage: reference deviation delta(z) of the stored values, one
    // per z (null at FP32); a stored value is (f - w_q (1 + delta(z))) scale,
    // z that of the cell whose index the slot carries
    const float* href;
    // work lists (device counts)
    int* wl; int* wl_count; int wl_cap;        // interface cells
    int* nl; int* nl_count; int nl_cap;        // cells becoming interface this step
    int* cl; int* cl_count;                    // interface cells converting this step (capacity wl_cap)
    int* tl; int* tl_count; int tl_cap;        // particle map transitions
    int* sl; int* sl_count; int sl_cap;        // solid cells with a fluid neighbour
    int* tiles; int* tile_count;               // SP_TILE-cell x-tiles holding a liquid cell
    // particle links taken from the fluid side: the bed segments (BED_SEG-cell
    // x-ranges of a row holding a liquid cell with a solid neighbour) are
    // flagged per segment and listed for the bed kernel
    int links_fused;
    int nsegx;                                  // segments per row, ceil(nx / BED_SEG)
    uint8_t* segflag;                           // [nz][ny][nsegx]
    int* bseg; int* bseg_count;
    unsigned* fbits; unsigned* ibits; unsigned* sbits;   // per 32 cells of a row: fluid / interface / solid bits
    int* tl_info;                               // per transition: new owner / new type
    double* pool;
    double* pool_share;
    double* rpart;     // partial sums of the lattice reduction, 8 per block
    double* rtail; int* rtail_count;   // the reduction's second level: 8 sums per tail block, blocks done
    int* err;
    unsigned long long* viol;
    // particles (FP64 state)
    int np, np_cap;
    double* X; double* U; double* W;            // current state
    // DEM sub-steps in FP32 (R-25): the changes of position, velocity and
    // angular velocity since the step's start, ping-pong over the sub-steps
    // (3 per particle each); per neighbour slot the offset of the partner's
    // centre at the step's start, per particle the distances to the six wall
    // faces then, (r, m, I) and the averaged hydrodynamic force plus weight
    // and torque, all in FP32
    float* dem_dx[2]; float* dem_du[2]; float* dem_dw[2];
    float4* nb_d0;                              // [np_cap][NB_SLOTS]
    float* dem_wall;                            // [np_cap][6]: x, L_x - x, y, L_y - y, z, L_z - z
    float4* dem_c;                              // (r, m, I, 0)
    float* Faf; float* Taf;                     // [np_cap][3]
    double* R; double* M; double* I;
    uint8_t* fixed;
    float4* Xr;                                 // (X, Y, Z, r) in FP32, r < 0 for fixed spheres
    int4* Xi;                                   // floor of the centre ...
    float4* Xfr;                                // ... and the fraction, for exact FP32 link offsets
    float4* Uf; float4* Wf;                     // FP32 copies of U and Omega for the links
    double* Fh; double* Th;                     // momentum exchange of this step
    double* Fp; double* Tp;                     // previous step
    double* Fa; double* Ta;                     // two-step average
    int* nb; int* nb_count;                     // DEM neighbour list [np_cap][NB_SLOTS]
    int* hist_partner;                          // [np_cap][HIST_SLOTS]
    float* hist_xi;                             // [np_cap][HIST_SLOTS][3]
    double rho_p, restitution, friction, poisson, collision_time;
    double kn_coef, dn_coef, kt_ratio;          // contact law constants (host-computed)
    double gxd, gyd, gzd;
    int dem_substeps;
    int lub;                                    // lubrication corrections on
    double lub_mu;                              // dynamic viscosity rho nu of the liquid
    // particle grid (DEM neighbours and the particle-to-cell map)
    int gnx, gny, gnz;
    double ghx, ghy, ghz;
    int* g_count; int* g_start; int* g_cursor; int* g_list; int* g_of;
    double r_max;
    int* zmax_cell;
    // incremental re-mapping: position of the last map, margin to the nearest
    // cell centre, shared-cell flag, active particles and their cells
    double* Xm;
    float* margin;
    // learned normal: operand copies of the network (null: Parker-Youngs)
    // and counters of stencils evaluated / normals taken from the network
    const struct MlpBf16* mlp;
    unsigned long long* mlp_stats;
    // the weights in fragment order for the in-step forward pass, with the
    // first layers of the mirror images of R-17g, and whether the normal
    // averages the network over those mirror images
    const struct MlpFrag* mlp_frag;
    int mlp_mirror;
    int* shared;
    int* act; int* act_count;
    uint8_t* dirty;
    uint8_t* scratch_a; uint8_t* scratch_b;     // byte fields for the neighbourhood OR
    int* dl; int* dl_count; int dl_cap;
    // static map of the fixed particles
    unsigned long long* fixkey;
    int* fixowner;
};

// ---------------------------------------------------------------- storage
template <typename S> struct Store;
// ld/st convert to and from the deviation f - w; ld_raw/st_raw move the
// stored value times `scale` (exact power of two), for kernels that fold the
// scale into the collision
template <> struct Store<float> {
    static constexpr float scale = 1.f;
    static constexpr bool HREF = false;    // no reference: the stored value is f - w
    __device__ static __forceinline__ float ld(const float* p) { return *p; }
    __device__ static __forceinline__ void st(float* p, float v) { *p = v; }
    __device__ static __forceinline__ float ld_raw(const float* p) { return *p; }
    __device__ static __forceinline__ void st_raw(float* p, float v) { *p = v; }
};
// FP16 holds (f - w) 2^12: the scale is exact, so rounding is FP16's own
// (11 significant bits), but the normal range starts at 1.5e-8 instead of
// 6.1e-5 and deviations of slow flows do not fall into subnormals; the
// largest deviation held is 16.
constexpr float FP16_SCALE = 4096.f, FP16_UNSCALE = 1.f / 4096.f;
template <> struct Store<__half> {
    static constexpr float scale = FP16_SCALE;
    static constexpr bool HREF = true;     // relative to w (1 + delta(z)), see Dev::href
    __device__ static __forceinline__ float ld(const __half* p) { return __half2float(*p) * FP16_UNSCALE; }
    __device__ static __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v * FP16_SCALE); }
    __device__ static __forceinline__ float ld_raw(const __half* p) { return __half2float(*p); }
    __device__ static __forceinline__ void st_raw(__half* p, float v) { *p = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    static constexpr float scale = 1.f;
    static constexpr bool HREF = true;
    __device__ static __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
    __device__ static __forceinline__ float ld_raw(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static __forceinline__ void st_raw(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// w_q delta(z) of slot i = q n + cell (16-bit storage): the part of f - w
// that the stored value leaves to the reference
__device__ __forceinline__ float slot_ref(const Dev& s, long long i) {
    if (s.idx32) {   // 32-bit division where the indices fit
        const unsigned u = (unsigned)i, un = (unsigned)s.n;
        const unsigned q = u / un;
        return wq((int)q) * s.href[(u - q * un) / ((unsigned)s.nx * (unsigned)s.ny)];
    }
    const int q = (int)(i / s.n);
    const long long c = i - (long long)q * s.n;
    return wq(q) * s.href[(int)(c / ((long long)s.nx * s.ny))];
}
// f - w at PDF slot i, in any storage format
__device__ __forceinline__ float ld_any(const Dev& s, const void* base, long long i) {
    if (s.storage == FSLBM_STORE_FP32) return static_cast<const float*>(base)[i];
    if (s.storage == FSLBM_STORE_FP16) return Store<__half>::ld(static_cast<const __half*>(base) + i) + slot_ref(s, i);
    return __bfloat162float(static_cast<const __nv_bfloat16*>(base)[i]) + slot_ref(s, i);
}
__device__ __forceinline__ void st_any(const Dev& s, void* base, long long i, float v) {
    if (s.storage == FSLBM_STORE_FP32) static_cast<float*>(base)[i] = v;
    else if (s.storage == FSLBM_STORE_FP16) Store<__half>::st(static_cast<__half*>(base) + i, v - slot_ref(s, i));
    else static_cast<__nv_bfloat16*>(base)[i] = __float2bfloat16_rn(v - slot_ref(s, i));
}
// z of the slot a PDF moving in direction (.., .., dz) from a cell at z
// lands in: z + dz, wrapped on a periodic z axis (the caller has excluded
// wall faces)
__device__ __forceinline__ int wrap_z(const Dev& s, int z) { return z < 0 ? z + s.nz : (z >= s.nz ? z - s.nz : z); }

// ---------------------------------------------------------------- geometry
__host__ __device__ __forceinline__ void coords(const Dev& s, long long c, int& x, int& y, int& z) {
    x = (int)(c % s.nx);
    long long r = c / s.nx;
    y = (int)(r % s.ny);
    z = (int)(r / s.ny);
}

// the same for a cell index below 2^31 (list entries), in 32-bit arithmetic
__device__ __forceinline__ void coords32(const Dev& s, int c, int& x, int& y, int& z) {
    const unsigned u = (unsigned)c, nx = (unsigned)s.nx, ny = (unsigned)s.ny;
    const unsigned r = u / nx;
    x = (int)(u - r * nx);
    z = (int)(r / ny);
    y = (int)(r - (unsigned)z * ny);
}

// coordinate of x + d along an axis of length L: wrapped if periodic, -1 if
// it lies beyond a wall face
__device__ __forceinline__ int shift(int x, int d, int L, int periodic) {
    int v = x + d;
    if (v < 0) return periodic ? v + L : -1;
    if (v >= L) return periodic ? v - L : -1;
    return v;
}

// neighbour of (x,y,z) at offset (dx,dy,dz); -1 beyond a wall
__device__ __forceinline__ long long nbr(const Dev& s, int x, int y, int z, int dx, int dy, int dz) {
    int a = shift(x, dx, s.nx, s.per_x);
    int b = shift(y, dy, s.ny, s.per_y);
    int c = shift(z, dz, s.nz, s.per_z);
    if (a < 0 || b < 0 || c < 0) return -1;
    return (long long)a + (long long)s.nx * ((long long)b + (long long)s.ny * c);
}

// AA pattern. After an even step the post-collision PDF f*_q(x) sits in slot
// (opp(q), x); after an odd step (and initially) it sits in slot
// (q, x + c_q), or (opp(q), x) when x + c_q lies beyond a wall.
__device__ __forceinline__ long long fstar_slot(const Dev& s, int q, int x, int y, int z, long long cell,
                                                int last_parity) {
    if (last_parity == 0) return (long long)opp(q) * s.n + cell;
    long long t = nbr(s, x, y, z, cx(q), cy(q), cz(q));
    if (t < 0) return (long long)opp(q) * s.n + cell;
    return (long long)q * s.n + t;
}

// ---------------------------------------------------------------- collision
// Per-axis (chimera) transforms on deviations from the rest state: a column
// of three values (c = -1, 0, +1) with rest part (1/6, 2/3, 1/6) R has
// moments (k0, k1, k2) about u with rest part (R, 0, R/3); only deviations
// are carried, so FP32 resolves them to their own precision.
// Backward per-axis transform of one line: (k0, k1, k2) are the zeroth,
// first and second moments about u of the deviations, R the rest value of
// the zeroth moment (K = R + k0 the full one). With the per-axis
// coefficients A = (u^2 - u)/2, B = u - 1/2, C = (u^2 + u)/2, D = u + 1/2:
// f_-1 = A K + B k1 + k2/2, f_+1 = C K + D k1 + k2/2, and, since the three
// values sum to the zeroth moment of the deviations, f_0 = k0 - f_-1 - f_+1.
struct AxisCoef {
    float A, B, C, D;
};
__device__ __forceinline__ AxisCoef axis_coef(float u) {
    const float uu = u * u;
    return {0.5f * (uu - u), u - 0.5f, 0.5f * (uu + u), u + 0.5f};
}
__device__ __forceinline__ void bwd_axis(float& a, float& b, float& c, const AxisCoef& w, float R) {
    const float k0 = a, k1 = b, k2 = c;
    const float K = R + k0;
    const float h = 0.5f * k2;
    const float lo = fmaf(w.A, K, fmaf(w.B, k1, h));
    const float hi = fmaf(w.C, K, fmaf(w.D, k1, h));
    a = lo;
    c = hi;
    b = k0 - lo - hi;
}

__device__ __forceinline__ float w1(int i) { return i == 1 ? 2.f / 3.f : 1.f / 6.f; }
__device__ __forceinline__ float mrest(int i) { return i == 0 ? 1.f : (i == 1 ? 0.f : 1.f / 3.f); }

// D3Q27 cumulant collision on f - w (in place). All relaxation rates are 1
// except omega for the shear parts of the second-order moments; the trace
// relaxes to rho; orders 3..6 take the Gaussian closure (all higher
// cumulants zero); the body force rho g enters through the half-shifted
// velocity and the sign flip of the first-order central moments. Returns
// rho and u (the collision velocity).
//
// Only rho, the momentum and the six second-order central moments survive
// the collision. Their raw sums (of the deviations) come from the per-axis
// (chimera) forward transform pruned to orders <= 2; the central moments
// follow as kappa_ab = Pi_ab - u_a j_b - u_b j_a + rho u_a u_b (diagonal
// relative to its rest value 1/3). The post-collision central moments go
// back through the per-axis backward transform.
//
// f may hold the deviations times an exact power of two `scale` (the FP16
// storage scale): the forward sums are unscaled once, and the backward
// transform, which is linear in the moments and the rest values, produces
// scaled values again.
//
// With gal, the Galilean-invariance correction of Geier et al. (2015): the
// diagonal velocity gradients follow from the non-equilibrium second-order
// moments (shear rate omega, bulk rate 1), d_x u_x = -omega/(2 rho)
// (2 k_xx - k_yy - k_zz) - (k_xx + k_yy + k_zz - (rho - 1))/(2 rho) in the
// deviation variables, d_y u_y = d_x u_x + 3 omega/(2 rho) (k_xx - k_yy),
// likewise z; the relaxed normal-stress differences lose 3 rho (1 - omega/2)
// (u_x^2 d_x u_x - u_y^2 d_y u_y) (and z), the trace 3 rho / 2 (u_x^2 d_x u_x
// + u_y^2 d_y u_y + u_z^2 d_z u_z).
__device__ __forceinline__ void collide_scaled(float (&f)[27], float scale, float omega, float gx, float gy,
                                               float gz, float& rho_out, float& ux_out, float& uy_out,
                                               float& uz_out, bool gal = false) {
    // x: per (b, c) line the sum, first and second raw moments
    float X0[9], X1[9], X2[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const float a = f[3 * l], b = f[3 * l + 1], c = f[3 * l + 2];
        const float t = a + c;
        X0[l] = t + b;
        X1[l] = c - a;
        X2[l] = t;
    }
    // y (line index l = b + 3c): only the combinations of total order <= 2
    float Y00[3], Y01[3], Y02[3], Y10[3], Y11[3], Y20[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float t0 = X0[3 * c] + X0[3 * c + 2];
        Y00[c] = t0 + X0[3 * c + 1];
        Y01[c] = X0[3 * c + 2] - X0[3 * c];
        Y02[c] = t0;
        Y10[c] = X1[3 * c] + X1[3 * c + 1] + X1[3 * c + 2];
        Y11[c] = X1[3 * c + 2] - X1[3 * c];
        Y20[c] = X2[3 * c] + X2[3 * c + 1] + X2[3 * c + 2];
    }
    // z
    const float inv_scale = 1.f / scale;
    const float tz = Y00[0] + Y00[2];
    const float drho = (tz + Y00[1]) * inv_scale;
    const float jz = (Y00[2] - Y00[0]) * inv_scale;
    const float pzz = tz * inv_scale;
    const float jy = (Y01[0] + Y01[1] + Y01[2]) * inv_scale;
    const float pyz = (Y01[2] - Y01[0]) * inv_scale;
    const float jx = (Y10[0] + Y10[1] + Y10[2]) * inv_scale;
    const float pxz = (Y10[2] - Y10[0]) * inv_scale;
    const float pyy = (Y02[0] + Y02[1] + Y02[2]) * inv_scale;
    const float pxy = (Y11[0] + Y11[1] + Y11[2]) * inv_scale;
    const float pxx = (Y20[0] + Y20[1] + Y20[2]) * inv_scale;

    const float rho = 1.f + drho;
    const float inv = 1.f / rho;
    const float Fx = rho * gx, Fy = rho * gy, Fz = rho * gz;
    const float ux = (jx + 0.5f * Fx) * inv;
    const float uy = (jy + 0.5f * Fy) * inv;
    const float uz = (jz + 0.5f * Fz) * inv;
    // central second-order moments (deviations of the diagonal from 1/3)
    const float kxx = pxx - 2.f * ux * jx + rho * ux * ux;
    const float kyy = pyy - 2.f * uy * jy + rho * uy * uy;
    const float kzz = pzz - 2.f * uz * jz + rho * uz * uz;
    const float kxy = pxy - ux * jy - uy * jx + rho * ux * uy;
    const float kxz = pxz - ux * jz - uz * jx + rho * ux * uz;
    const float kyz = pyz - uy * jz - uz * jy + rho * uy * uz;
    // m[a + 3b + 9c]: post-collision central-moment deviation of orders (a, b, c)
    const float om1 = 1.f - omega;
    float Dxy = om1 * (kxx - kyy);
    float Dxz = om1 * (kxx - kzz);
    float trace = drho;   // relaxed trace less 1 (rate 1: rho - 1)
    if (gal) {
        const float dxu = -omega * 0.5f * inv * (2.f * kxx - kyy - kzz) - 0.5f * inv * (kxx + kyy + kzz - drho);
        const float dyv = dxu + 1.5f * omega * inv * (kxx - kyy);
        const float dzw = dxu + 1.5f * omega * inv * (kxx - kzz);
        const float ax = ux * ux * dxu, ay = uy * uy * dyv, az = uz * uz * dzw;
        const float c1 = 3.f * rho * (1.f - 0.5f * omega);
        Dxy -= c1 * (ax - ay);
        Dxz -= c1 * (ax - az);
        trace -= 1.5f * rho * (ax + ay + az);
    }
    const float k200 = (Dxy + Dxz + trace) * (1.f / 3.f);
    const float k020 = (Dxz - 2.f * Dxy + trace) * (1.f / 3.f);
    const float k002 = (Dxy - 2.f * Dxz + trace) * (1.f / 3.f);
    const float k110 = om1 * kxy;
    const float k101 = om1 * kxz;
    const float k011 = om1 * kyz;
    const float sxx = (k200 - drho * (1.f / 3.f)) * inv;
    const float syy = (k020 - drho * (1.f / 3.f)) * inv;
    const float szz = (k002 - drho * (1.f / 3.f)) * inv;
    const float Sxy = k110 * inv, Sxz = k101 * inv, Syz = k011 * inv;
    const float third = 1.f / 3.f;
    const float rs = rho * scale;
    f[0] = drho * scale;
    f[1] = 0.5f * Fx * scale;
    f[3] = 0.5f * Fy * scale;
    f[9] = 0.5f * Fz * scale;
    f[2] = k200 * scale; f[6] = k020 * scale; f[18] = k002 * scale;
    f[4] = k110 * scale; f[10] = k101 * scale; f[12] = k011 * scale;
    f[5] = f[11] = f[7] = f[15] = f[19] = f[21] = f[13] = 0.f;
    f[8] = drho * (scale / 9.f) + rs * ((sxx + syy) * third + sxx * syy + 2.f * Sxy * Sxy);
    f[20] = drho * (scale / 9.f) + rs * ((sxx + szz) * third + sxx * szz + 2.f * Sxz * Sxz);
    f[24] = drho * (scale / 9.f) + rs * ((syy + szz) * third + syy * szz + 2.f * Syz * Syz);
    f[14] = rs * ((third + sxx) * Syz + 2.f * Sxy * Sxz);
    f[16] = rs * ((third + syy) * Sxz + 2.f * Sxy * Syz);
    f[22] = rs * ((third + szz) * Sxy + 2.f * Sxz * Syz);
    f[17] = f[23] = f[25] = 0.f;
    f[26] = drho * (scale / 27.f)
            + rs * ((sxx + syy + szz) * (1.f / 9.f) + (sxx * syy + sxx * szz + syy * szz) * third
                    + sxx * syy * szz
                    + 2.f * ((third + sxx) * Syz * Syz + (third + syy) * Sxz * Sxz + (third + szz) * Sxy * Sxy)
                    + 8.f * Sxy * Sxz * Syz);
    // backward: x, then y, then z (rest values scaled with the moments)
    const AxisCoef wx = axis_coef(ux), wy = axis_coef(uy), wz = axis_coef(uz);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            bwd_axis(f[3 * b + 9 * c], f[1 + 3 * b + 9 * c], f[2 + 3 * b + 9 * c], wx,
                     scale * mrest(b) * mrest(c));
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            bwd_axis(f[a + 9 * c], f[a + 3 + 9 * c], f[a + 6 + 9 * c], wy, scale * w1(a) * mrest(c));
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            bwd_axis(f[a + 3 * b], f[a + 3 * b + 9], f[a + 3 * b + 18], wz, scale * w1(a) * w1(b));
    rho_out = rho;
    ux_out = ux;
    uy_out = uy;
    uz_out = uz;
}

__device__ __forceinline__ void collide(float (&f)[27], float omega, float gx, float gy, float gz,
                                        float& rho_out, float& ux_out, float& uy_out, float& uz_out) {
    collide_scaled(f, 1.f, omega, gx, gy, gz, rho_out, ux_out, uy_out, uz_out);
}

// second-order equilibrium minus the weight: w_q [(rho - 1) + rho (3 cu +
// 9/2 cu^2 - 3/2 u^2)]
__device__ __forceinline__ float feq_dev(int q, float rho, float ux, float uy, float uz) {
    float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
    float uu = ux * ux + uy * uy + uz * uz;
    return wq(q) * ((rho - 1.f) + rho * (3.f * cu + 4.5f * cu * cu - 1.5f * uu));
}

__device__ __forceinline__ void set_error(const Dev& s, int bit) { atomicOr(s.err, bit); }

// byte-granular atomic OR on the flag array; returns the previous byte
__device__ __forceinline__ uint8_t flag_or(uint8_t* flags, long long i, uint8_t bits) {
    uintptr_t addr = reinterpret_cast<uintptr_t>(flags + i);
    unsigned int* word = reinterpret_cast<unsigned int*>(addr & ~uintptr_t(3));
    unsigned int sh = 8u * (unsigned int)(addr & 3);
    unsigned int old = atomicOr(word, (unsigned int)bits << sh);
    return (uint8_t)((old >> sh) & 0xffu);
}

// Block-aggregated append to a device list: one atomic per block. Every
// thread of the block must call it (it synchronises the block); blockDim.x
// must be a multiple of 32 and at most 1024. Returns the slot written, or -1.
__device__ __forceinline__ int block_append(const Dev& s, bool pred, int v, int* list, int* count, int cap) {
    __shared__ int warp_n[32];
    __shared__ int block_base;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(full, pred);
    if (lane == 0) warp_n[wid] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int c = warp_n[w];
            warp_n[w] = tot;
            tot += c;
        }
        block_base = tot ? atomicAdd(count, tot) : 0;
    }
    __syncthreads();
    int slot = -1;
    if (pred) {
        const int k = block_base + warp_n[wid] + __popc(m & ((1u << lane) - 1u));
        if (k < cap) {
            list[k] = v;
            slot = k;
        } else {
            set_error(s, ERR_CAPACITY);
        }
    }
    __syncthreads();
    return slot;
}

// Warp-aggregated append: one atomic per warp. Every lane of the warp must
// call it.
__device__ __forceinline__ void warp_append(const Dev& s, bool pred, int v, int* list, int* count, int cap) {
    const unsigned full = 0xffffffffu;
    const unsigned m = __ballot_sync(full, pred);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(full, base, leader);
    if (pred) {
        const int k = base + __popc(m & ((1u << lane) - 1u));
        if (k < cap) list[k] = v;
        else set_error(s, ERR_CAPACITY);
    }
}

// post-collision PDFs of a cell read from the AA layout (outside the
// stream-collide kernel, where no slot is being rewritten)
__device__ __forceinline__ void load_fstar(const Dev& s, long long cell, int last_parity, float (&f)[27]) {
    int x, y, z;
    coords(s, cell, x, y, z);
#pragma unroll
    for (int q = 0; q < 27; ++q) f[q] = ld_any(s, s.f, fstar_slot(s, q, x, y, z, cell, last_parity));
}
__device__ __forceinline__ void store_fstar(const Dev& s, long long cell, int last_parity, const float (&f)[27]) {
    int x, y, z;
    coords(s, cell, x, y, z);
#pragma unroll
    for (int q = 0; q < 27; ++q) st_any(s, s.f, fstar_slot(s, q, x, y, z, cell, last_parity), f[q]);
}
// density and collision velocity from post-collision PDFs (f - w):
// rho = 1 + sum, u = (sum c f* - rho g / 2) / rho
__device__ __forceinline__ void post_moments(const Dev& s, const float (&f)[27], float& rho, float& ux, float& uy,
                                             float& uz) {
    float d = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        d += f[q];
        jx += cx(q) * f[q];
        jy += cy(q) * f[q];
        jz += cz(q) * f[q];
    }
    rho = 1.f + d;
    float inv = 1.f / rho;
    ux = (jx - 0.5f * rho * s.gx) * inv;
    uy = (jy - 0.5f * rho * s.gy) * inv;
    uz = (jz - 0.5f * rho * s.gz) * inv;
}

// ---------------------------------------------------------------- launchers
// (defined in the translation units, called from the host orchestration)
// launchers used inside a time step return the number of kernels enqueued
// links_done (may be null) is recorded on st once the particle forces of the
// step are complete: after the link pass, or after the sweep with fluid-side
// links
int launch_stream_collide(const Dev& s, int parity, cudaStream_t st, cudaEvent_t links_done);
int launch_classify(const Dev& s, cudaStream_t st);
void launch_check_invariant(const Dev& s, cudaStream_t st);
int launch_normals(const Dev& s, float4* out, cudaStream_t st);
void launch_log_stencils(const Dev& s, long long cap, float* fill, float* target, float* fd, int* cells,
                         unsigned long long* found, cudaStream_t st);
int launch_conversion(const Dev& s, int last_parity, cudaStream_t st);
int launch_pool_spread(const Dev& s, cudaStream_t st);
void launch_cell_counts(const Dev& s, unsigned long long* out, cudaStream_t st);
void launch_init_flat(const Dev& s, double H, cudaStream_t st);
void launch_init_surface(const Dev& s, const double* H, cudaStream_t st);
int launch_dem(const Dev& s, int have_prev, cudaStream_t st);
int launch_remap(const Dev& s, int last_parity, cudaStream_t st);
void launch_particles_add(const Dev& s, int first, int count, cudaStream_t st);
void launch_particle_copies(const Dev& s, cudaStream_t st);
int launch_grid_build(const Dev& s, cudaStream_t st);
void launch_export(const Dev& s, int last_parity, uint32_t which, double* out, cudaStream_t st);
void launch_export_type(const Dev& s, uint8_t* out, cudaStream_t st);
void launch_import_pdf(const Dev& s, int last_parity, const double* in, cudaStream_t st);
void launch_import_mass(const Dev& s, const double* in, cudaStream_t st);
void launch_reduce(const Dev& s, int last_parity, double* out, cudaStream_t st);
int reduce_blocks(const Dev& s);

inline int blocks_for(long long n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace fsl
