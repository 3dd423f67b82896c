// Geometrically resolved spheres (Section 2.2): two-step averaging of the
// momentum-exchange force, DEM sub-steps (linear spring-dashpot contacts
// parameterised by the restitution coefficient and the collision time,
// tangential spring with Coulomb limit, walls, gravity; semi-implicit
// Newton-Euler), the particle grid, and the particle-to-cell map with the
// cells it covers and uncovers. Particle state and forces are FP64; the map
// test is evaluated in FP64 without fused multiply-add so that cell types do
// not depend on contraction choices.
#include <limits.h>

#include "fslbm_dev.cuh"

namespace fsl {

constexpr int HIST_EMPTY = INT_MIN;

// ------------------------------------------------------------ particle grid
__device__ __forceinline__ int gcoord(double v, double h, int g) {
    int k = (int)floor(v / h);
    return k < 0 ? 0 : (k >= g ? g - 1 : k);
}

__global__ void k_grid_count(Dev s) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.np) return;
    int a = gcoord(s.X[3 * p], s.ghx, s.gnx);
    int b = gcoord(s.X[3 * p + 1], s.ghy, s.gny);
    int c = gcoord(s.X[3 * p + 2], s.ghz, s.gnz);
    int g = a + s.gnx * (b + s.gny * c);
    s.g_of[p] = g;
    atomicAdd(&s.g_count[g], 1);
}

// exclusive scan of the grid counts by one block of 32 warps: warp w owns a
// contiguous chunk, read 32 counts at a time (coalesced); its total joins a
// scan of the 32 warp totals, then the warp scans its chunk from that offset
__global__ void __launch_bounds__(1024) k_grid_scan(Dev s, int G) {
    __shared__ int wtot[32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rows = (G + 31) / 32;                    // rows of 32 counts
    const int per = (rows + 31) / 32;                  // rows per warp
    const int r0 = warp * per, r1 = min(rows, r0 + per);
    int sum = 0;
    for (int r = r0; r < r1; ++r) {
        const int i = 32 * r + lane;
        sum += i < G ? s.g_count[i] : 0;
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(full, sum, o);
    if (lane == 0) wtot[warp] = sum;
    __syncthreads();
    if (warp == 0) {
        int v = wtot[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(full, v, o);
            if (lane >= o) v += u;
        }
        wtot[lane] = v - wtot[lane];                   // exclusive
    }
    __syncthreads();
    int run = wtot[warp];
    for (int r = r0; r < r1; ++r) {
        const int i = 32 * r + lane;
        const int c = i < G ? s.g_count[i] : 0;
        int v = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(full, v, o);
            if (lane >= o) v += u;
        }
        if (i < G) {
            s.g_start[i] = run + v - c;
            s.g_cursor[i] = run + v - c;
        }
        run += __shfl_sync(full, v, 31);
    }
}

__global__ void k_grid_fill(Dev s) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.np) return;
    int pos = atomicAdd(&s.g_cursor[s.g_of[p]], 1);
    s.g_list[pos] = p;
}

// particles of a grid cell in index order (deterministic summation order)
__global__ void k_grid_sort(Dev s, int G) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    int b = s.g_start[g], e = b + s.g_count[g];
    for (int i = b + 1; i < e; ++i) {
        int v = s.g_list[i];
        int j = i - 1;
        while (j >= b && s.g_list[j] > v) {
            s.g_list[j + 1] = s.g_list[j];
            --j;
        }
        s.g_list[j + 1] = v;
    }
}

int launch_grid_build(const Dev& s, cudaStream_t st) {
    const int G = s.gnx * s.gny * s.gnz;
    cudaMemsetAsync(s.g_count, 0, sizeof(int) * G, st);
    k_grid_count<<<blocks_for(s.np, 128), 128, 0, st>>>(s);
    k_grid_scan<<<1, 1024, 0, st>>>(s, G);
    k_grid_fill<<<blocks_for(s.np, 128), 128, 0, st>>>(s);
    k_grid_sort<<<blocks_for(G, 128), 128, 0, st>>>(s, G);
    return 4;
}

// distinct grid coordinates within [k0, k1] along one axis
struct GRange {
    int v[3];
    int n;
};
__device__ __forceinline__ GRange grange(int k0, int k1, int g, int periodic) {
    GRange r;
    r.n = 0;
    if (periodic && k1 - k0 + 1 >= g) {
        for (int k = 0; k < g && r.n < 3; ++k) r.v[r.n++] = k;
        return r;
    }
    for (int k = k0; k <= k1 && r.n < 3; ++k) {
        int kk = k;
        if (kk < 0 || kk >= g) {
            if (!periodic) continue;
            kk = (kk % g + g) % g;
        }
        r.v[r.n++] = kk;
    }
    return r;
}

// ------------------------------------------------------------ DEM
__global__ void k_force_avg(Dev s, int have_prev) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 3 * s.np) return;
    double fh = s.Fh[k], th = s.Th[k];
    const double fa = have_prev ? 0.5 * (fh + s.Fp[k]) : fh;
    const double ta = have_prev ? 0.5 * (th + s.Tp[k]) : th;
    s.Fa[k] = fa;
    s.Ta[k] = ta;
    s.Fp[k] = fh;
    s.Tp[k] = th;
    // the sub-steps' FP32 copies: averaged hydrodynamic force plus the weight
    const int a = k % 3;
    const double g = a == 0 ? s.gxd : (a == 1 ? s.gyd : s.gzd);
    s.Faf[k] = (float)(fa + s.M[k / 3] * g);
    s.Taf[k] = (float)ta;
}

// The history slot of a partner among the particle's slots held in
// registers: its own, else the first empty one, whose spring starts at zero;
// -1 (and the sticky history bit) when none is left.
__device__ __forceinline__ int hist_slot(const Dev& s, int p, int partner, int (&hpart)[HIST_SLOTS],
                                         unsigned& seen) {
    int found = -1, freeslot = -1;
#pragma unroll
    for (int k = 0; k < HIST_SLOTS; ++k) {
        if (hpart[k] == partner && found < 0) found = k;
        if (hpart[k] == HIST_EMPTY && freeslot < 0) freeslot = k;
    }
    if (found < 0) {
        if (freeslot < 0) {
            set_error(s, ERR_HISTORY);
            return -1;
        }
        found = freeslot;
#pragma unroll
        for (int k = 0; k < HIST_SLOTS; ++k)
            if (k == found) hpart[k] = partner;
        float* xi = s.hist_xi + ((long long)p * HIST_SLOTS + found) * 3;
        xi[0] = xi[1] = xi[2] = 0.f;
    }
    seen |= 1u << found;
    return found;
}

// minimal image of an integer displacement along a periodic axis
__device__ __forceinline__ int wrap_int(int d, int L, int periodic) {
    if (periodic) {
        if (d > L / 2) d -= L;
        else if (d < -L / 2) d += L;
    }
    return d;
}

// minimal image of a displacement along a periodic axis (|d| < 1.5 L)
__device__ __forceinline__ double wrapd(double d, int L, int periodic) {
    if (periodic) {
        const double h = 0.5 * L;
        if (d > h) d -= L;
        else if (d < -h) d += L;
    }
    return d;
}
__device__ __forceinline__ float wrapf(float d, int L, int periodic) {
    if (periodic) {
        const float h = 0.5f * L;
        if (d > h) d -= L;
        else if (d < -h) d += L;
    }
    return d;
}

// Lubrication corrections (Section 2.2): the paper augments the DEM with
// normal and tangential lubrication forces where a gap is too small for the
// lattice to resolve and gives no formula. These are the asymptotic
// resistances of two nearly touching spheres with effective radius R,
// normal 6 pi mu R^2 / h and tangential 6 pi mu R (8/15) ln(1 / h), each less
// its value at the resolved gap h_c = 2/3 cell, with h clamped at 1e-2.
constexpr float LUB_HC = 2.f / 3.f, LUB_HMIN = 1e-2f;
// force on the particle (n toward the partner or wall, vrel the relative
// velocity of the surfaces at the contact point) and its tangential part
__device__ __forceinline__ void lub_f(const Dev& s, float R, const float n[3], float h, const float vrel[3],
                                      float Fl[3], float Ft[3]) {
    const float hh = fmaxf(h, LUB_HMIN);
    const float vn = vrel[0] * n[0] + vrel[1] * n[1] + vrel[2] * n[2];
    const float k = 6.f * 3.14159265f * (float)s.lub_mu * R;
    const float cn = k * R * (1.f / hh - 1.f / LUB_HC);
    const float ct = k * (8.f / 15.f) * logf(LUB_HC / hh);
    for (int a = 0; a < 3; ++a) {
        Ft[a] = -ct * (vrel[a] - vn * n[a]);
        Fl[a] = -cn * vn * n[a] + Ft[a];
    }
}

// a partner of p for the neighbour list: surfaces within 3/4 cell
__device__ __forceinline__ bool dem_partner(const Dev& s, int p, int j, const float4& xri) {
    if (j == p) return false;
    const float4 xrj = s.Xr[j];
    const float ex = wrapf(xrj.x - xri.x, s.nx, s.per_x), ey = wrapf(xrj.y - xri.y, s.ny, s.per_y),
                ez = wrapf(xrj.z - xri.z, s.nz, s.per_z);
    const float reach = fabsf(xri.w) + fabsf(xrj.w) + 0.75f;
    return ex * ex + ey * ey + ez * ez <= reach * reach;
}

// Neighbour list of every mobile particle for the sub-steps of one LBM
// step: particles whose surfaces are within 3/4 cell (beyond the
// lubrication range; the motion within a step is far below the margin).
// With it the FP32 start of the sub-steps (R-25): per neighbour slot the
// partner's centre offset, per mobile particle the distances to the wall
// faces, and zero changes of position, velocity and angular velocity.
// A warp per particle: lane t scans grid cell t of the (up to) 3x3x3 cells
// around the particle's, in the order (z, y, x) of the cells and of the
// particles within a cell; the accepted partners are compacted into the
// slots in that order (a warp prefix sum over the lanes' counts).
__global__ void k_dem_neighbours(Dev s) {
    const unsigned full = 0xffffffffu;
    const int p = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (p >= s.np) return;   // whole warps leave together
    if (lane < 3) s.dem_dx[0][3 * p + lane] = s.dem_du[0][3 * p + lane] = s.dem_dw[0][3 * p + lane] = 0.f;
    if (s.fixed[p]) {
        if (lane == 0) s.nb_count[p] = 0;
        return;
    }
    // offsets from the integer part and the FP32 fraction of the centres
    // (exact integer differences, minimal image on periodic axes): exact to
    // FP32 rounding and antisymmetric between the two partners
    const int4 ip = s.Xi[p];
    const float4 fp = s.Xfr[p];
    if (lane == 0) {
        s.dem_wall[6 * p + 0] = (float)ip.x + fp.x;
        s.dem_wall[6 * p + 1] = (float)(s.nx - ip.x) - fp.x;
        s.dem_wall[6 * p + 2] = (float)ip.y + fp.y;
        s.dem_wall[6 * p + 3] = (float)(s.ny - ip.y) - fp.y;
        s.dem_wall[6 * p + 4] = (float)ip.z + fp.z;
        s.dem_wall[6 * p + 5] = (float)(s.nz - ip.z) - fp.z;
    }
    const float4 xri = s.Xr[p];
    const int g = s.g_of[p];
    const int ga = g % s.gnx, gb = (g / s.gnx) % s.gny, gc = g / (s.gnx * s.gny);
    const GRange ra = grange(ga - 1, ga + 1, s.gnx, s.per_x);
    const GRange rb = grange(gb - 1, gb + 1, s.gny, s.per_y);
    const GRange rc = grange(gc - 1, gc + 1, s.gnz, s.per_z);
    const int ncell = ra.n * rb.n * rc.n;
    int b = 0, e = 0;
    if (lane < ncell) {
        const int ia = lane % ra.n, ib = (lane / ra.n) % rb.n, ic = lane / (ra.n * rb.n);
        const int gg = ra.v[ia] + s.gnx * (rb.v[ib] + s.gny * rc.v[ic]);
        b = s.g_start[gg];
        e = b + s.g_count[gg];
    }
    int mine = 0;
    for (int k = b; k < e; ++k) mine += dem_partner(s, p, s.g_list[k], xri) ? 1 : 0;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(full, incl, 31);
    int slot = incl - mine;
    for (int k = b; k < e; ++k) {
        const int j = s.g_list[k];
        if (!dem_partner(s, p, j, xri)) continue;
        if (slot < NB_SLOTS) {
            s.nb[(long long)p * NB_SLOTS + slot] = j;
            const int4 ij = s.Xi[j];
            const float4 fj = s.Xfr[j];
            s.nb_d0[(long long)p * NB_SLOTS + slot] =
                make_float4((float)wrap_int(ij.x - ip.x, s.nx, s.per_x) + (fj.x - fp.x),
                            (float)wrap_int(ij.y - ip.y, s.ny, s.per_y) + (fj.y - fp.y),
                            (float)wrap_int(ij.z - ip.z, s.nz, s.per_z) + (fj.z - fp.z), 0.f);
        }
        ++slot;
    }
    if (lane == 0) {
        if (total > NB_SLOTS) set_error(s, ERR_HISTORY);
        s.nb_count[p] = total > NB_SLOTS ? NB_SLOTS : total;
    }
}

// FP32 copies of the particle state used by the lattice kernels
__global__ void k_particle_copies(Dev s) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.np) return;
    const double X = s.X[3 * p], Y = s.X[3 * p + 1], Z = s.X[3 * p + 2];
    const double r = s.R[p];
    s.Xr[p] = make_float4((float)X, (float)Y, (float)Z, s.fixed[p] ? -(float)r : (float)r);
    const double fx = floor(X), fy = floor(Y), fz = floor(Z);
    s.Xi[p] = make_int4((int)fx, (int)fy, (int)fz, 0);
    s.Xfr[p] = make_float4((float)(X - fx), (float)(Y - fy), (float)(Z - fz), 0.f);
    s.Uf[p] = make_float4((float)s.U[3 * p], (float)s.U[3 * p + 1], (float)s.U[3 * p + 2], 0.f);
    s.Wf[p] = make_float4((float)s.W[3 * p], (float)s.W[3 * p + 1], (float)s.W[3 * p + 2], 0.f);
    s.dem_c[p] = make_float4((float)r, (float)s.M[p], (float)s.I[p], 0.f);
}

void launch_particle_copies(const Dev& s, cudaStream_t st) {
    if (s.np > 0) k_particle_copies<<<blocks_for(s.np, 128), 128, 0, st>>>(s);
}

// FP32 linear spring-dashpot with tangential history (same law as above)
__device__ void contact_f(const Dev& s, float meff, const float n[3], float delta, const float vrel[3], float* xi,
                          float dts, float F[3], float Ft[3]) {
    const float kn = meff * (float)s.kn_coef;
    const float dn = meff * (float)s.dn_coef;
    const float kt = kn * (float)s.kt_ratio;
    const float dt_ = dn;
    const float vn = vrel[0] * n[0] + vrel[1] * n[1] + vrel[2] * n[2];
    const float vt[3] = {vrel[0] - vn * n[0], vrel[1] - vn * n[1], vrel[2] - vn * n[2]};
    const float fn = kn * delta + dn * vn;
    float x[3] = {xi[0], xi[1], xi[2]};
    const float xn = x[0] * n[0] + x[1] * n[1] + x[2] * n[2];
    for (int a = 0; a < 3; ++a) x[a] = x[a] - xn * n[a] + vt[a] * dts;
    for (int a = 0; a < 3; ++a) Ft[a] = -kt * x[a] - dt_ * vt[a];
    const float ftl = sqrtf(Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2]);
    const float lim = (float)s.friction * fabsf(fn);
    if (ftl > lim && ftl > 0.f) {
        const float sc = lim / ftl;
        for (int a = 0; a < 3; ++a) {
            Ft[a] *= sc;
            x[a] = -(Ft[a] + dt_ * vt[a]) / kt;
        }
    }
    for (int a = 0; a < 3; ++a) {
        xi[a] = x[a];
        F[a] = -fn * n[a] + Ft[a];
    }
}

// One DEM sub-step, a thread per particle over its neighbour list and the
// walls, in FP32 (R-25): a particle's position, velocity and angular velocity
// are its FP64 state at the step's start plus the changes dx, du, dw the
// sub-steps have made (small numbers, exact to FP32 rounding of themselves);
// the offset to a partner is the start offset (formed in FP64 with the
// neighbour list) plus the difference of their dx, a wall distance the start
// distance plus or minus dx. Contact law and sums in FP32, semi-implicit
// Euler on the changes; the last sub-step adds them to the FP64 state.
__global__ void __launch_bounds__(64) k_dem_substep(Dev s, const float* __restrict__ dxa,
                                                   const float* __restrict__ dua, const float* __restrict__ dwa,
                                                   float* dxb, float* dub, float* dwb, float dts, int last) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.np) return;
    const float dx[3] = {dxa[3 * p], dxa[3 * p + 1], dxa[3 * p + 2]};
    const float du[3] = {dua[3 * p], dua[3 * p + 1], dua[3 * p + 2]};
    const float dw[3] = {dwa[3 * p], dwa[3 * p + 1], dwa[3 * p + 2]};
    if (s.fixed[p]) {
        for (int a = 0; a < 3; ++a) { dxb[3 * p + a] = dx[a]; dub[3 * p + a] = du[a]; dwb[3 * p + a] = dw[a]; }
        // the top of the particle cells counts the fixed particles too
        if (last) atomicMax(s.zmax_cell, (int)ceil(s.X[3 * p + 2] + s.R[p]) + 2);
        return;
    }
    const float4 cp = s.dem_c[p];
    const float rif = cp.x, mif = cp.y, Iif = cp.z;
    const float4 u0 = s.Uf[p], w0 = s.Wf[p];
    const float Uf[3] = {u0.x + du[0], u0.y + du[1], u0.z + du[2]};
    const float Wf[3] = {w0.x + dw[0], w0.y + dw[1], w0.z + dw[2]};
    float F[3] = {s.Faf[3 * p], s.Faf[3 * p + 1], s.Faf[3 * p + 2]};
    float T[3] = {s.Taf[3 * p], s.Taf[3 * p + 1], s.Taf[3 * p + 2]};
    unsigned seen = 0;
    // the particle's tangential-history partners, held in registers for the
    // sub-step (slot k: partner index, a wall code, or HIST_EMPTY)
    int hpart[HIST_SLOTS];
    {
        const int4* hp4 = reinterpret_cast<const int4*>(s.hist_partner + (long long)p * HIST_SLOTS);
#pragma unroll
        for (int k = 0; k < HIST_SLOTS / 4; ++k) {
            const int4 v = hp4[k];
            hpart[4 * k] = v.x; hpart[4 * k + 1] = v.y; hpart[4 * k + 2] = v.z; hpart[4 * k + 3] = v.w;
        }
    }
    const int nbc = s.nb_count[p];
    const int* nbl = s.nb + (long long)p * NB_SLOTS;
    const float4* nd0 = s.nb_d0 + (long long)p * NB_SLOTS;
    // neighbours four at a time: their indices, offsets and changes load together
    for (int k0 = 0; k0 < nbc; k0 += 4) {
        int jj[4];
        float4 d0[4], cj[4];
        float dxj[4][3];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            jj[u] = k0 + u < nbc ? nbl[k0 + u] : -1;
            d0[u] = k0 + u < nbc ? nd0[k0 + u] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            cj[u] = jj[u] >= 0 ? s.dem_c[jj[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int a = 0; a < 3; ++a) dxj[u][a] = jj[u] >= 0 ? dxa[3 * jj[u] + a] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = jj[u];
            if (j < 0) continue;
            const float d[3] = {d0[u].x + (dxj[u][0] - dx[0]), d0[u].y + (dxj[u][1] - dx[1]),
                                d0[u].z + (dxj[u][2] - dx[2])};
            const float rjf = cj[u].x;
            const float dist2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            const float rs = rif + rjf;
            const bool touch = dist2 < rs * rs;
            const bool lub = s.lub && dist2 < (rs + LUB_HC) * (rs + LUB_HC);
            if (!touch && !lub) continue;
            const float dist = sqrtf(dist2);
            const float inv = 1.f / dist;
            const float n[3] = {d[0] * inv, d[1] * inv, d[2] * inv};
            const float delta = rs - dist;
            const float4 uj0 = s.Uf[j], wj0 = s.Wf[j];
            const float Uj[3] = {uj0.x + dua[3 * j], uj0.y + dua[3 * j + 1], uj0.z + dua[3 * j + 2]};
            const float Wj[3] = {wj0.x + dwa[3 * j], wj0.y + dwa[3 * j + 1], wj0.z + dwa[3 * j + 2]};
            float wsum[3];
            for (int a = 0; a < 3; ++a) wsum[a] = rif * Wf[a] + rjf * Wj[a];
            const float wn[3] = {wsum[1] * n[2] - wsum[2] * n[1], wsum[2] * n[0] - wsum[0] * n[2],
                                 wsum[0] * n[1] - wsum[1] * n[0]};
            float vrel[3];
            for (int a = 0; a < 3; ++a) vrel[a] = Uf[a] - Uj[a] + wn[a];
            if (lub) {
                float Fl[3], Ftl[3];
                lub_f(s, rif * rjf / rs, n, -delta, vrel, Fl, Ftl);
                const float tq[3] = {rif * (n[1] * Ftl[2] - n[2] * Ftl[1]), rif * (n[2] * Ftl[0] - n[0] * Ftl[2]),
                                     rif * (n[0] * Ftl[1] - n[1] * Ftl[0])};
                for (int a = 0; a < 3; ++a) { F[a] += Fl[a]; T[a] += tq[a]; }
            }
            if (!touch) continue;
            const float mj = cj[u].y;
            const float meff = mif * mj / (mif + mj);
            const int slot = hist_slot(s, p, j, hpart, seen);
            if (slot < 0) continue;
            float* xi = s.hist_xi + ((long long)p * HIST_SLOTS + slot) * 3;
            float Fc[3], Ft[3];
            contact_f(s, meff, n, delta, vrel, xi, dts, Fc, Ft);
            const float tq[3] = {rif * (n[1] * Ft[2] - n[2] * Ft[1]), rif * (n[2] * Ft[0] - n[0] * Ft[2]),
                                 rif * (n[0] * Ft[1] - n[1] * Ft[0])};
            for (int a = 0; a < 3; ++a) { F[a] += Fc[a]; T[a] += tq[a]; }
        }
    }
    // walls on non-periodic axes
    const int per[3] = {s.per_x, s.per_y, s.per_z};
    for (int a = 0; a < 3; ++a) {
        if (per[a]) continue;
        for (int side = 0; side < 2; ++side) {
            const float dist = side == 0 ? s.dem_wall[6 * p + 2 * a] + dx[a] : s.dem_wall[6 * p + 2 * a + 1] - dx[a];
            const float delta = rif - dist;
            const bool lub = s.lub && -delta < LUB_HC;
            if (delta <= 0.f && !lub) continue;
            float n[3] = {0.f, 0.f, 0.f};
            n[a] = side == 0 ? -1.f : 1.f;
            const float rw[3] = {rif * Wf[0], rif * Wf[1], rif * Wf[2]};
            const float wn[3] = {rw[1] * n[2] - rw[2] * n[1], rw[2] * n[0] - rw[0] * n[2],
                                 rw[0] * n[1] - rw[1] * n[0]};
            const float vrel[3] = {Uf[0] + wn[0], Uf[1] + wn[1], Uf[2] + wn[2]};
            if (lub) {
                float Fl[3], Ftl[3];
                lub_f(s, rif, n, -delta, vrel, Fl, Ftl);
                const float tq[3] = {rif * (n[1] * Ftl[2] - n[2] * Ftl[1]), rif * (n[2] * Ftl[0] - n[0] * Ftl[2]),
                                     rif * (n[0] * Ftl[1] - n[1] * Ftl[0])};
                for (int b = 0; b < 3; ++b) { F[b] += Fl[b]; T[b] += tq[b]; }
            }
            if (delta <= 0.f) continue;
            const int slot = hist_slot(s, p, -1 - (2 * a + side), hpart, seen);
            if (slot < 0) continue;
            float* xi = s.hist_xi + ((long long)p * HIST_SLOTS + slot) * 3;
            float Fc[3], Ft[3];
            contact_f(s, mif, n, delta, vrel, xi, dts, Fc, Ft);
            const float tq[3] = {rif * (n[1] * Ft[2] - n[2] * Ft[1]), rif * (n[2] * Ft[0] - n[0] * Ft[2]),
                                 rif * (n[0] * Ft[1] - n[1] * Ft[0])};
            for (int b = 0; b < 3; ++b) { F[b] += Fc[b]; T[b] += tq[b]; }
        }
    }
    // partners not met in this sub-step lose their springs
    {
        int4* hp4 = reinterpret_cast<int4*>(s.hist_partner + (long long)p * HIST_SLOTS);
#pragma unroll
        for (int k = 0; k < HIST_SLOTS / 4; ++k) {
            int4 v;
            v.x = (seen >> (4 * k)) & 1u ? hpart[4 * k] : HIST_EMPTY;
            v.y = (seen >> (4 * k + 1)) & 1u ? hpart[4 * k + 1] : HIST_EMPTY;
            v.z = (seen >> (4 * k + 2)) & 1u ? hpart[4 * k + 2] : HIST_EMPTY;
            v.w = (seen >> (4 * k + 3)) & 1u ? hpart[4 * k + 3] : HIST_EMPTY;
            hp4[k] = v;
        }
    }
    // semi-implicit Euler on the changes
    const float im = 1.f / mif, iI = 1.f / Iif;
    float dxn[3], dun[3], dwn[3];
    for (int a = 0; a < 3; ++a) {
        dun[a] = du[a] + dts * F[a] * im;
        dwn[a] = dw[a] + dts * T[a] * iI;
        const float u0a = a == 0 ? u0.x : (a == 1 ? u0.y : u0.z);
        dxn[a] = dx[a] + dts * (u0a + dun[a]);
        dxb[3 * p + a] = dxn[a];
        dub[3 * p + a] = dun[a];
        dwb[3 * p + a] = dwn[a];
    }
    if (last) {
        // the FP64 state of the step's end (positions wrapped on periodic axes)
        const int L[3] = {s.nx, s.ny, s.nz};
        for (int a = 0; a < 3; ++a) {
            double x = s.X[3 * p + a] + (double)dxn[a];
            if (per[a]) x = x < 0.0 ? x + L[a] : (x >= L[a] ? x - L[a] : x);
            s.X[3 * p + a] = x;
            s.U[3 * p + a] += (double)dun[a];
            s.W[3 * p + a] += (double)dwn[a];
        }
        atomicMax(s.zmax_cell, (int)ceil(s.X[3 * p + 2] + s.R[p]) + 2);
    }
}

// ------------------------------------------------------------ particle map
__device__ __forceinline__ double map_metric(double kx, double ky, double kz, const double* Xp, double r) {
    // ((dx^2 + dy^2) + dz^2) - r^2, rounded step by step (no contraction)
    double dx = __dsub_rn(kx, Xp[0]);
    double dy = __dsub_rn(ky, Xp[1]);
    double dz = __dsub_rn(kz, Xp[2]);
    double s2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return __dsub_rn(s2, __dmul_rn(r, r));
}

// unwrapped cell-centre coordinate of the periodic image nearest to X
__device__ __forceinline__ double image_centre(int k, double X, int L, int periodic) {
    double c = k + 0.5;
    if (periodic) {
        if (c - X > 0.5 * L) c = (k - L) + 0.5;
        else if (X - c > 0.5 * L) c = (k + L) + 0.5;
    }
    return c;
}

// best covering particle (lowest metric, then lowest index) among the
// particles of the selected kind near cell (x, y, z); every covering mobile
// particle of a cell covered more than once is flagged as sharing cells
__device__ void best_cover(const Dev& s, int x, int y, int z, int want_fixed, double& best, int& bestp,
                           int* ncover = nullptr, int* cov = nullptr) {
    const double rm = s.r_max;
    const double xc = x + 0.5, yc = y + 0.5, zc = z + 0.5;
    GRange ra = grange((int)floor((xc - rm) / s.ghx), (int)floor((xc + rm) / s.ghx), s.gnx, s.per_x);
    GRange rb = grange((int)floor((yc - rm) / s.ghy), (int)floor((yc + rm) / s.ghy), s.gny, s.per_y);
    GRange rc = grange((int)floor((zc - rm) / s.ghz), (int)floor((zc + rm) / s.ghz), s.gnz, s.per_z);
    for (int ic = 0; ic < rc.n; ++ic)
        for (int ib = 0; ib < rb.n; ++ib)
            for (int ia = 0; ia < ra.n; ++ia) {
                int gg = ra.v[ia] + s.gnx * (rb.v[ib] + s.gny * rc.v[ic]);
                int b = s.g_start[gg], e = b + s.g_count[gg];
                for (int k = b; k < e; ++k) {
                    int p = s.g_list[k];
                    const float4 xr = s.Xr[p];
                    if ((xr.w < 0.f) != (want_fixed != 0)) continue;
                    // cheap reject in FP32 with a margin far above its rounding
                    float fx = (float)xc - xr.x, fy = (float)yc - xr.y, fz = (float)zc - xr.z;
                    if (s.per_x) fx -= (float)s.nx * rintf(fx / (float)s.nx);
                    if (s.per_y) fy -= (float)s.ny * rintf(fy / (float)s.ny);
                    if (s.per_z) fz -= (float)s.nz * rintf(fz / (float)s.nz);
                    const float d2 = fx * fx + fy * fy + fz * fz;
                    const float rr = fabsf(xr.w);
                    if (d2 > rr * rr + 1e-2f * (1.f + rr * rr)) continue;
                    const double* Xp = s.X + 3 * p;
                    const double r = s.R[p];
                    double m = map_metric(image_centre(x, Xp[0], s.nx, s.per_x), image_centre(y, Xp[1], s.ny, s.per_y),
                                          image_centre(z, Xp[2], s.nz, s.per_z), Xp, r);
                    if (m > 0.0) continue;
                    if (ncover) {
                        if (*ncover < 4) cov[*ncover] = p;
                        (*ncover)++;
                    }
                    if (m < best || (m == best && p < bestp)) {
                        best = m;
                        bestp = p;
                    }
                }
            }
}

__global__ void k_fixed_map(Dev s) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.n) return;
    int x, y, z;
    coords(s, c, x, y, z);
    double best = __longlong_as_double(0x7ff0000000000000LL);
    int bestp = -1;
    // above every particle's top (z not periodic) no sphere covers the cell
    if (s.per_z || z <= *s.zmax_cell) best_cover(s, x, y, z, 1, best, bestp);
    reinterpret_cast<double*>(s.fixkey)[c] = best;
    s.fixowner[c] = bestp;
}

// Mobile particles covering cell (x, y, z). The inside test is decided in
// FP32 where |d^2 - r^2| exceeds a bound far above the FP32 rounding of the
// offsets (the FP64 result has the same sign there) and in FP64 without
// fused multiply-add otherwise. Returns the number of covering particles
// (up to 4 are listed).
__device__ int covering_mobile(const Dev& s, int x, int y, int z, int* cov) {
    const double rm = s.r_max;
    const double xc = x + 0.5, yc = y + 0.5, zc = z + 0.5;
    GRange ra = grange((int)floor((xc - rm) / s.ghx), (int)floor((xc + rm) / s.ghx), s.gnx, s.per_x);
    GRange rb = grange((int)floor((yc - rm) / s.ghy), (int)floor((yc + rm) / s.ghy), s.gny, s.per_y);
    GRange rc = grange((int)floor((zc - rm) / s.ghz), (int)floor((zc + rm) / s.ghz), s.gnz, s.per_z);
    int n = 0;
    for (int ic = 0; ic < rc.n; ++ic)
        for (int ib = 0; ib < rb.n; ++ib)
            for (int ia = 0; ia < ra.n; ++ia) {
                const int gg = ra.v[ia] + s.gnx * (rb.v[ib] + s.gny * rc.v[ic]);
                const int b = s.g_start[gg], e = b + s.g_count[gg];
                for (int k = b; k < e; ++k) {
                    const int p = s.g_list[k];
                    const float4 xr = s.Xr[p];
                    if (xr.w < 0.f) continue;
                    float fx = (float)xc - xr.x, fy = (float)yc - xr.y, fz = (float)zc - xr.z;
                    if (s.per_x) fx -= (float)s.nx * rintf(fx / (float)s.nx);
                    if (s.per_y) fy -= (float)s.ny * rintf(fy / (float)s.ny);
                    if (s.per_z) fz -= (float)s.nz * rintf(fz / (float)s.nz);
                    const float m32 = fx * fx + fy * fy + fz * fz - xr.w * xr.w;
                    const float tol = 1e-3f * (1.f + xr.w * xr.w);
                    if (m32 > tol) continue;
                    if (m32 >= -tol) {
                        const double* Xp = s.X + 3 * p;
                        const double m = map_metric(image_centre(x, Xp[0], s.nx, s.per_x),
                                                    image_centre(y, Xp[1], s.ny, s.per_y),
                                                    image_centre(z, Xp[2], s.nz, s.per_z), Xp, s.R[p]);
                        if (m > 0.0) continue;
                    }
                    if (n < 4) cov[n] = p;
                    n++;
                }
            }
    return n;
}

// new owner of a cell; at set-up covered cells simply become solid, during a
// run every change is listed for the transition pass
__device__ void remap_cell(const Dev& s, long long c, int init_mode) {
    int x, y, z;
    coords(s, c, x, y, z);
    const int fo = s.fixowner[c];
    int cov[4];
    const int nm = covering_mobile(s, x, y, z, cov);
    if (nm > 4) set_error(s, ERR_CAPACITY);
    int bestp;
    if (nm + (fo >= 0) <= 1) {
        bestp = nm ? cov[0] : fo;
    } else {
        // several covers: exact metrics decide (lowest, then lowest index)
        double best = reinterpret_cast<const double*>(s.fixkey)[c];
        bestp = fo;
        for (int k = 0; k < min(nm, 4); ++k) {
            const int p = cov[k];
            const double* Xp = s.X + 3 * p;
            const double m = map_metric(image_centre(x, Xp[0], s.nx, s.per_x), image_centre(y, Xp[1], s.ny, s.per_y),
                                        image_centre(z, Xp[2], s.nz, s.per_z), Xp, s.R[p]);
            if (m < best || (m == best && p < bestp)) {
                best = m;
                bestp = p;
            }
            s.shared[p] = 1;
        }
    }
    const uint8_t t0 = s.flags[c] & TYPE_MASK;
    if (init_mode) {
        if (bestp >= 0) {
            s.flags[c] = T_SOL;
            s.owner[c] = bestp;
            s.mass[c] = 0.f;
            s.phi[c] = 0.f;
        }
        return;
    }
    const bool was = t0 == T_SOL;
    if ((bestp >= 0) != was || (was && bestp != s.owner[c])) {
        int k = atomicAdd(s.tl_count, 1);
        if (k < s.tl_cap) {
            s.tl[k] = (int)c;
            s.tl_info[2 * k] = bestp;
        } else {
            set_error(s, ERR_CAPACITY);
        }
    }
}

__global__ void k_remap_all(Dev s, int init_mode) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.n) return;
    int x, y, z;
    coords(s, c, x, y, z);
    if (z > *s.zmax_cell) return;
    remap_cell(s, c, init_mode);
}

// Every mobile particle that moved since its last map (|dX| > 0) marks the
// cells whose inside/outside status it can have changed: a cell changes only
// if |x_c - X_new| - r lies within |dX| of zero (triangle inequality), so
// the thin shell |  |x_c - X_new| - r | <= |dX| + 1e-3 is marked (the slack
// covers the FP32 evaluation of the offsets, exact to ~1e-6 through the
// integer-plus-fraction form of the centre). A particle that shares a cell
// with another one marks its whole box, since the owner of a shared cell is
// decided by comparing the two metrics.
__global__ void k_active(Dev s) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.np || s.fixed[p]) return;
    const double dx = s.X[3 * p] - s.Xm[3 * p], dy = s.X[3 * p + 1] - s.Xm[3 * p + 1],
                 dz = s.X[3 * p + 2] - s.Xm[3 * p + 2];
    const double d = sqrt(dx * dx + dy * dy + dz * dz);
    if (s.shared[p] || d > 0.0) {
        s.margin[p] = s.shared[p] ? -1.f : (float)d;   // shell half-width (negative: whole box)
        s.shared[p] = 0;
        int k = atomicAdd(s.act_count, 1);
        s.act[k] = p;
    }
}

__device__ __forceinline__ void bbox_axis(double a, double b, double r, int L, int periodic, int& lo, int& hi) {
    double mn = a < b ? a : b, mx = a < b ? b : a;
    lo = (int)floor(mn - r - 0.5) - 1;
    hi = (int)ceil(mx + r - 0.5) + 1;
    if (!periodic) {
        lo = lo < 0 ? 0 : lo;
        hi = hi > L - 1 ? L - 1 : hi;
    } else if (hi - lo + 1 > L) {
        lo = 0;
        hi = L - 1;
    }
}

// Cells of the shell (or of the old and new boxes) of every active particle
// join the dirty list, each once. A warp per particle, a lane per (y, z)
// row of its box: the row meets the shell | |x_c - X| - r | <= band in at
// most two x-intervals, found from the row's distance to the centre; the
// radii are widened by 1e-3 cells so that rounding can only add cells (a
// cell re-mapped without need keeps its owner).
__global__ void k_dirty(Dev s) {
    const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (wid >= *s.act_count) return;   // whole warps leave together
    const int p = s.act[wid];
    const double r = s.R[p];
    const float w = s.margin[p];
    const bool whole = w < 0.f;
    int lo[3], hi[3];
    bbox_axis(s.Xm[3 * p], s.X[3 * p], r, s.nx, s.per_x, lo[0], hi[0]);
    bbox_axis(s.Xm[3 * p + 1], s.X[3 * p + 1], r, s.ny, s.per_y, lo[1], hi[1]);
    bbox_axis(s.Xm[3 * p + 2], s.X[3 * p + 2], r, s.nz, s.per_z, lo[2], hi[2]);
    const int4 xi = s.Xi[p];
    const float4 xf = s.Xfr[p];
    const float rf = (float)r, band = w + 1e-3f;
    const float ro = rf + band + 1e-3f, ri = fmaxf(rf - band - 1e-3f, 0.f);
    const int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
    const int rows = ey * ez;
    // relative x index of a cell = a + xoff, with a its x offset from the centre
    const float xoff = (float)(xi.x - lo[0]) - 0.5f + xf.x;
    for (int r0 = 0; r0 < rows; r0 += 32) {
        const int rr = r0 + lane;
        int a0 = 0, a1 = -1, b0 = 0, b1 = -1;    // relative x ranges of the row
        int ub = 0, uc = 0;
        if (rr < rows) {
            ub = lo[1] + rr % ey;
            uc = lo[2] + rr / ey;
            if (whole) {
                a1 = ex - 1;
            } else {
                const float bb = (float)(ub - xi.y) + 0.5f - xf.y;
                const float cc = (float)(uc - xi.z) + 0.5f - xf.z;
                const float rho2 = bb * bb + cc * cc;
                if (rho2 <= ro * ro) {
                    const float ho = sqrtf(ro * ro - rho2);
                    const float hin = rho2 < ri * ri ? sqrtf(ri * ri - rho2) : 0.f;
                    if (hin == 0.f) {
                        a0 = (int)ceilf(xoff - ho);
                        a1 = (int)floorf(xoff + ho);
                    } else {
                        a0 = (int)ceilf(xoff - ho);
                        a1 = (int)floorf(xoff - hin);
                        b0 = (int)ceilf(xoff + hin);
                        b1 = (int)floorf(xoff + ho);
                    }
                    a0 = max(a0, 0); a1 = min(a1, ex - 1);
                    b0 = max(b0, 0); b1 = min(b1, ex - 1);
                }
            }
        }
        const int n1 = max(0, a1 - a0 + 1), n2 = max(0, b1 - b0 + 1), nc = n1 + n2;
        for (int k = 0; __any_sync(0xffffffffu, k < nc); ++k) {
            bool first = false;
            int cell = 0;
            if (k < nc) {
                const int ua = lo[0] + (k < n1 ? a0 + k : b0 + k - n1);
                const int a = (ua % s.nx + s.nx) % s.nx, b = (ub % s.ny + s.ny) % s.ny, c = (uc % s.nz + s.nz) % s.nz;
                cell = a + s.nx * (b + s.ny * c);
                first = !(flag_or(s.dirty, cell, 1) & 1);
            }
            warp_append(s, first, cell, s.dl, s.dl_count, s.dl_cap);
        }
    }
}

__global__ void k_remap_list(Dev s) {
    const int cnt = min(*s.dl_count, s.dl_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const int c = s.dl[i];
        s.dirty[c] = 0;
        remap_cell(s, c, 0);
    }
}

// the active particles' map positions move to their current centres
__global__ void k_map_position(Dev s) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *s.act_count) return;
    const int p = s.act[k];
    s.Xm[3 * p] = s.X[3 * p];
    s.Xm[3 * p + 1] = s.X[3 * p + 1];
    s.Xm[3 * p + 2] = s.X[3 * p + 2];
}

#define FOR_TL(i)                                                                             \
    for (int i = blockIdx.x * blockDim.x + threadIdx.x, _cnt = min(*s.tl_count, s.tl_cap); i < _cnt; \
         i += gridDim.x * blockDim.x)

enum : int { NT_UNCOVERED_LIQ = 0x100 };

// covered cells give their mass to the pool; uncovered cells become liquid
// (interface next to gas, gas without fluid neighbours) with f_eq(mean rho,
// u_b) and take their mass from the pool (snapshot of the cell types)
__global__ void k_transitions(Dev s, int last_parity) {
    // a warp per transition: the 27 PDFs of a covered cell, the 26
    // neighbours of an uncovered one and its 27 new PDFs are spread over the
    // lanes, so no thread walks a long chain of dependent loads
    double dpool = 0.0;   // lane 0's change of the pool (one atomic per block)
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int count = min(*s.tl_count, s.tl_cap);
    for (int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); i < count; i += nwarps) {
        const int c = s.tl[i];
        const int o1 = s.tl_info[2 * i];
        const int t0 = s.flags[c] & TYPE_MASK;
        int x, y, z;
        coords(s, c, x, y, z);
        int nt;
        if (o1 >= 0) {
            // covered: its liquid mass goes to the pool
            float v = (t0 == T_LIQ && lane < 27) ? ld_any(s, s.f, fstar_slot(s, lane, x, y, z, c, last_parity)) : 0.f;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(full, v, o);
            if (lane == 0) {
                if (t0 == T_LIQ) dpool += (double)(1.f + v);
                else if (t0 == T_IFC) dpool += (double)s.mass[c];
            }
            nt = T_SOL;
        } else {
            // uncovered: lane k takes neighbour q = k (k < 13) or k + 1
            float rs = 0.f;
            int cnt = 0;
            bool gas = false;
            if (lane < 26) {
                const int q = lane < 13 ? lane : lane + 1;
                const long long nb = nbr(s, x, y, z, cx(q), cy(q), cz(q));
                if (nb >= 0) {
                    const int tn = s.flags[nb] & TYPE_MASK;
                    if (tn == T_IFC) {
                        rs = s.ru[nb].x;
                        cnt = 1;
                    } else if (tn == T_LIQ) {
                        float g[27];
                        load_fstar(s, nb, last_parity, g);
                        float d = 0.f;
                        for (int k = 0; k < 27; ++k) d += g[k];
                        rs = 1.f + d;
                        cnt = 1;
                    }
                    gas = tn == T_GAS;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                rs += __shfl_xor_sync(full, rs, o);
                cnt += __shfl_xor_sync(full, cnt, o);
            }
            gas = __any_sync(full, gas);
            if (cnt == 0) {
                nt = T_GAS;
            } else {
                const float rb = rs / cnt;
                int po = s.owner[c];
                if (po < 0 || po >= s.np) {
                    if (lane == 0) set_error(s, ERR_INVARIANT);
                    po = 0;
                }
                const double* Xp = s.X + 3 * po;
                const double d[3] = {wrapd(x + 0.5 - Xp[0], s.nx, s.per_x), wrapd(y + 0.5 - Xp[1], s.ny, s.per_y),
                                     wrapd(z + 0.5 - Xp[2], s.nz, s.per_z)};
                const double* Up = s.U + 3 * po;
                const double* Wp = s.W + 3 * po;
                const float ub[3] = {(float)(Up[0] + (Wp[1] * d[2] - Wp[2] * d[1])),
                                     (float)(Up[1] + (Wp[2] * d[0] - Wp[0] * d[2])),
                                     (float)(Up[2] + (Wp[0] * d[1] - Wp[1] * d[0]))};
                if (lane < 27) {
                    const float fq = feq_dev(lane, rb, ub[0], ub[1], ub[2]);
                    st_any(s, s.f, fstar_slot(s, lane, x, y, z, c, last_parity), fq);
                    st_any(s, s.fs, (long long)lane * s.n + c, fq);
                }
                if (lane == 0) {
                    s.ru[c] = make_float4(rb, ub[0], ub[1], ub[2]);
                    s.mass[c] = gas ? 0.f : rb;
                    if (!gas) dpool -= (double)rb;
                }
                nt = gas ? T_IFC : (T_LIQ | NT_UNCOVERED_LIQ);
            }
        }
        if (lane == 0) s.tl_info[2 * i + 1] = nt;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) dpool += __shfl_xor_sync(full, dpool, o);
    if (lane == 0) red[threadIdx.x >> 5] = dpool;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        if (t != 0.0) atomicAdd(s.pool, t);
    }
}

__global__ void k_apply_transitions(Dev s) {
    FOR_TL(i) {
        const int c = s.tl[i];
        const int nt = s.tl_info[2 * i + 1];
        const int t = nt & TYPE_MASK;
        s.flags[c] = (uint8_t)t;
        if (t == T_SOL) {
            s.owner[c] = s.tl_info[2 * i];
            s.mass[c] = 0.f;
            s.phi[c] = 0.f;
        } else {
            s.owner[c] = -1;
            if (t == T_GAS) { s.mass[c] = 0.f; s.phi[c] = 0.f; }
            else if (t == T_IFC) s.phi[c] = s.mass[c] / s.ru[c].x;
        }
    }
}

// an uncovered liquid cell that ended next to a gas cell becomes interface
__global__ void k_repair(Dev s) {
    FOR_TL(i) {
        if (!(s.tl_info[2 * i + 1] & NT_UNCOVERED_LIQ)) continue;
        const int c = s.tl[i];
        int x, y, z;
        coords(s, c, x, y, z);
        for (int q = 0; q < 27; ++q) {
            if (q == 13) continue;
            long long nb = nbr(s, x, y, z, cx(q), cy(q), cz(q));
            if (nb >= 0 && (s.flags[nb] & TYPE_MASK) == T_GAS) {
                s.flags[c] = T_IFC;
                s.phi[c] = s.mass[c] / s.ru[c].x;
                break;
            }
        }
    }
}

// The particle part of a step in two halves. The DEM half (force average,
// neighbour list, sub-steps, FP32 copies, particle grid) reads and writes
// particle state only, so it can run beside the free-surface conversion,
// which reads and writes cell state only; the re-map half needs both.
int launch_dem(const Dev& s, int have_prev, cudaStream_t st) {
    if (s.np == 0) return 0;
    int launches = 0;
    const int n3 = 3 * s.np;
    const int ns = s.dem_substeps;
    k_force_avg<<<blocks_for(n3, 128), 128, 0, st>>>(s, have_prev);
    k_dem_neighbours<<<blocks_for(32LL * s.np, 128), 128, 0, st>>>(s);
    cudaMemsetAsync(s.zmax_cell, 0, sizeof(int), st);
    launches += 2 + ns;
    const float dts = 1.f / (float)ns;
    for (int k = 0; k < ns; ++k) {
        const int a = k % 2, b = 1 - a;
        k_dem_substep<<<blocks_for(s.np, 64), 64, 0, st>>>(s, s.dem_dx[a], s.dem_du[a], s.dem_dw[a], s.dem_dx[b],
                                                          s.dem_du[b], s.dem_dw[b], dts, k == ns - 1);
    }
    k_particle_copies<<<blocks_for(s.np, 128), 128, 0, st>>>(s);
    launches += 1 + launch_grid_build(s, st);
    return launches;
}

int launch_remap(const Dev& s, int last_parity, cudaStream_t st) {
    if (s.np == 0) return 0;
    cudaMemsetAsync(s.tl_count, 0, sizeof(int), st);
    cudaMemsetAsync(s.act_count, 0, sizeof(int), st);
    cudaMemsetAsync(s.dl_count, 0, sizeof(int), st);
    k_active<<<blocks_for(s.np, 128), 128, 0, st>>>(s);
    k_dirty<<<blocks_for(32LL * s.np, 128), 128, 0, st>>>(s);
    k_remap_list<<<152 * 8, 128, 0, st>>>(s);
    k_map_position<<<blocks_for(s.np, 256), 256, 0, st>>>(s);
    k_transitions<<<152 * 4, 128, 0, st>>>(s, last_parity);
    k_apply_transitions<<<152 * 4, 256, 0, st>>>(s);
    k_repair<<<152 * 4, 256, 0, st>>>(s);
    return 7;
}

__global__ void k_init_particles(Dev s, int first, int count, double rho_p) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    int p = first + k;
    double r = s.R[p];
    s.M[p] = rho_p * (4.0 / 3.0) * 3.14159265358979323846 * r * r * r;
    s.I[p] = 0.4 * s.M[p] * r * r;
    for (int a = 0; a < 3; ++a) {
        s.U[3 * p + a] = s.W[3 * p + a] = 0.0;
        s.Fh[3 * p + a] = s.Th[3 * p + a] = s.Fp[3 * p + a] = s.Tp[3 * p + a] = 0.0;
        s.Fa[3 * p + a] = s.Ta[3 * p + a] = 0.0;
    }
    for (int j = 0; j < HIST_SLOTS; ++j) s.hist_partner[(long long)p * HIST_SLOTS + j] = HIST_EMPTY;
    s.margin[p] = 0.f;
    // the set-up map (k_remap_all) flags every particle that shares a cell;
    // the others re-map their thin shell from the first step on
    s.shared[p] = 0;
    for (int a = 0; a < 3; ++a) s.Xm[3 * p + a] = s.X[3 * p + a];
    atomicMax(s.zmax_cell, (int)ceil(s.X[3 * p + 2] + r) + 2);
}

void launch_particles_add(const Dev& s, int first, int count, cudaStream_t st) {
    k_init_particles<<<blocks_for(count, 128), 128, 0, st>>>(s, first, count, s.rho_p);
    k_particle_copies<<<blocks_for(s.np, 128), 128, 0, st>>>(s);
    launch_grid_build(s, st);
    k_fixed_map<<<blocks_for(s.n, 256), 256, 0, st>>>(s);
    k_remap_all<<<blocks_for(s.n, 256), 256, 0, st>>>(s, 1);
}

}  // namespace fsl
