// Field export/import in the canonical layout of the C ABI (direction-major
// post-collision PDFs, FP64 scalars) and the FP64 diagnostic reductions of
// Section 3.2 (liquid mass, momentum, bulk velocity, interface count,
// bedload rate of Eq. (1)).
#include <algorithm>
#include <type_traits>

#include "collide_pair.cuh"
#include "fslbm_dev.cuh"

namespace fsl {

__device__ __forceinline__ bool fluid(uint8_t fl) {
    int t = fl & TYPE_MASK;
    return t == T_LIQ || t == T_IFC;
}

// which & 0xff: FSLBM_FIELD_PDF, MASS, PHI, RHO, U or NORMAL; which >> 8: the
// direction (PDF) or component (U, NORMAL) written to out[0..n)
__global__ void k_export(Dev s, int last_parity, uint32_t which, double* out) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.n) return;
    const uint8_t fl = s.flags[c];
    const int t = fl & TYPE_MASK;
    const uint32_t field = which & 0xffu;
    const int sub = (int)(which >> 8);
    if (field == FSLBM_FIELD_PDF) {
        if (!fluid(fl)) { out[c] = 0.0; return; }
        int x, y, z;
        coords(s, c, x, y, z);
        out[c] = wqd(sub) + (double)ld_any(s, s.f, fstar_slot(s, sub, x, y, z, c, last_parity));
        return;
    }
    if (field == FSLBM_FIELD_NORMAL) {
        float4 v = t == T_IFC ? s.nrm[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        out[c] = sub == 0 ? v.x : (sub == 1 ? v.y : v.z);
        return;
    }
    if (field == FSLBM_FIELD_PHI) {
        out[c] = t == T_LIQ ? 1.0 : (t == T_IFC ? (double)s.phi[c] : 0.0);
        return;
    }
    double rho = 0.0, u[3] = {0, 0, 0};
    if (fluid(fl)) {
        float f[27];
        load_fstar(s, c, last_parity, f);
        double d = 0, j[3] = {0, 0, 0};
        for (int q = 0; q < 27; ++q) {
            d += f[q];
            j[0] += cx(q) * (double)f[q];
            j[1] += cy(q) * (double)f[q];
            j[2] += cz(q) * (double)f[q];
        }
        rho = 1.0 + d;
        u[0] = (j[0] - 0.5 * rho * s.gxd) / rho;
        u[1] = (j[1] - 0.5 * rho * s.gyd) / rho;
        u[2] = (j[2] - 0.5 * rho * s.gzd) / rho;
    }
    if (field == FSLBM_FIELD_MASS) out[c] = t == T_LIQ ? rho : (t == T_IFC ? (double)s.mass[c] : 0.0);
    else if (field == FSLBM_FIELD_RHO) out[c] = rho;
    else if (field == FSLBM_FIELD_U) out[c] = u[sub];
}

__global__ void k_export_type(Dev s, uint8_t* out) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < s.n) out[c] = s.flags[c] & TYPE_MASK;
}
__global__ void k_export_owner(Dev s, int* out) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < s.n) out[c] = (s.flags[c] & TYPE_MASK) == T_SOL ? s.owner[c] : -1;
}

void launch_export(const Dev& s, int last_parity, uint32_t which, double* out, cudaStream_t st) {
    k_export<<<blocks_for(s.n, 128), 128, 0, st>>>(s, last_parity, which, out);
}
void launch_export_type(const Dev& s, uint8_t* out, cudaStream_t st) {
    k_export_type<<<blocks_for(s.n, 256), 256, 0, st>>>(s, out);
}
void launch_export_owner(const Dev& s, int* out, cudaStream_t st) {
    k_export_owner<<<blocks_for(s.n, 256), 256, 0, st>>>(s, out);
}

// arg & 1: layout parity, arg >> 8: direction q. For q < 27 the PDF f*_q
// (double, canonical) becomes f - w in its AA slot (and in the side buffer of
// interface cells); q == 27 refreshes (rho, u) and phi of interface cells.
__global__ void k_import_pdf(Dev s, int arg, const double* in) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.n) return;
    const uint8_t fl = s.flags[c];
    if (!fluid(fl)) return;
    const int last_parity = arg & 1;
    const int q = arg >> 8;
    const bool ifc = (fl & TYPE_MASK) == T_IFC;
    if (q < 27) {
        int x, y, z;
        coords(s, c, x, y, z);
        const float v = (float)(in[c] - wqd(q));
        st_any(s, s.f, fstar_slot(s, q, x, y, z, c, last_parity), v);
        if (ifc) st_any(s, s.fs, (long long)q * s.n + c, v);
        return;
    }
    if (!ifc) return;
    float f[27];
    for (int k = 0; k < 27; ++k) f[k] = ld_any(s, s.fs, (long long)k * s.n + c);
    float rho, ux, uy, uz;
    post_moments(s, f, rho, ux, uy, uz);
    s.ru[c] = make_float4(rho, ux, uy, uz);
    s.phi[c] = s.mass[c] / rho;
}
void launch_import_pdf(const Dev& s, int arg, const double* in, cudaStream_t st) {
    k_import_pdf<<<blocks_for(s.n, 128), 128, 0, st>>>(s, arg, in);
}

__global__ void k_import_mass(Dev s, const double* in) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.n) return;
    if ((s.flags[c] & TYPE_MASK) != T_IFC) return;
    s.mass[c] = (float)in[c];
    s.phi[c] = (float)(in[c] / (double)s.ru[c].x);
}
void launch_import_mass(const Dev& s, const double* in, cudaStream_t st) {
    k_import_mass<<<blocks_for(s.n, 256), 256, 0, st>>>(s, in);
}

// ------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// compensated FP32 sum (Kahan): per-thread partial sums keep about twice
// FP32's precision before they enter the FP64 block reduction
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Fluid-cell sums: liquid mass (liquid rho + interface m), momentum, and the
// phi-weighted sums of the bulk velocity. Threads run along x, blocks over
// rows (a few rows per thread, so that many cells are in flight); every
// block writes its partial sums to its own row of `part`, and k_reduce_tail
// adds the rows in a fixed order. Each cell's 27 post-collision PDFs come from
// the slots the last step wrote: (opp q, x) after an even step, (q, x + c_q)
// after an odd one (constant offsets inside the lattice, the general lookup
// at the faces). The liquid density enters as a count plus the sum of
// deviations, so no rounding of 1 + d is accumulated.
template <typename S, int LP>
__global__ void __launch_bounds__(256, 3) k_reduce_cells(Dev s, double* part) {
    __shared__ double sh[7][8];
    KSum acc[6];
    long long nfluid = 0;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const S* f = static_cast<const S*>(s.f);
    const long long n = s.n;
    const int nrows = s.ny * s.nz, sxy = s.nx * s.ny;
    const float gx = s.gx, gy = s.gy, gz = s.gz;
    if (x < s.nx) {
        for (int row = blockIdx.y; row < nrows; row += gridDim.y) {
            const int cell = x + s.nx * row;
            const uint8_t fl = s.flags[cell];
            if (!fluid(fl)) continue;
            const int t = fl & TYPE_MASK;
            const int y = row % s.ny, z = row / s.ny;
            // f - w of the cell's post-collision PDFs. With 16-bit storage
            // each slot's reference w_q delta(z_slot) is added back: in closed
            // form where every slot of direction c_z sits at the same z (after
            // an even step all at z; after an odd step, inside the lattice, at
            // z + c_z: per-axis weights 1/6, 2/3, 1/6), value by value at the
            // faces
            float fv[27];
            float rd = 0.f, rz = 0.f;   // reference part of sum f and sum c_z f
            if (LP == 0) {
#pragma unroll
                for (int q = 0; q < 27; ++q) fv[q] = Store<S>::ld(f + (long long)opp(q) * n + cell);
                if (Store<S>::HREF) rd = s.href[z];
            } else if (x > 0 && x < s.nx - 1 && y > 0 && y < s.ny - 1 && z > 0 && z < s.nz - 1) {
#pragma unroll
                for (int q = 0; q < 27; ++q)
                    fv[q] = Store<S>::ld(f + (long long)q * n + (cell + cx(q) + s.nx * cy(q) + sxy * cz(q)));
                if (Store<S>::HREF) {
                    const float hm = s.href[z - 1], h0 = s.href[z], hp = s.href[z + 1];
                    rd = (hm + hp) * (1.f / 6.f) + h0 * (2.f / 3.f);
                    rz = (hp - hm) * (1.f / 6.f);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 27; ++q) {
                    // slot (q, x + c_q), or (opp q, x) beyond a wall face
                    const int tx = shift(x, cx(q), s.nx, s.per_x), ty = shift(y, cy(q), s.ny, s.per_y),
                              tz = shift(z, cz(q), s.nz, s.per_z);
                    const bool wall = tx < 0 || ty < 0 || tz < 0;
                    const long long i = wall ? (long long)opp(q) * n + cell
                                             : (long long)q * n + tx + (long long)s.nx * (ty + (long long)s.ny * tz);
                    fv[q] = Store<S>::ld(f + i);
                    if (Store<S>::HREF) fv[q] += wq(q) * s.href[wall ? z : tz];
                }
            }
            float d = rd, jx = 0.f, jy = 0.f, jz = rz;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                d += fv[q];
                jx += cx(q) * fv[q];
                jy += cy(q) * fv[q];
                jz += cz(q) * fv[q];
            }
            if (!isfinite(d) || !isfinite(jx) || !isfinite(jy) || !isfinite(jz)) set_error(s, ERR_NAN);
            const float rho = 1.f + d;
            const float mx = jx - 0.5f * rho * gx;   // rho u
            // sums over fluid cells, the 1 of every cell counted apart:
            // mass - 1 (liquid d, interface m - 1), momentum, phi rho - 1,
            // phi rho u_x
            ++nfluid;
            acc[1].add(mx);
            acc[2].add(jy - 0.5f * rho * gy);
            acc[3].add(jz - 0.5f * rho * gz);
            if (t == T_LIQ) {
                acc[0].add(d);
                acc[4].add(d);
                acc[5].add(mx);
            } else {
                const float m = s.mass[cell], phi = s.phi[cell];
                if (!isfinite(m)) set_error(s, ERR_NAN);
                acc[0].add(m - 1.f);
                acc[4].add(phi * rho - 1.f);
                acc[5].add(phi * mx);
            }
        }
    }
    // out[0..5]: mass, momentum x, y, z, sum phi rho u_x, sum phi rho
    double v[7] = {acc[0].value(), acc[1].value(), acc[2].value(), acc[3].value(), acc[5].value(),
                   acc[4].value(), (double)nfluid};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 7; ++k) {
        const double w = warp_sum(v[k]);
        if (lane == 0) sh[k][wid] = w;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double w = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) w += sh[threadIdx.x][i];
        part[8 * ((long long)blockIdx.y * gridDim.x + blockIdx.x) + threadIdx.x] = w;
    }
}

// A block's seven partial sums (mass, momentum x, y, z, sum phi rho u_x, sum
// phi rho, fluid cells) into its row `row` of the partial array (blockDim.x
// a multiple of 32, at most 128 threads).
__device__ __forceinline__ void block_partials(const KSum (&acc)[6], long long nfluid, double* row,
                                               double (&sh)[7][4]) {
    double v[7] = {acc[0].value(), acc[1].value(), acc[2].value(), acc[3].value(), acc[5].value(),
                   acc[4].value(), (double)nfluid};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 7; ++k) {
        const double w = warp_sum(v[k]);
        if (lane == 0) sh[k][wid] = w;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double w = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) w += sh[threadIdx.x][i];
        row[threadIdx.x] = w;
    }
}

// One fluid cell's contribution: d = sum (f - w), j = sum c (f - w).
__device__ __forceinline__ void reduce_cell(const Dev& s, KSum (&acc)[6], long long& nfluid, int cell, int t,
                                            float d, float jx, float jy, float jz) {
    if (!isfinite(d) || !isfinite(jx) || !isfinite(jy) || !isfinite(jz)) set_error(s, ERR_NAN);
    const float rho = 1.f + d;
    const float mx = jx - 0.5f * rho * s.gx;   // rho u
    ++nfluid;
    acc[1].add(mx);
    acc[2].add(jy - 0.5f * rho * s.gy);
    acc[3].add(jz - 0.5f * rho * s.gz);
    if (t == T_LIQ) {
        acc[0].add(d);
        acc[4].add(d);
        acc[5].add(mx);
    } else {
        const float m = s.mass[cell], phi = s.phi[cell];
        if (!isfinite(m)) set_error(s, ERR_NAN);
        acc[0].add(m - 1.f);
        acc[4].add(phi * rho - 1.f);
        acc[5].add(phi * mx);
    }
}

// The same sums with two x-adjacent cells (x even, x + 1) per thread and the
// sweep's pair loads: after an even step the two slots of every direction are
// adjacent and aligned, after an odd step those of the directions with
// c_x = 0 are, and the others take two loads from one address; the stored
// values are summed raw (times the storage scale, on packed FP32) and scaled
// once. Blocks of 128 threads cover 256 cells of a row; the partial rows are
// those of k_reduce_cells. Needs nx even and 32-bit element indices.
// The same sums with two x-adjacent cells (x even, x + 1) per thread and the
// sweep's pair loads: after an even step the two slots of every direction are
// adjacent and aligned, after an odd step those of the directions with
// c_x = 0 are, and the others take two loads from one address; the stored
// values are summed raw (times the storage scale, on packed FP32) and scaled
// once. Blocks of 128 threads cover 256 cells of a row; the partial rows are
// those of k_reduce_cells. After an odd step the pairs whose neighbours are
// not all inside the lattice without wrap (face rows and the pairs at x = 0,
// nx - 2) are left to k_reduce_edges, so that this kernel carries no boundary
// code. Needs nx even and 32-bit element indices.
template <typename S, int LP>
__global__ void __launch_bounds__(128, 6) k_reduce_pairs(Dev s, double* part) {
    __shared__ double sh[7][4];
    KSum acc[6];
    long long nfluid = 0;
    const int x = blockIdx.x * 256 + 2 * (int)threadIdx.x;
    const S* f = static_cast<const S*>(s.f);
    const unsigned un = (unsigned)s.n;
    const int nrows = s.ny * s.nz, sxy = s.nx * s.ny;
    constexpr float UNS = 1.f / Store<S>::scale;
    if (x < s.nx && (LP == 0 || (x > 0 && x + 1 < s.nx - 1))) {
        for (int row = blockIdx.y; row < nrows; row += gridDim.y) {
            const int y = row % s.ny, z = row / s.ny;
            if (LP == 1 && (y == 0 || y == s.ny - 1 || z == 0 || z == s.nz - 1)) continue;
            const int cell = x + s.nx * row;
            const uchar2 fl = *reinterpret_cast<const uchar2*>(s.flags + cell);
            const int t0 = fl.x & TYPE_MASK, t1 = fl.y & TYPE_MASK;
            const bool f0 = t0 == T_LIQ || t0 == T_IFC, f1 = t1 == T_LIQ || t1 == T_IFC;
            if (!f0 && !f1) continue;
            float2 D = make_float2(0.f, 0.f), JX = D, JY = D, JZ = D;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                float2 v;
                if (LP == 0) {
                    v = Pair<S>::ld2(f + ((unsigned)opp(q) * un + (unsigned)cell));
                } else {
                    const unsigned a = (unsigned)q * un + (unsigned)(cell + cx(q) + s.nx * cy(q) + sxy * cz(q));
                    v = cx(q) == 0 ? Pair<S>::ld2(f + a)
                                   : make_float2(Store<S>::ld_raw(f + a), Store<S>::ld_raw(f + a + 1));
                }
                D = p_add(D, v);
                if (cx(q)) JX = cx(q) > 0 ? p_add(JX, v) : p_sub(JX, v);
                if (cy(q)) JY = cy(q) > 0 ? p_add(JY, v) : p_sub(JY, v);
                if (cz(q)) JZ = cz(q) > 0 ? p_add(JZ, v) : p_sub(JZ, v);
            }
            float rd = 0.f, rz = 0.f;   // reference part of sum f and sum c_z f
            if (Store<S>::HREF) {
                if (LP == 0) {
                    rd = s.href[z];
                } else {
                    const float hm = s.href[z - 1], h0 = s.href[z], hp = s.href[z + 1];
                    rd = (hm + hp) * (1.f / 6.f) + h0 * (2.f / 3.f);
                    rz = (hp - hm) * (1.f / 6.f);
                }
            }
            const float2 us = p_set(UNS);
            D = p_fma(D, us, p_set(rd));
            JX = p_mul(JX, us);
            JY = p_mul(JY, us);
            JZ = p_fma(JZ, us, p_set(rz));
            if (f0) reduce_cell(s, acc, nfluid, cell, t0, D.x, JX.x, JY.x, JZ.x);
            if (f1) reduce_cell(s, acc, nfluid, cell + 1, t1, D.y, JX.y, JY.y, JZ.y);
        }
    }
    block_partials(acc, nfluid, part + 8 * ((long long)blockIdx.y * gridDim.x + blockIdx.x), sh);
}

// four x-adjacent 16-bit stored values from an 8-byte aligned address, as
// two pairs
template <typename S>
__device__ __forceinline__ void ld4(const S* p, float2& lo, float2& hi) {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
    if constexpr (std::is_same<S, __half>::value) {
        lo = __half22float2(*reinterpret_cast<const __half2*>(&w.x));
        hi = __half22float2(*reinterpret_cast<const __half2*>(&w.y));
    } else {
        lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w.x));
        hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w.y));
    }
}

// y and z of face row r of an odd step's reduction (the y face rows of every
// z, then the z face rows of the inner y)
__device__ __forceinline__ void face_row(const Dev& s, int r, int& y, int& z) {
    if (r < 2 * s.nz) {
        z = r >> 1;
        y = (r & 1) ? s.ny - 1 : 0;
    } else {
        const int k = r - 2 * s.nz;
        y = 1 + (k >> 1);
        z = (k & 1) ? s.nz - 1 : 0;
    }
}

// The sums of k_reduce_pairs with four x-adjacent cells (x a multiple of 4)
// per thread, for 16-bit storage: after an even step every direction's four
// slots are one aligned 8-byte load; after an odd step the slots x + c_q of
// the directions with c_x = +1 or -1 are three of the aligned four plus one
// value beyond them, so 45 loads serve four cells (90 for two pairs) and a
// thread keeps twice the bytes in flight. Blocks of 64 threads cover 256 cells
// of a row, so the partial rows are those of k_reduce_pairs. After an odd step
// FACE 0 takes the inner rows and FACE 1 the face rows (y or z on a face),
// where a direction's source row (y + c_y, z + c_z) is wrapped, or beyond a
// wall the cell's own slot (opp q, x) is read; either way the same for the
// whole row, so the quad loads stay aligned and each slot's reference is
// summed per row. With walls in x the quads at x = 0 and nx - 4 of every row
// are left to k_reduce_edges; with periodic x they take their value beyond
// the aligned four across the seam.
template <typename S, int LP, int FACE>
__global__ void __launch_bounds__(64, FACE ? 8 : 12) k_reduce_quads(Dev s, double* part) {
    __shared__ double sh[7][4];
    KSum acc[6];
    long long nfluid = 0;
    const int x = blockIdx.x * 256 + 4 * (int)threadIdx.x;
    const S* f = static_cast<const S*>(s.f);
    const unsigned un = (unsigned)s.n;
    const int nrows = FACE ? 2 * s.nz + 2 * (s.ny - 2) : s.ny * s.nz, sxy = s.nx * s.ny;
    constexpr float UNS = 1.f / Store<S>::scale;
    // periodic x: the quads at the x ends take their one value beyond the
    // aligned four across the seam
    const unsigned ep = x + 4 < s.nx ? 4u : 4u - (unsigned)s.nx;
    const unsigned em = x > 0 ? 0u - 1u : (unsigned)s.nx - 1u;
    if (x < s.nx && (LP == 0 || s.per_x || (x > 0 && x + 4 < s.nx))) {
        for (int r = blockIdx.y; r < nrows; r += gridDim.y) {
            int y, z;
            if (FACE) {
                face_row(s, r, y, z);
            } else {
                y = r % s.ny;
                z = r / s.ny;
                if (LP == 1 && (y == 0 || y == s.ny - 1 || z == 0 || z == s.nz - 1)) continue;
            }
            const int cell = x + s.nx * (y + s.ny * z);
            const uchar4 fl = *reinterpret_cast<const uchar4*>(s.flags + cell);
            const int tk[4] = {fl.x & TYPE_MASK, fl.y & TYPE_MASK, fl.z & TYPE_MASK, fl.w & TYPE_MASK};
            bool fk[4], any = false;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                fk[k] = tk[k] == T_LIQ || tk[k] == T_IFC;
                any |= fk[k];
            }
            if (!any) continue;
            float2 D[2], JX[2], JY[2], JZ[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) D[h] = JX[h] = JY[h] = JZ[h] = make_float2(0.f, 0.f);
            // reference part of sum f and sum c f (face rows: slot by slot,
            // from the references of z and of its wrapped neighbours)
            float rd = 0.f, rx = 0.f, ry = 0.f, rz = 0.f;
            float hm = 0.f, h0 = 0.f, hp = 0.f;
            if (FACE) {
                const int zm = shift(z, -1, s.nz, s.per_z), zp = shift(z, 1, s.nz, s.per_z);
                h0 = s.href[z];
                hm = zm >= 0 ? s.href[zm] : h0;
                hp = zp >= 0 ? s.href[zp] : h0;
            }
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                float2 v[2];
                if (LP == 0) {
                    ld4<S>(f + ((unsigned)opp(q) * un + (unsigned)cell), v[0], v[1]);
                } else {
                    // slots x + c_q .. x + 3 + c_q of the source row
                    unsigned a;
                    bool own = false;
                    if (FACE) {
                        const int yy = shift(y, cy(q), s.ny, s.per_y), zz = shift(z, cz(q), s.nz, s.per_z);
                        own = yy < 0 || zz < 0;
                        a = own ? (unsigned)opp(q) * un + (unsigned)cell
                                : (unsigned)q * un + (unsigned)(x + s.nx * (yy + s.ny * zz));
                        const float rq = wq(q) * (own || cz(q) == 0 ? h0 : (cz(q) < 0 ? hm : hp));
                        rd += rq;
                        if (cx(q)) rx = cx(q) > 0 ? rx + rq : rx - rq;
                        if (cy(q)) ry = cy(q) > 0 ? ry + rq : ry - rq;
                        if (cz(q)) rz = cz(q) > 0 ? rz + rq : rz - rq;
                    } else {
                        a = (unsigned)q * un + (unsigned)(cell + s.nx * cy(q) + sxy * cz(q));
                    }
                    float2 A0, A1;
                    ld4<S>(f + a, A0, A1);
                    if (cx(q) == 0 || own) {
                        v[0] = A0;
                        v[1] = A1;
                    } else if (cx(q) > 0) {
                        const float e = Store<S>::ld_raw(f + (a + ep));
                        v[0] = make_float2(A0.y, A1.x);
                        v[1] = make_float2(A1.y, e);
                    } else {
                        const float e = Store<S>::ld_raw(f + (a + em));
                        v[0] = make_float2(e, A0.x);
                        v[1] = make_float2(A0.y, A1.x);
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    D[h] = p_add(D[h], v[h]);
                    if (cx(q)) JX[h] = cx(q) > 0 ? p_add(JX[h], v[h]) : p_sub(JX[h], v[h]);
                    if (cy(q)) JY[h] = cy(q) > 0 ? p_add(JY[h], v[h]) : p_sub(JY[h], v[h]);
                    if (cz(q)) JZ[h] = cz(q) > 0 ? p_add(JZ[h], v[h]) : p_sub(JZ[h], v[h]);
                }
            }
            if (LP == 0) {
                rd = s.href[z];
            } else if (!FACE) {
                // every slot of direction c_z at z + c_z: per-axis weights 1/6, 2/3, 1/6
                const float zm = s.href[z - 1], z0 = s.href[z], zp = s.href[z + 1];
                rd = (zm + zp) * (1.f / 6.f) + z0 * (2.f / 3.f);
                rz = (zp - zm) * (1.f / 6.f);
            }
            const float2 us = p_set(UNS);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                D[h] = p_fma(D[h], us, p_set(rd));
                JX[h] = p_fma(JX[h], us, p_set(rx));
                JY[h] = p_fma(JY[h], us, p_set(ry));
                JZ[h] = p_fma(JZ[h], us, p_set(rz));
            }
            if (fk[0]) reduce_cell(s, acc, nfluid, cell, tk[0], D[0].x, JX[0].x, JY[0].x, JZ[0].x);
            if (fk[1]) reduce_cell(s, acc, nfluid, cell + 1, tk[1], D[0].y, JX[0].y, JY[0].y, JZ[0].y);
            if (fk[2]) reduce_cell(s, acc, nfluid, cell + 2, tk[2], D[1].x, JX[1].x, JY[1].x, JZ[1].x);
            if (fk[3]) reduce_cell(s, acc, nfluid, cell + 3, tk[3], D[1].y, JX[1].y, JY[1].y, JZ[1].y);
        }
    }
    block_partials(acc, nfluid, part + 8 * ((long long)blockIdx.y * gridDim.x + blockIdx.x), sh);
}

// pairs of an odd step that k_reduce_pairs or k_reduce_quads leave out, one
// per thread: after k_reduce_pairs (as k_liquid_pair_edges lists them) every
// pair of the y and z face rows, then the pairs at x = 0 and nx - 2 of the
// other rows; after k_reduce_quads (ends_only) the pairs at x = 0, 2, nx - 4
// and nx - 2 of every row. Each slot is (q, x + c_q), or (opp q, x) beyond a
// wall face, with its own reference; partial rows from `part` on
template <typename S>
__global__ void __launch_bounds__(128) k_reduce_edges(Dev s, double* part, int xe, int ends_only) {
    __shared__ double sh[7][4];
    KSum acc[6];
    long long nfluid = 0;
    const S* f = static_cast<const S*>(s.f);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int hp = s.nx / 2;
    const long long nface = 2LL * s.nz + 2LL * (s.ny > 2 ? s.ny - 2 : 0);
    int y = 0, z = 0, x = 0;
    bool in = true;
    if (ends_only) {
        // the xe pairs at the x ends of every row
        if (t < (long long)xe * s.ny * s.nz) {
            const int e = (int)(t % xe);
            x = e < xe / 2 ? 2 * e : s.nx - 2 * (xe - e);
            const long long r = t / xe;
            y = (int)(r % s.ny);
            z = (int)(r / s.ny);
        } else {
            in = false;
        }
    } else if (t < nface * hp) {
        const int r = (int)(t / hp);
        x = 2 * (int)(t % hp);
        if (r < 2 * s.nz) { z = r >> 1; y = (r & 1) ? s.ny - 1 : 0; }
        else { const int k = r - 2 * s.nz; y = 1 + (k >> 1); z = (k & 1) ? s.nz - 1 : 0; }
    } else if (t < nface * hp + (long long)xe * (s.ny - 2) * (s.nz - 2)) {
        // xe pairs per row: x = 0, nx - 2, or x = 0, 2, nx - 4, nx - 2
        const long long k = t - nface * hp;
        const int e = (int)(k % xe);
        x = e < xe / 2 ? 2 * e : s.nx - 2 * (xe - e);
        const long long r = k / xe;
        y = 1 + (int)(r % (s.ny - 2));
        z = 1 + (int)(r / (s.ny - 2));
    } else {
        in = false;
    }
    if (in) {
        const int cell = x + s.nx * (y + s.ny * z);
#pragma unroll 1
        for (int k = 0; k < 2; ++k) {
            const int tk = s.flags[cell + k] & TYPE_MASK;
            if (tk != T_LIQ && tk != T_IFC) continue;
            const int xk = x + k;
            float d = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const int tx = shift(xk, cx(q), s.nx, s.per_x), ty = shift(y, cy(q), s.ny, s.per_y),
                          tz = shift(z, cz(q), s.nz, s.per_z);
                const bool wall = tx < 0 || ty < 0 || tz < 0;
                const long long i = wall ? (long long)opp(q) * s.n + cell + k
                                         : (long long)q * s.n + tx + (long long)s.nx * (ty + (long long)s.ny * tz);
                float v = Store<S>::ld(f + i);
                if (Store<S>::HREF) v += wq(q) * s.href[wall ? z : tz];
                d += v;
                jx += cx(q) * v;
                jy += cy(q) * v;
                jz += cz(q) * v;
            }
            reduce_cell(s, acc, nfluid, cell + k, tk, d, jx, jy, jz);
        }
    }
    block_partials(acc, nfluid, part + 8 * (long long)blockIdx.x, sh);
}

// pairs of k_reduce_edges: after k_reduce_pairs (face rows, then two pairs
// per inner row), or the xe pairs at the x ends of every row
inline long long reduce_edge_pairs(const Dev& s, int xe, bool ends_only) {
    if (ends_only) return (long long)xe * s.ny * s.nz;
    return (2LL * s.nz + 2LL * (s.ny > 2 ? s.ny - 2 : 0)) * (s.nx / 2) +
           2LL * (s.ny > 2 ? s.ny - 2 : 0) * (s.nz > 2 ? s.nz - 2 : 0);
}
// face rows of an odd step (y or z on a face)
inline int reduce_face_rows(const Dev& s) { return 2 * s.nz + 2 * (s.ny > 2 ? s.ny - 2 : 0); }

// four cells per thread for 16-bit storage where nx is a multiple of 4 (the
// x ends of a row after an odd step then leave two pairs each to the edges)
inline bool reduce_quads(const Dev& s) {
    return s.storage != FSLBM_STORE_FP32 && s.idx32 && s.nx % 4 == 0;
}
inline int reduce_xe(const Dev& s) { return s.nx >= 8 ? 4 : 2; }

// The result from the blocks' partial rows and the particles, in a fixed
// order over REDUCE_TAIL_BLOCKS blocks of 256 threads (FP64 adds are slow on
// one SM): block b sums its contiguous share of the rows and of the
// particles (thread t of it items t, t + 256, ...; then the warps' shuffle
// trees and a pass over the warps) into its row of s.rtail; the block that
// finishes last sums those rows in order and writes out[0] liquid mass (the
// fluid-cell count added back, plus the pool), out[1..3] momentum, out[4]
// bulk velocity, out[5] interface cells, out[6] the bedload rate of Eq. (1)
// sum u_x,p V_p / (L_x L_y), out[7] pool; it then clears the block counter.
__global__ void __launch_bounds__(256) k_reduce_tail(Dev s, const double* part, int blocks, double* out) {
    __shared__ double sh[8][8];
    __shared__ bool last;
    // v: mass - count, momentum x, y, z, sum phi rho u_x, sum phi rho - count,
    // fluid cells; v[7] the particles' sum u_x V
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int nb = gridDim.x;
    const int rc = (blocks + nb - 1) / nb, r0 = blockIdx.x * rc, r1 = min(blocks, r0 + rc);
    const int pc = (s.np + nb - 1) / nb, p0 = blockIdx.x * pc, p1 = min(s.np, p0 + pc);
#pragma unroll 4
    for (int b = r0 + threadIdx.x; b < r1; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 7; ++k) v[k] += part[8 * (long long)b + k];
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const double r = s.R[p];
        v[7] += s.U[3 * p] * (4.0 / 3.0) * 3.14159265358979323846 * r * r * r;
        if (!isfinite(s.X[3 * p]) || !isfinite(s.U[3 * p])) set_error(s, ERR_NAN);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const double w = warp_sum(v[k]);
        if (lane == 0) sh[k][wid] = w;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[threadIdx.x][i];
        s.rtail[8 * blockIdx.x + threadIdx.x] = t;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(s.rtail_count, 1) == nb - 1;
    __syncthreads();
    if (!last) return;
    __shared__ double tot[8];
    if (threadIdx.x < 8) {
        __threadfence();
        double t = 0.0;
        for (int i = 0; i < nb; ++i) t += __ldcg(&s.rtail[8 * i + threadIdx.x]);
        tot[threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double count = tot[6], pool = *s.pool;
        const double den = tot[5] + count;
        out[0] = tot[0] + count + pool;
        out[1] = tot[1];
        out[2] = tot[2];
        out[3] = tot[3];
        out[4] = den > 0 ? tot[4] / den : 0.0;
        out[5] = (double)*s.wl_count;
        out[6] = tot[7] / ((double)s.nx * (double)s.ny);
        out[7] = pool;
        if (!isfinite(pool)) set_error(s, ERR_NAN);
        *s.rtail_count = 0;
    }
}

// streaming multiprocessors of the current device (read once)
static int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        n = v > 0 ? v : 1;
    }
    return n;
}

// partial rows of the lattice reduction: the row grid's blocks, then those
// of the edge pairs after an odd step
int reduce_blocks(const Dev& s) {
    const int bx = (s.nx + 255) / 256;
    const int rows = s.ny * s.nz;
    const int face = reduce_face_rows(s);
    const long long edges = reduce_quads(s) ? reduce_edge_pairs(s, reduce_xe(s), true) : reduce_edge_pairs(s, 2, false);
    return bx * (rows < REDUCE_MAX_BY ? rows : REDUCE_MAX_BY) + (reduce_quads(s) ? bx * (face < REDUCE_MAX_BY ? face : REDUCE_MAX_BY) : 0) +
           blocks_for(edges, 128);
}

void launch_reduce(const Dev& s, int last_parity, double* out, cudaStream_t st) {
    const unsigned bx = (unsigned)((s.nx + 255) / 256);
    const int rows = s.ny * s.nz;
    const unsigned by = (unsigned)(rows < REDUCE_MAX_BY ? rows : REDUCE_MAX_BY);
    const dim3 grid(bx, by);
    double* part = s.rpart;
    int blocks = (int)(bx * by);
    // pairs (128 threads per 256-cell block); after an odd step the edge
    // pairs in a kernel of their own, whose listing needs ny, nz >= 3, nx >= 4
    const bool pairs = s.idx32 && s.nx % 2 == 0 && (last_parity == 0 || (s.nx >= 4 && s.ny >= 3 && s.nz >= 3));
    if (pairs && reduce_quads(s)) {
        // 16-bit storage, nx a multiple of 4: quads, the row blocks one
        // resident wave (12 blocks of 64 threads per SM), so that each thread
        // strides over rows and the partial rows stay few; after an odd step
        // the face rows as quads too, and with walls in x the x-end pairs of
        // every row in the edge kernel
        const unsigned wave = (unsigned)(12 * num_sms());
        const unsigned qby = (unsigned)std::min<long long>(std::min(rows, REDUCE_MAX_BY), (wave + bx - 1) / bx);
        const dim3 qgrid(bx, qby);
        blocks = (int)(bx * qby);
        if (last_parity == 0) {
            if (s.storage == FSLBM_STORE_FP16) k_reduce_quads<__half, 0, 0><<<qgrid, 64, 0, st>>>(s, part);
            else k_reduce_quads<__nv_bfloat16, 0, 0><<<qgrid, 64, 0, st>>>(s, part);
        } else {
            const int face = reduce_face_rows(s);
            const dim3 fgrid(bx, (unsigned)std::min<long long>(face, qby));
            const int xe = reduce_xe(s);
            const int eb = s.per_x ? 0 : blocks_for(reduce_edge_pairs(s, xe, true), 128);
            double* fpart = part + 8LL * blocks;
            double* epart = fpart + 8LL * fgrid.x * fgrid.y;
            if (s.storage == FSLBM_STORE_FP16) {
                k_reduce_quads<__half, 1, 0><<<qgrid, 64, 0, st>>>(s, part);
                k_reduce_quads<__half, 1, 1><<<fgrid, 64, 0, st>>>(s, fpart);
                if (eb) k_reduce_edges<__half><<<eb, 128, 0, st>>>(s, epart, xe, 1);
            } else {
                k_reduce_quads<__nv_bfloat16, 1, 0><<<qgrid, 64, 0, st>>>(s, part);
                k_reduce_quads<__nv_bfloat16, 1, 1><<<fgrid, 64, 0, st>>>(s, fpart);
                if (eb) k_reduce_edges<__nv_bfloat16><<<eb, 128, 0, st>>>(s, epart, xe, 1);
            }
            blocks += (int)(fgrid.x * fgrid.y) + eb;
        }
    } else if (pairs) {
        const int eb = last_parity == 1 ? blocks_for(reduce_edge_pairs(s, 2, false), 128) : 0;
        if (s.storage == FSLBM_STORE_FP32) {
            if (last_parity == 0) k_reduce_pairs<float, 0><<<grid, 128, 0, st>>>(s, part);
            else k_reduce_pairs<float, 1><<<grid, 128, 0, st>>>(s, part);
            if (eb) k_reduce_edges<float><<<eb, 128, 0, st>>>(s, part + 8LL * blocks, 2, 0);
        } else if (s.storage == FSLBM_STORE_FP16) {
            if (last_parity == 0) k_reduce_pairs<__half, 0><<<grid, 128, 0, st>>>(s, part);
            else k_reduce_pairs<__half, 1><<<grid, 128, 0, st>>>(s, part);
            if (eb) k_reduce_edges<__half><<<eb, 128, 0, st>>>(s, part + 8LL * blocks, 2, 0);
        } else {
            if (last_parity == 0) k_reduce_pairs<__nv_bfloat16, 0><<<grid, 128, 0, st>>>(s, part);
            else k_reduce_pairs<__nv_bfloat16, 1><<<grid, 128, 0, st>>>(s, part);
            if (eb) k_reduce_edges<__nv_bfloat16><<<eb, 128, 0, st>>>(s, part + 8LL * blocks, 2, 0);
        }
        blocks += eb;
    } else if (s.storage == FSLBM_STORE_FP32) {
        if (last_parity == 0) k_reduce_cells<float, 0><<<grid, 256, 0, st>>>(s, part);
        else k_reduce_cells<float, 1><<<grid, 256, 0, st>>>(s, part);
    } else if (s.storage == FSLBM_STORE_FP16) {
        if (last_parity == 0) k_reduce_cells<__half, 0><<<grid, 256, 0, st>>>(s, part);
        else k_reduce_cells<__half, 1><<<grid, 256, 0, st>>>(s, part);
    } else {
        if (last_parity == 0) k_reduce_cells<__nv_bfloat16, 0><<<grid, 256, 0, st>>>(s, part);
        else k_reduce_cells<__nv_bfloat16, 1><<<grid, 256, 0, st>>>(s, part);
    }
    k_reduce_tail<<<REDUCE_TAIL_BLOCKS, 256, 0, st>>>(s, part, blocks, out);
}

// ------------------------------------------------------------ bed height
// Bed topography of Section 3.2: phi_b(x, z), the fraction of the cells of
// the column (x, ., z) that a particle covers, then h_b(x), the z at which
// phi_b crosses the threshold, linearly interpolated between cell centres
// (cell k at z = k + 1/2). The topmost crossing counts; above the lattice
// phi_b is 0, and below it the bottom wall counts as solid (phi_b = 1 at
// z = -1/2).
__global__ void k_bed_fraction(Dev s, double* phi) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)s.nx * s.nz) return;
    const int x = (int)(t % s.nx), z = (int)(t / s.nx);
    const uint8_t* fl = s.flags + x + (long long)s.nx * s.ny * z;
    int c = 0;
    for (int y = 0; y < s.ny; ++y) c += (fl[(long long)s.nx * y] & TYPE_MASK) == T_SOL;
    phi[t] = (double)c / (double)s.ny;
}
__global__ void k_bed_height(Dev s, const double* phi, double phi_b, double* h) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= s.nx) return;
    int k = s.nz - 1;
    while (k >= 0 && !(phi[x + (long long)s.nx * k] >= phi_b)) --k;
    double pk, pn;
    if (k < 0) {
        pk = 1.0;
        pn = phi[x];
    } else {
        pk = phi[x + (long long)s.nx * k];
        pn = k + 1 < s.nz ? phi[x + (long long)s.nx * (k + 1)] : 0.0;
    }
    h[x] = __dadd_rn((double)k + 0.5, __ddiv_rn(pk - phi_b, pk - pn));
}

void launch_bed_height(const Dev& s, double phi_b, double* phi, double* h, cudaStream_t st) {
    k_bed_fraction<<<blocks_for((long long)s.nx * s.nz, 256), 256, 0, st>>>(s, phi);
    k_bed_height<<<blocks_for(s.nx, 128), 128, 0, st>>>(s, phi, phi_b, h);
}

// ------------------------------------------------------------ water depth
// Free-surface elevation of every column (x, y): its liquid and solid
// volume, 1 per liquid or solid cell and the fill level per interface cell
// (Section 4.2 mean water depth, with the bed height h_b of Section 3.2).
__global__ void k_surface_elevation(Dev s, double* eta) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)s.nx * s.ny) return;
    const long long sxy = (long long)s.nx * s.ny;
    double v = 0.0;
    for (int z = 0; z < s.nz; ++z) {
        const long long c = t + sxy * z;
        const int ty = s.flags[c] & TYPE_MASK;
        v += (ty == T_LIQ || ty == T_SOL) ? 1.0 : (ty == T_IFC ? (double)s.phi[c] : 0.0);
    }
    eta[t] = v;
}
// out[0]: mean over x of (y-mean elevation - h_b(x)); out[1]: mean h_b. One
// block; the sums run in a fixed order.
__global__ void k_water_depth(Dev s, const double* eta, const double* hb, double* out) {
    __shared__ double sh[2][256];
    double d = 0.0, b = 0.0;
    for (int x = threadIdx.x; x < s.nx; x += blockDim.x) {
        double e = 0.0;
        for (int y = 0; y < s.ny; ++y) e += eta[x + (long long)s.nx * y];
        d += e / s.ny - hb[x];
        b += hb[x];
    }
    sh[0][threadIdx.x] = d;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + off];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0][0] / s.nx;
        out[1] = sh[1][0] / s.nx;
    }
}

void launch_water_depth(const Dev& s, double* bed, double* eta, double* out, cudaStream_t st) {
    const size_t nxz = (size_t)s.nx * s.nz;
    launch_bed_height(s, 0.3, bed, bed + nxz, st);
    k_surface_elevation<<<blocks_for((long long)s.nx * s.ny, 256), 256, 0, st>>>(s, eta);
    k_water_depth<<<1, 256, 0, st>>>(s, eta, bed + nxz, out);
}

// ------------------------------------------------------------ bed spectrum
// Power spectral density of a bed-height series h(t, x) (Section 4.1): the
// squared modulus of its two-dimensional discrete Fourier transform, mean
// removed, over the number of samples; the transforms along x and then t are
// direct sums in FP64 with tabulated twiddles exp(-2 pi i k / N).
__global__ void k_twiddle(double2* tw, int N) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double sn, cs;
    sincospi(2.0 * (double)k / (double)N, &sn, &cs);
    tw[k] = make_double2(cs, -sn);
}
// mean of n values by one block in a fixed order
__global__ void k_series_mean(const double* h, long long n, double* mean) {
    __shared__ double sh[1024];
    double v = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) v += h[i];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 512; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) *mean = sh[0] / (double)n;
}
// X1[t][j] = sum_x (h[t][x] - mean) exp(-2 pi i j x / nx); a block per
// (t, 256 wavenumbers), the row staged through shared memory in chunks
constexpr int SPEC_CHUNK = 2048;
__global__ void k_dft_x(const double* h, const double* mean, const double2* tw, int nx, double2* X1) {
    __shared__ double row[SPEC_CHUNK];
    const int t = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const double m = *mean;
    double re = 0.0, im = 0.0;
    int k = 0;                       // (j x) mod nx
    for (int x0 = 0; x0 < nx; x0 += SPEC_CHUNK) {
        const int len = min(SPEC_CHUNK, nx - x0);
        __syncthreads();
        for (int i = threadIdx.x; i < len; i += blockDim.x) row[i] = h[(long long)t * nx + x0 + i] - m;
        __syncthreads();
        if (j < nx) {
            for (int i = 0; i < len; ++i) {
                const double2 w = tw[k];
                re = fma(row[i], w.x, re);
                im = fma(row[i], w.y, im);
                k += j;
                if (k >= nx) k -= nx;
            }
        }
    }
    if (j < nx) X1[(long long)t * nx + j] = make_double2(re, im);
}
// psd[l][j] = |sum_t X1[t][j] exp(-2 pi i l t / nt)|^2 / (nt nx)
__global__ void k_dft_t(const double2* X1, const double2* tw, int nt, int nx, double* psd) {
    const int l = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nx) return;
    double re = 0.0, im = 0.0;
    int k = 0;                       // (l t) mod nt
    for (int t = 0; t < nt; ++t) {
        const double2 a = X1[(long long)t * nx + j];
        const double2 w = tw[k];
        re += a.x * w.x - a.y * w.y;
        im += a.x * w.y + a.y * w.x;
        k += l;
        if (k >= nt) k -= nt;
    }
    psd[(long long)l * nx + j] = (re * re + im * im) / ((double)nt * (double)nx);
}
// largest PSD value at wavenumbers 1 <= j <= nx / 2 (ties: lowest l, then j);
// out[0] value, out[1] l, out[2] j
__global__ void k_psd_peak(const double* psd, int nt, int nx, double* out) {
    __shared__ double sv[1024];
    __shared__ long long si[1024];
    const int jm = nx / 2;
    double best = -1.0;
    long long bi = -1;
    for (long long i = threadIdx.x; i < (long long)nt * jm; i += blockDim.x) {
        const int l = (int)(i / jm), j = 1 + (int)(i % jm);
        const double v = psd[(long long)l * nx + j];
        if (v > best) { best = v; bi = i; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int off = 512; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            const double v = sv[threadIdx.x + off];
            const long long i = si[threadIdx.x + off];
            if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && i >= 0 && (si[threadIdx.x] < 0 || i < si[threadIdx.x]))) {
                sv[threadIdx.x] = v;
                si[threadIdx.x] = i;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sv[0];
        out[1] = (double)(si[0] / jm);
        out[2] = (double)(1 + si[0] % jm);
    }
}

int launch_bed_spectrum(const double* h, int nt, int nx, double* psd, double* work, double* peak3, cudaStream_t st) {
    // work: nx + nt twiddles, nt * nx transformed values (complex), the mean
    double2* twx = reinterpret_cast<double2*>(work);
    double2* twt = twx + nx;
    double2* X1 = twt + nt;
    double* mean = reinterpret_cast<double*>(X1 + (size_t)nt * nx);
    k_twiddle<<<blocks_for(nx, 256), 256, 0, st>>>(twx, nx);
    k_twiddle<<<blocks_for(nt, 256), 256, 0, st>>>(twt, nt);
    k_series_mean<<<1, 1024, 0, st>>>(h, (long long)nt * nx, mean);
    k_dft_x<<<dim3((unsigned)blocks_for(nx, 256), (unsigned)nt), 256, 0, st>>>(h, mean, twx, nx, X1);
    k_dft_t<<<dim3((unsigned)blocks_for(nx, 256), (unsigned)nt), 256, 0, st>>>(X1, twt, nt, nx, psd);
    k_psd_peak<<<1, 1024, 0, st>>>(psd, nt, nx, peak3);
    return 6;
}

}  // namespace fsl
