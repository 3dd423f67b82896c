// Fused stream + boundary conditions + mass exchange + cumulant collision
// (Sections 2.1 and 2.2), in place with the AA pattern. One thread per cell.
//
// Even step: each cell reads its own slots (q, x), writes (opp(q), x).
// Odd step: each cell reads (opp(q), x - c_q), writes (q, x + c_q).
// Every boundary condition is applied where a PDF is read: the value a cell
// needs for bounce-back or reconstruction is its own post-collision PDF
// f*_opp(q)(x), which sits in a slot no running cell touches (the slot of a
// solid/gas neighbour, or of the cell itself across a wall face). Interface
// cells read it from a side buffer instead, because the normal-based
// reconstruction also replaces PDFs pulled from fluid neighbours, whose slots
// are being rewritten.
//
// Three kernels share the work: a lean one for bulk liquid cells (all 26
// neighbours liquid), one for the other liquid cells (walls, particle
// links), and one for the interface cells of the interface list.
#include "fslbm_dev.cuh"

namespace fsl {

template <typename S, int PAR>
__global__ void __launch_bounds__(256, 3) k_bulk(Dev s) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= s.n) return;
    if (!(s.flags[cell] & F_BULK)) return;
    int x, y, z;
    coords(s, cell, x, y, z);
    S* f = static_cast<S*>(s.f);
    const long long n = s.n;
    float v[27];
    if (PAR == 0) {
#pragma unroll
        for (int q = 0; q < 27; ++q) v[q] = Store<S>::ld(f + (long long)q * n + cell);
    } else {
        // bulk cells have every neighbour inside the domain; only periodic
        // axes wrap. Offsets of the x, y, z neighbours (-1, 0, +1):
        const int sxy = s.nx * s.ny;
        const int ox[3] = {x == 0 ? s.nx - 1 : -1, 0, x == s.nx - 1 ? 1 - s.nx : 1};
        const int oy[3] = {y == 0 ? (s.ny - 1) * s.nx : -s.nx, 0, y == s.ny - 1 ? (1 - s.ny) * s.nx : s.nx};
        const int oz[3] = {z == 0 ? (s.nz - 1) * sxy : -sxy, 0, z == s.nz - 1 ? (1 - s.nz) * sxy : sxy};
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const int src = cell + ox[1 - cx(q)] + oy[1 - cy(q)] + oz[1 - cz(q)];
            v[q] = Store<S>::ld(f + (long long)opp(q) * n + src);
        }
    }
    float rho, ux, uy, uz;
    collide(v, s.omega, s.gx, s.gy, s.gz, rho, ux, uy, uz);
    if (PAR == 0) {
#pragma unroll
        for (int q = 0; q < 27; ++q) Store<S>::st(f + (long long)opp(q) * n + cell, v[q]);
    } else {
        const int sxy = s.nx * s.ny;
        const int ox[3] = {x == 0 ? s.nx - 1 : -1, 0, x == s.nx - 1 ? 1 - s.nx : 1};
        const int oy[3] = {y == 0 ? (s.ny - 1) * s.nx : -s.nx, 0, y == s.ny - 1 ? (1 - s.ny) * s.nx : s.nx};
        const int oz[3] = {z == 0 ? (s.nz - 1) * sxy : -sxy, 0, z == s.nz - 1 ? (1 - s.nz) * sxy : sxy};
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const int dst = cell + ox[1 + cx(q)] + oy[1 + cy(q)] + oz[1 + cz(q)];
            Store<S>::st(f + (long long)q * n + dst, v[q]);
        }
    }
}

// Warp segmented reduction of per-lane (key, F, T) for runs of equal keys,
// then one FP64 atomic per run and component.
__device__ __forceinline__ void flush_mem(const Dev& s, int key, const float (&F)[3], const float (&T)[3]) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (!__any_sync(full, key >= 0)) return;
    int kprev = __shfl_up_sync(full, key, 1);
    bool head = (lane == 0) || (kprev != key);
    unsigned heads = __ballot_sync(full, head);
    unsigned below = heads & ((2u << lane) - 1u);
    int start = 31 - __clz(below);
    float v[6] = {F[0], F[1], F[2], T[0], T[1], T[2]};
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float t = __shfl_up_sync(full, v[k], off);
            if (lane - off >= start) v[k] += t;
        }
    }
    int knext = __shfl_down_sync(full, key, 1);
    bool tail = (lane == 31) || (knext != key);
    if (tail && key >= 0) {
        atomicAdd(&s.Fh[3 * key + 0], (double)v[0]);
        atomicAdd(&s.Fh[3 * key + 1], (double)v[1]);
        atomicAdd(&s.Fh[3 * key + 2], (double)v[2]);
        atomicAdd(&s.Th[3 * key + 0], (double)v[3]);
        atomicAdd(&s.Th[3 * key + 1], (double)v[4]);
        atomicAdd(&s.Th[3 * key + 2], (double)v[5]);
    }
}

// Per-thread momentum-exchange accumulator with two owner slots; a third
// distinct owner goes straight to the FP64 accumulators.
struct MemAcc {
    int k0, k1;
    float F0[3], T0[3], F1[3], T1[3];
    __device__ __forceinline__ void init() {
        k0 = k1 = -1;
#pragma unroll
        for (int a = 0; a < 3; ++a) F0[a] = T0[a] = F1[a] = T1[a] = 0.f;
    }
    __device__ __forceinline__ void add(const Dev& s, int p, float fx, float fy, float fz, float tx, float ty,
                                        float tz) {
        if (k0 < 0 || k0 == p) {
            k0 = p;
            F0[0] += fx; F0[1] += fy; F0[2] += fz; T0[0] += tx; T0[1] += ty; T0[2] += tz;
        } else if (k1 < 0 || k1 == p) {
            k1 = p;
            F1[0] += fx; F1[1] += fy; F1[2] += fz; T1[0] += tx; T1[1] += ty; T1[2] += tz;
        } else {
            atomicAdd(&s.Fh[3 * p + 0], (double)fx);
            atomicAdd(&s.Fh[3 * p + 1], (double)fy);
            atomicAdd(&s.Fh[3 * p + 2], (double)fz);
            atomicAdd(&s.Th[3 * p + 0], (double)tx);
            atomicAdd(&s.Th[3 * p + 1], (double)ty);
            atomicAdd(&s.Th[3 * p + 2], (double)tz);
        }
    }
    // all lanes of the warp must call this
    __device__ __forceinline__ void flush(const Dev& s) {
        flush_mem(s, k0, F0, T0);
        flush_mem(s, k1, F1, T1);
    }
};

__device__ __forceinline__ float min_image(float d, int L, int periodic) {
    if (periodic) d -= (float)L * rintf(d / (float)L);
    return d;
}

// particle surface velocity at a link midpoint and the link force
// (Section 2.2): f_q = f*_opp + 6 w_q c_q.u_b, force on the particle
// -c_q (f*_opp + f_q) - u_b (f*_opp - f_q) with zero-centred PDFs; torque
// about the centre. The offset from the centre is formed from the integer
// part and the FP32 fraction of the centre, so it is exact to FP32 rounding
// at any lattice size.
__device__ __forceinline__ int wrap_int(int d, int L, int periodic) {
    if (periodic) {
        if (d > L / 2) d -= L;
        else if (d < -L / 2) d += L;
    }
    return d;
}

struct PData {
    int4 xi;
    float4 xf, u, w;
};
__device__ __forceinline__ PData particle_data(const Dev& s, int p) {
    PData d;
    d.xi = s.Xi[p];
    d.xf = s.Xfr[p];
    d.u = s.Uf[p];
    d.w = s.Wf[p];
    return d;
}

__device__ __forceinline__ float particle_link(const Dev& s, int q, int x, int y, int z, int p, const PData& P,
                                               float fo, MemAcc& acc) {
    const float dx = (float)wrap_int(x - P.xi.x, s.nx, s.per_x) + (0.5f - 0.5f * cx(q)) - P.xf.x;
    const float dy = (float)wrap_int(y - P.xi.y, s.ny, s.per_y) + (0.5f - 0.5f * cy(q)) - P.xf.y;
    const float dz = (float)wrap_int(z - P.xi.z, s.nz, s.per_z) + (0.5f - 0.5f * cz(q)) - P.xf.z;
    const float ubx = P.u.x + (P.w.y * dz - P.w.z * dy);
    const float uby = P.u.y + (P.w.z * dx - P.w.x * dz);
    const float ubz = P.u.z + (P.w.x * dy - P.w.y * dx);
    const float cu = cx(q) * ubx + cy(q) * uby + cz(q) * ubz;
    const float val = fo + 6.f * wq(q) * cu;
    const float sum = fo + val, dif = fo - val;
    const float Fx = -cx(q) * sum - ubx * dif;
    const float Fy = -cy(q) * sum - uby * dif;
    const float Fz = -cz(q) * sum - ubz * dif;
    acc.add(s, p, Fx, Fy, Fz, dy * Fz - dz * Fy, dz * Fx - dx * Fz, dx * Fy - dy * Fx);
    return val;
}

// Liquid cells that are not bulk: walls and particle links. All neighbour
// types are read first, then all 27 PDF loads are issued from computed
// addresses (no load sits behind a branch), then the particle links.
constexpr int BOUNDARY_THREADS = 128;

template <typename S, int PAR>
__global__ void __launch_bounds__(BOUNDARY_THREADS) k_boundary(Dev s) {
    __shared__ float sv[27][BOUNDARY_THREADS];
    __shared__ int so[27][BOUNDARY_THREADS];
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool inrange = cell < s.n;
    const uint8_t fl = inrange ? s.flags[cell] : (uint8_t)0;
    const bool work = inrange && (fl & (TYPE_MASK | F_BULK)) == T_LIQ;
    MemAcc acc;
    acc.init();
    if (work) {
        int x, y, z;
        coords(s, cell, x, y, z);
        S* f = static_cast<S*>(s.f);
        const long long n = s.n;
        const int xs[3] = {shift(x, -1, s.nx, s.per_x), x, shift(x, 1, s.nx, s.per_x)};
        const int ys[3] = {shift(y, -1, s.ny, s.per_y), y, shift(y, 1, s.ny, s.per_y)};
        const int zs[3] = {shift(z, -1, s.nz, s.per_z), z, shift(z, 1, s.nz, s.per_z)};
        unsigned wallm = 0, solidm = 0, gasm = 0;
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const int sx = xs[1 - cx(q)], sy = ys[1 - cy(q)], sz = zs[1 - cz(q)];
            if (sx < 0 || sy < 0 || sz < 0) {
                wallm |= 1u << q;
            } else {
                const int ts = s.flags[sx + (long long)s.nx * (sy + (long long)s.ny * sz)] & TYPE_MASK;
                if (ts == T_SOL) solidm |= 1u << q;
                else if (ts == T_GAS) gasm |= 1u << q;
            }
        }
        float v[27];
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const int sx = xs[1 - cx(q)], sy = ys[1 - cy(q)], sz = zs[1 - cz(q)];
            const bool wall = (wallm >> q) & 1u;
            const bool fluid_src = !(((wallm | solidm | gasm) >> q) & 1u);
            const long long src = wall ? cell : sx + (long long)s.nx * (sy + (long long)s.ny * sz);
            long long a;
            if (PAR == 0) a = (fluid_src || wall) ? (long long)q * n + cell : (long long)opp(q) * n + src;
            else a = fluid_src ? (long long)opp(q) * n + src : (long long)q * n + cell;
            v[q] = Store<S>::ld(f + a);
        }
        // a liquid cell must not touch gas; if it does, the gas-side PDF is
        // bounced back and the event counted
        if (gasm) atomicAdd(s.viol, 1ull);
        if (solidm) {
            // particle links: the owners of all solid directions are loaded
            // together, the cell's values staged in shared memory, and one
            // copy of the link code runs over the solid directions with the
            // particle data cached per owner
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                sv[q][threadIdx.x] = v[q];
                if ((solidm >> q) & 1u) {
                    const int sx = xs[1 - cx(q)], sy = ys[1 - cy(q)], sz = zs[1 - cz(q)];
                    so[q][threadIdx.x] = s.owner[sx + (long long)s.nx * (sy + (long long)s.ny * sz)];
                }
            }
            int pc = -1;
            PData P;
            unsigned m = solidm;
            while (m) {
                const int q = __ffs(m) - 1;
                m &= m - 1;
                const int p = so[q][threadIdx.x];
                if (p < 0 || p >= s.np) { set_error(s, ERR_INVARIANT); continue; }
                if (p != pc) {
                    P = particle_data(s, p);
                    pc = p;
                }
                sv[q][threadIdx.x] = particle_link(s, q, x, y, z, p, P, sv[q][threadIdx.x], acc);
            }
#pragma unroll
            for (int q = 0; q < 27; ++q) v[q] = sv[q][threadIdx.x];
        }
        float rho, ux, uy, uz;
        collide(v, s.omega, s.gx, s.gy, s.gz, rho, ux, uy, uz);
        if (PAR == 0) {
#pragma unroll
            for (int q = 0; q < 27; ++q) Store<S>::st(f + (long long)opp(q) * n + cell, v[q]);
        } else {
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const int tx = xs[1 + cx(q)], ty = ys[1 + cy(q)], tz = zs[1 + cz(q)];
                const bool out = tx < 0 || ty < 0 || tz < 0;
                const long long a = out ? (long long)opp(q) * n + cell
                                        : (long long)q * n + tx + (long long)s.nx * (ty + (long long)s.ny * tz);
                Store<S>::st(f + a, v[q]);
            }
        }
    }
    acc.flush(s);
}

// Interface cells, from the interface list: gas-pressure reconstruction
// (Section 2.1), mass exchange, particle links, collision; the cell's own
// post-collision PDFs come from and go to the side buffer.
template <typename S, int PAR>
__global__ void __launch_bounds__(128) k_interface(Dev s) {
    const int count = min(*s.wl_count, s.wl_cap);
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < count; base += stride) {
        const int i = base + threadIdx.x;
        const bool work = i < count;
        MemAcc acc;
        acc.init();
        if (work) {
            const long long cell = s.wl[i];
            int x, y, z;
            coords(s, cell, x, y, z);
            S* f = static_cast<S*>(s.f);
            S* fs = static_cast<S*>(s.fs);
            const long long n = s.n;
            const int xs[3] = {shift(x, -1, s.nx, s.per_x), x, shift(x, 1, s.nx, s.per_x)};
            const int ys[3] = {shift(y, -1, s.ny, s.per_y), y, shift(y, 1, s.ny, s.per_y)};
            const int zs[3] = {shift(z, -1, s.nz, s.per_z), z, shift(z, 1, s.nz, s.per_z)};
            unsigned wallm = 0, solidm = 0, gasm = 0, liqm = 0;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const int sx = xs[1 - cx(q)], sy = ys[1 - cy(q)], sz = zs[1 - cz(q)];
                if (sx < 0 || sy < 0 || sz < 0) {
                    wallm |= 1u << q;
                } else {
                    const int ts = s.flags[sx + (long long)s.nx * (sy + (long long)s.ny * sz)] & TYPE_MASK;
                    if (ts == T_SOL) solidm |= 1u << q;
                    else if (ts == T_GAS) gasm |= 1u << q;
                    else if (ts == T_LIQ) liqm |= 1u << q;
                }
            }
            const float phix = s.phi[cell];
            const float mx = s.mass[cell];
            const float4 nn = s.nrm[cell];
            float fo[27];
#pragma unroll
            for (int q = 0; q < 27; ++q) fo[q] = Store<S>::ld(fs + (long long)q * n + cell);
            float v[27];
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const int sx = xs[1 - cx(q)], sy = ys[1 - cy(q)], sz = zs[1 - cz(q)];
                const bool fluid_src = !(((wallm | solidm | gasm) >> q) & 1u);
                const long long src = fluid_src ? sx + (long long)s.nx * (sy + (long long)s.ny * sz) : cell;
                const long long a = PAR == 0 ? (long long)q * n + cell : (long long)opp(q) * n + src;
                v[q] = fluid_src ? Store<S>::ld(f + a) : 0.f;
            }
            // own collision velocity from the post-collision PDFs
            float d = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                d += fo[q];
                jx += cx(q) * fo[q];
                jy += cy(q) * fo[q];
                jz += cz(q) * fo[q];
            }
            const float rr = 1.f + d;
            const float urx = (jx - 0.5f * rr * s.gx) / rr;
            const float ury = (jy - 0.5f * rr * s.gy) / rr;
            const float urz = (jz - 0.5f * rr * s.gz) / rr;
            const float uur = urx * urx + ury * ury + urz * urz;
            const float rhoG = s.rho_gas;
            float dm = 0.f;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const float fob = fo[opp(q)];
                if ((wallm >> q) & 1u) {
                    v[q] = fob;
                    continue;
                }
                const int sx = xs[1 - cx(q)], sy = ys[1 - cy(q)], sz = zs[1 - cz(q)];
                const long long src = sx + (long long)s.nx * (sy + (long long)s.ny * sz);
                if ((solidm >> q) & 1u) {
                    const int p = s.owner[src];
                    if (p < 0 || p >= s.np) { set_error(s, ERR_INVARIANT); v[q] = fob; continue; }
                    v[q] = particle_link(s, q, x, y, z, p, particle_data(s, p), fob, acc);
                    continue;
                }
                const bool gas = (gasm >> q) & 1u;
                if (!gas) {
                    // fluid source: mass exchange with the pulled post-collision PDF
                    const bool liq = (liqm >> q) & 1u;
                    const float sc = liq ? 1.f : 0.5f * (phix + s.phi[src]);
                    dm += sc * (v[q] - fob);
                }
                bool rebuild = gas;
                if (!rebuild && s.recon_normal) rebuild = (nn.x * cx(q) + nn.y * cy(q) + nn.z * cz(q)) < -s.eps_normal;
                if (rebuild) {
                    const float cu = cx(q) * urx + cy(q) * ury + cz(q) * urz;
                    v[q] = wq(q) * (2.f * (rhoG - 1.f) + rhoG * (9.f * cu * cu - 3.f * uur)) - fob;
                }
            }
            float rho, ux, uy, uz;
            collide(v, s.omega, s.gx, s.gy, s.gz, rho, ux, uy, uz);
            if (PAR == 0) {
#pragma unroll
                for (int q = 0; q < 27; ++q) Store<S>::st(f + (long long)opp(q) * n + cell, v[q]);
            } else {
#pragma unroll
                for (int q = 0; q < 27; ++q) {
                    const int tx = xs[1 + cx(q)], ty = ys[1 + cy(q)], tz = zs[1 + cz(q)];
                    const bool out = tx < 0 || ty < 0 || tz < 0;
                    const long long a = out ? (long long)opp(q) * n + cell
                                            : (long long)q * n + tx + (long long)s.nx * (ty + (long long)s.ny * tz);
                    Store<S>::st(f + a, v[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < 27; ++q) Store<S>::st(fs + (long long)q * n + cell, v[q]);
            // phi = m / rho is refreshed after the sweep: neighbours read the
            // old phi in their mass exchange
            s.mass[cell] = mx + dm;
            s.ru[cell] = make_float4(rho, ux, uy, uz);
        }
        acc.flush(s);
    }
}

template <typename S>
static void launch_typed(const Dev& s, int parity, cudaStream_t st) {
    const int th = 256;
    const int bl = blocks_for(s.n, th);
    const int ib = 152 * 8;
    if (parity == 0) {
        k_bulk<S, 0><<<bl, th, 0, st>>>(s);
        k_boundary<S, 0><<<blocks_for(s.n, BOUNDARY_THREADS), BOUNDARY_THREADS, 0, st>>>(s);
        k_interface<S, 0><<<ib, 128, 0, st>>>(s);
    } else {
        k_bulk<S, 1><<<bl, th, 0, st>>>(s);
        k_boundary<S, 1><<<blocks_for(s.n, BOUNDARY_THREADS), BOUNDARY_THREADS, 0, st>>>(s);
        k_interface<S, 1><<<ib, 128, 0, st>>>(s);
    }
}

int launch_stream_collide(const Dev& s, int parity, cudaStream_t st) {
    if (s.storage == FSLBM_STORE_FP32) launch_typed<float>(s, parity, st);
    else if (s.storage == FSLBM_STORE_FP16) launch_typed<__half>(s, parity, st);
    else launch_typed<__nv_bfloat16>(s, parity, st);
    return 3;
}

}  // namespace fsl
