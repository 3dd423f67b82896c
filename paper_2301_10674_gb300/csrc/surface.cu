// Free-surface (volume-of-fluid) update after the stream-collide sweep
// (Section 2.1): fill levels, interface normals, conversion of interface
// cells, filling/emptying of their neighbours, excess-mass redistribution,
// the FP64 mass pool, and the interface work list. Every kernel below works
// on the device-counted list of interface cells (or of cells becoming
// interface), so its cost scales with the surface, not the lattice; each
// cell computes its own result from a snapshot of its neighbourhood, so no
// result depends on thread order.
#include "fslbm_dev.cuh"
#include "mlp_dev.cuh"

namespace fsl {

constexpr int LIST_THREADS = 256;
constexpr int LIST_BLOCKS = 152 * 4;

#define FOR_LIST(i, countp)                                                       \
    for (int i = blockIdx.x * blockDim.x + threadIdx.x, _cnt = *(countp); i < _cnt; \
         i += gridDim.x * blockDim.x)

__device__ __forceinline__ bool is_fluid(int t) { return t == T_LIQ || t == T_IFC; }

// ------------------------------------------------------------ fill levels
__global__ void k_update_phi(Dev s) {
    FOR_LIST(i, s.wl_count) {
        int c = s.wl[i];
        s.phi[c] = s.mass[c] / s.ru[c].x;
    }
}

// Parker-Youngs normal: gradient sum_c w(c) c phi(x+c) with weights 4 (face),
// 2 (edge), 1 (corner); solid and wall neighbours take the centre value;
// n = -grad/|grad| points toward the gas.
__device__ float4 py_normal(const Dev& s, long long c) {
    int x, y, z;
    coords(s, c, x, y, z);
    const int t0 = s.flags[c] & TYPE_MASK;
    const float p0 = t0 == T_LIQ ? 1.f : (t0 == T_IFC ? s.phi[c] : 0.f);
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        if (q == 13) continue;
        const float w = nnz(q) == 1 ? 4.f : (nnz(q) == 2 ? 2.f : 1.f);
        long long nb = nbr(s, x, y, z, cx(q), cy(q), cz(q));
        float v;
        if (nb < 0) v = p0;
        else {
            int tn = s.flags[nb] & TYPE_MASK;
            v = tn == T_LIQ ? 1.f : (tn == T_IFC ? s.phi[nb] : (tn == T_GAS ? 0.f : p0));
        }
        gx += w * cx(q) * v;
        gy += w * cy(q) * v;
        gz += w * cz(q) * v;
    }
    float len = sqrtf(gx * gx + gy * gy + gz * gz);
    if (len > 0.f) return make_float4(-gx / len, -gy / len, -gz / len, 0.f);
    return make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_normals(Dev s, float4* out, const int* list, const int* countp) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x, cnt = min(*countp, s.wl_cap); i < cnt;
         i += gridDim.x * blockDim.x) {
        int c = list[i];
        out[c] = py_normal(s, c);
    }
}

// Learned normal (R-17), a warp per 16 interface cells of the list. Lane
// (g, t) loads the stencil columns of its input fragments for the cells of
// rows g and g + 8; together the four lanes of a group cover all 27, agree on
// whether a wall or solid cell lies in the block, and sum the Parker-Youngs
// gradient from the same values (walls and solids taking the centre value).
// The Parker-Youngs normal is both the fallback (wall or solid in the block,
// raw length outside [1/2, 2]) and the check on the network (its normal more
// than 30 degrees away falls back too). out[c] = (n, curvature), curvature 0 where the fallback is
// taken.
__global__ void __launch_bounds__(128, 5) k_mlp_normals(Dev s, float4* out, const int* list, const int* countp) {
    const int count = min(*countp, s.wl_cap);
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const unsigned full = 0xffffffffu;
    unsigned long long evaluated = 0, taken = 0;
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 16; base < count; base += nwarps * 16) {
        int cell[2];
        float v[2][8];
        bool bad[2];
        float gr[2][3];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int li = base + g + 8 * r;
            cell[r] = li < count ? list[li] : -1;
            bad[r] = false;
            gr[r][0] = gr[r][1] = gr[r][2] = 0.f;
            int x = 0, y = 0, z = 0;
            float p0 = 0.f;
            if (cell[r] >= 0) {
                coords(s, cell[r], x, y, z);
                p0 = s.phi[cell[r]];
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = frag_col(j >> 2, j & 3, t);
                float in = 0.f, raw = p0;
                if (cell[r] >= 0 && col < 27) {
                    const long long nb = nbr(s, x, y, z, cx(col), cy(col), cz(col));
                    if (nb < 0) {
                        bad[r] = true;
                    } else {
                        const int tn = s.flags[nb] & TYPE_MASK;
                        if (tn == T_SOL) {
                            bad[r] = true;
                        } else {
                            raw = tn == T_LIQ ? 1.f : (tn == T_IFC ? s.phi[nb] : 0.f);
                            in = fminf(fmaxf(raw, 0.f), 1.f);
                        }
                    }
                    if (col != 13) {
                        const float w = nnz(col) == 1 ? 4.f : (nnz(col) == 2 ? 2.f : 1.f);
                        gr[r][0] += w * cx(col) * raw;
                        gr[r][1] += w * cy(col) * raw;
                        gr[r][2] += w * cz(col) * raw;
                    }
                }
                v[r][j] = in;
            }
            bad[r] |= __shfl_xor_sync(full, bad[r], 1);
            bad[r] |= __shfl_xor_sync(full, bad[r], 2);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gr[r][k] += __shfl_xor_sync(full, gr[r][k], 1);
                gr[r][k] += __shfl_xor_sync(full, gr[r][k], 2);
            }
        }
        uint32_t xf[2][4];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            xf[kk][0] = pack_bf16(v[0][4 * kk + 0], v[0][4 * kk + 1]);
            xf[kk][1] = pack_bf16(v[1][4 * kk + 0], v[1][4 * kk + 1]);
            xf[kk][2] = pack_bf16(v[0][4 * kk + 2], v[0][4 * kk + 3]);
            xf[kk][3] = pack_bf16(v[1][4 * kk + 2], v[1][4 * kk + 3]);
        }
        // R-17g with mlp_mirror: the network also on the stencil mirrored in
        // x, in y and in both (the first layer with permuted columns on the
        // same inputs), each output mapped back and the four averaged
        MlpAct act;
        float y[2][4];
        const int passes = s.mlp_mirror ? 4 : 1;
#pragma unroll 1
        for (int m = 0; m < passes; ++m) {
            const MlpBf16* W = s.mlp;
            const MlpFrag* G = s.mlp_frag;
            // the operands are reloaded in every pass rather than held in
            // registers across passes
            asm volatile("" : "+l"(W), "+l"(G));
            mlp_forward_frag(*W, *G, m, xf, act);
            float ym[2][4];
            mlp_outputs(act, ym[0], ym[1]);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (m == 0) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) y[r][k] = ym[r][k];
                } else {
                    y[r][0] += (m & 1) ? -ym[r][0] : ym[r][0];
                    y[r][1] += (m & 2) ? -ym[r][1] : ym[r][1];
                    y[r][2] += ym[r][2];
                    y[r][3] += ym[r][3];
                }
            }
        }
        if (passes == 4) {
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int k = 0; k < 4; ++k) y[r][k] *= 0.25f;
        }
        if (t < 2 && cell[t] >= 0) {
            const int c = cell[t];
            const float gl = sqrtf(gr[t][0] * gr[t][0] + gr[t][1] * gr[t][1] + gr[t][2] * gr[t][2]);
            const float4 fd = gl > 0.f ? make_float4(-gr[t][0] / gl, -gr[t][1] / gl, -gr[t][2] / gl, 0.f)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 res = fd;
            ++evaluated;
            const float len = sqrtf(y[t][0] * y[t][0] + y[t][1] * y[t][1] + y[t][2] * y[t][2]);
            if (!bad[t] && len >= 0.5f && len <= 2.f) {
                const float mx = y[t][0] / len, my = y[t][1] / len, mz = y[t][2] / len;
                if (mx * fd.x + my * fd.y + mz * fd.z >= 0.8660254f) {   // cos 30 degrees
                    res = make_float4(mx, my, mz, y[t][3]);
                    ++taken;
                }
            }
            out[c] = res;
        }
    }
    if (s.mlp_stats) {
        for (int o = 16; o > 0; o >>= 1) {
            evaluated += __shfl_xor_sync(full, evaluated, o);
            taken += __shfl_xor_sync(full, taken, o);
        }
        if (lane == 0 && evaluated) {
            atomicAdd(&s.mlp_stats[0], evaluated);
            atomicAdd(&s.mlp_stats[1], taken);
        }
    }
}

// normals of the cells of a list (the interface list, or the cells that
// convert in this step)
static int normals_into(const Dev& s, float4* out, const int* list, const int* count, cudaStream_t st) {
    if (s.mlp) k_mlp_normals<<<152 * 8, 128, 0, st>>>(s, out, list, count);
    else k_normals<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(s, out, list, count);
    return 1;
}

// ------------------------------------------------------------ conversion
// candidates: fill level beyond 1 + eps or below -eps, or isolation (no gas
// neighbour -> liquid, no liquid neighbour -> gas)
__global__ void k_candidates(Dev s) {
    FOR_LIST(i, s.wl_count) {
        int c = s.wl[i];
        int x, y, z;
        coords(s, c, x, y, z);
        bool has_gas = false, has_liq = false;
        for (int q = 0; q < 27; ++q) {
            if (q == 13) continue;
            long long nb = nbr(s, x, y, z, cx(q), cy(q), cz(q));
            if (nb < 0) continue;
            int tn = s.flags[nb] & TYPE_MASK;
            has_gas |= tn == T_GAS;
            has_liq |= tn == T_LIQ;
        }
        float ph = s.phi[c];
        uint8_t cv = 0;
        if (ph > 1.f + s.eps_conv) cv = CV_TO_LIQ;
        else if (ph < -s.eps_conv) cv = CV_TO_GAS;
        else if (!has_gas) cv = CV_TO_LIQ;
        else if (!has_liq) cv = CV_TO_GAS;
        s.conv[c] = cv;
    }
}

__device__ __forceinline__ void list_push(const Dev& s, int* list, int* count, int cap, int v) {
    int k = atomicAdd(count, 1);
    if (k < cap) list[k] = v;
    else set_error(s, ERR_CAPACITY);
}

// filling wins: a to-gas cell next to a to-liquid cell stays interface. The
// cells that still convert are listed (their normals give the excess-mass
// weights).
__global__ void k_conflict(Dev s) {
    FOR_LIST(i, s.wl_count) {
        int c = s.wl[i];
        const uint8_t cv = s.conv[c];
        if (!cv) continue;
        if (cv == CV_TO_GAS) {
            int x, y, z;
            coords(s, c, x, y, z);
            bool clash = false;
            for (int q = 0; q < 27 && !clash; ++q) {
                if (q == 13) continue;
                long long nb = nbr(s, x, y, z, cx(q), cy(q), cz(q));
                if (nb >= 0 && s.conv[nb] == CV_TO_LIQ) clash = true;
            }
            if (clash) {
                s.conv[c] = 0;
                continue;
            }
        }
        list_push(s, s.cl, s.cl_count, s.wl_cap, c);
    }
}

// gas neighbours of filled cells and liquid neighbours of emptied cells
// become interface cells; each is listed once (first setter of its mark)
// (over the cells that convert, listed by k_conflict)
__global__ void k_mark(Dev s) {
    const int ncl = min(*s.cl_count, s.wl_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncl; i += gridDim.x * blockDim.x) {
        int c = s.cl[i];
        uint8_t cv = s.conv[c];
        if (!cv) continue;
        int x, y, z;
        coords(s, c, x, y, z);
        for (int q = 0; q < 27; ++q) {
            if (q == 13) continue;
            long long nb = nbr(s, x, y, z, cx(q), cy(q), cz(q));
            if (nb < 0) continue;
            int tn = s.flags[nb] & TYPE_MASK;
            uint8_t bit = 0;
            if (cv == CV_TO_LIQ && tn == T_GAS) bit = F_NEW;
            if (cv == CV_TO_GAS && tn == T_LIQ) bit = F_EMPTIED;
            if (!bit) continue;
            uint8_t old = flag_or(s.flags, nb, bit);
            if (!(old & bit)) list_push(s, s.nl, s.nl_count, s.nl_cap, (int)nb);
        }
    }
}

// new interface cells: from gas, f* = f_eq(mean rho, mean u) of the liquid
// and interface neighbours (cell types of the snapshot) with m = 0; from
// liquid, PDFs kept and m = rho. Both get their own PDFs in the side buffer.
__global__ void k_init_new(Dev s, int last_parity) {
    FOR_LIST(i, s.nl_count) {
        if (i >= s.nl_cap) break;
        const int c = s.nl[i];
        const uint8_t fl = s.flags[c];
        float f[27];
        float rho, ux, uy, uz;
        if (fl & F_NEW) {
            int x, y, z;
            coords(s, c, x, y, z);
            float rs = 0.f, us = 0.f, vs = 0.f, ws = 0.f;
            int cnt = 0;
            // rolled: the 27 loads per liquid neighbour make an unrolled loop
            // bound by instruction fetch
#pragma unroll 1
            for (int q = 0; q < 27; ++q) {
                if (q == 13) continue;
                long long nb = nbr(s, x, y, z, cx(q), cy(q), cz(q));
                if (nb < 0) continue;
                int tn = s.flags[nb] & TYPE_MASK;
                if (tn == T_IFC) {
                    float4 r = s.ru[nb];
                    rs += r.x; us += r.y; vs += r.z; ws += r.w;
                    cnt++;
                } else if (tn == T_LIQ) {
                    float g[27];
                    load_fstar(s, nb, last_parity, g);
                    float r0, a, b, d;
                    post_moments(s, g, r0, a, b, d);
                    rs += r0; us += a; vs += b; ws += d;
                    cnt++;
                }
            }
            float inv = cnt ? 1.f / cnt : 0.f;
            rho = cnt ? rs * inv : s.rho_gas;
            ux = us * inv; uy = vs * inv; uz = ws * inv;
#pragma unroll
            for (int q = 0; q < 27; ++q) f[q] = feq_dev(q, rho, ux, uy, uz);
            store_fstar(s, c, last_parity, f);
            s.mass[c] = 0.f;
        } else {
            load_fstar(s, c, last_parity, f);
            post_moments(s, f, rho, ux, uy, uz);
            s.mass[c] = rho;
        }
        for (int q = 0; q < 27; ++q) st_any(s, s.fs, (long long)q * s.n + c, f[q]);
        s.ru[c] = make_float4(rho, ux, uy, uz);
    }
}

__device__ __forceinline__ bool is_receiver(const Dev& s, long long c) {
    uint8_t fl = s.flags[c];
    if (fl & (F_NEW | F_EMPTIED)) return true;
    return (fl & TYPE_MASK) == T_IFC && (s.conv[c] & 3) == 0;
}

// excess mass of converting cells: m - rho (to liquid, m := rho) or m (to
// gas, m := 0), spread over interface neighbours with weights max(0, n.c)
// (filled) or max(0, -n.c) (emptied), evenly if all weights vanish or the
// even variant is selected, into the FP64 pool if there is no interface
// neighbour
__global__ void k_excess_prep(Dev s) {
    const int ncl = min(*s.cl_count, s.wl_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncl; i += gridDim.x * blockDim.x) {
        int c = s.cl[i];
        uint8_t cv = s.conv[c];
        if (!cv) continue;
        float rho = s.ru[c].x;
        float m = s.mass[c];
        float ex;
        if (cv == CV_TO_LIQ) { ex = m - rho; s.mass[c] = rho; }
        else { ex = m; s.mass[c] = 0.f; }
        float sg = cv == CV_TO_LIQ ? 1.f : -1.f;
        float4 n1 = s.nrm1[c];
        int x, y, z;
        coords(s, c, x, y, z);
        float wsum = 0.f;
        int nrec = 0;
        for (int q = 0; q < 27; ++q) {
            if (q == 13) continue;
            long long nb = nbr(s, x, y, z, cx(q), cy(q), cz(q));
            if (nb < 0 || !is_receiver(s, nb)) continue;
            float w = sg * (n1.x * cx(q) + n1.y * cy(q) + n1.z * cz(q));
            wsum += w > 0.f ? w : 0.f;
            nrec++;
        }
        if (nrec == 0) {
            atomicAdd(s.pool, (double)ex);
            s.exscale[c] = 0.f;
        } else if (wsum > 0.f && !s.excess_even) {
            s.exscale[c] = ex / wsum;
        } else {
            s.exscale[c] = ex / (float)nrec;
            s.conv[c] = cv | CV_EVEN;
        }
    }
}

__device__ void gather_excess(const Dev& s, int c) {
    if (!is_receiver(s, c)) return;
    int x, y, z;
    coords(s, c, x, y, z);
    float add = 0.f;
    for (int q = 0; q < 27; ++q) {
        if (q == 13) continue;
        long long nb = nbr(s, x, y, z, cx(q), cy(q), cz(q));
        if (nb < 0) continue;
        uint8_t cv = s.conv[nb];
        if (!(cv & 3)) continue;
        float w;
        if (cv & CV_EVEN) w = 1.f;
        else {
            // direction from the converting cell to this receiver is -c_q
            float4 n1 = s.nrm1[nb];
            float sg = (cv & 3) == CV_TO_LIQ ? 1.f : -1.f;
            w = -sg * (n1.x * cx(q) + n1.y * cy(q) + n1.z * cz(q));
            w = w > 0.f ? w : 0.f;
        }
        add += s.exscale[nb] * w;
    }
    s.mass[c] += add;
}

__global__ void k_excess_gather(Dev s) {
    // without a converting cell no receiver gets anything
    if (*s.cl_count == 0) return;
    FOR_LIST(i, s.wl_count) gather_excess(s, s.wl[i]);
    const int cap = s.nl_cap;
    FOR_LIST(i, s.nl_count) {
        if (i >= cap) break;
        gather_excess(s, s.nl[i]);
    }
}

__global__ void k_finalize_old(Dev s) {
    FOR_LIST(i, s.wl_count) {
        int c = s.wl[i];
        uint8_t cv = s.conv[c] & 3;
        if (cv == CV_TO_LIQ) {
            s.flags[c] = T_LIQ;
        } else if (cv == CV_TO_GAS) {
            s.flags[c] = T_GAS;
            s.mass[c] = 0.f;
            s.phi[c] = 0.f;
        } else {
            s.phi[c] = s.mass[c] / s.ru[c].x;
        }
    }
}
__global__ void k_finalize_new(Dev s) {
    const int cap = s.nl_cap;
    FOR_LIST(i, s.nl_count) {
        if (i >= cap) break;
        int c = s.nl[i];
        s.flags[c] = T_IFC;
        s.phi[c] = s.mass[c] / s.ru[c].x;
    }
}
// conversion codes are left only on the cells k_conflict listed
__global__ void k_clear_conv(Dev s) {
    const int ncl = min(*s.cl_count, s.wl_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncl; i += gridDim.x * blockDim.x) s.conv[s.cl[i]] = 0;
}

// Interface stencils of the current state with height-function labels (R-17e):
// a thread per interface cell. The input is the learned normal's: the fill
// levels of the 3x3x3 block (liquid 1, interface phi clamped to [0, 1], gas
// 0), stencil index (dx+1) + 3(dy+1) + 9(dz+1); a block with a wall or solid
// cell is not logged. The label follows the height-function method: along
// the axis a where the Parker-Youngs normal is largest (gas toward sign
// sg), the fill levels of the 3x3 columns of 7 cells centred on the cell's
// row sum to the heights eta(i, j) = sum - 7/2 of the surface above the
// column's centre plane, measured toward the gas; a column counts only if
// its liquid end cell is liquid and its gas end cell gas. With eta_u, eta_v
// the central differences and eta_uu, eta_vv, eta_uv the second ones, the
// normal toward the gas is (sg e_a - eta_u e_u - eta_v e_v) / |.| and the
// mean curvature, positive for a convex liquid body,
//   kappa = -(eta_uu (1 + eta_v^2) + eta_vv (1 + eta_u^2) - 2 eta_u eta_v eta_uv)
//           / (2 (1 + eta_u^2 + eta_v^2)^(3/2)).
// Written per logged cell: fill[27], target = (n, kappa), fd = (Parker-Youngs
// normal, 0) and the cell index, at slots taken in no fixed order; `found`
// counts every valid cell, the first `cap` of them are written.
// fill level (clamped, and raw in `raw`) and type of a neighbour; false
// beyond a wall face or at a solid cell
__device__ __forceinline__ bool fill_at(const Dev& s, int x, int y, int z, int dx, int dy, int dz, float& v, int& t,
                                        float& raw) {
    const long long nb = nbr(s, x, y, z, dx, dy, dz);
    if (nb < 0) return false;
    t = s.flags[nb] & TYPE_MASK;
    if (t == T_SOL) return false;
    raw = t == T_LIQ ? 1.f : (t == T_IFC ? s.phi[nb] : 0.f);
    v = fminf(fmaxf(raw, 0.f), 1.f);
    return true;
}

__global__ void k_log_stencils(Dev s, long long cap, float* fill, float4* target, float4* fd, int* cells,
                               unsigned long long* found) {
    const int count = min(*s.wl_count, s.wl_cap);
    const int stride = gridDim.x * blockDim.x;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < count; base += stride) {
        const int i = base + threadIdx.x;
        bool ok = false;
        float in[27];
        float4 lab = make_float4(0.f, 0.f, 0.f, 0.f), pyn = lab;
        int c = -1;
        if (i < count) {
            c = s.wl[i];
            int x, y, z;
            coords(s, c, x, y, z);
            ok = true;
            float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                float v = 0.f, raw = 0.f;
                int t = 0;
                if (!fill_at(s, x, y, z, cx(q), cy(q), cz(q), v, t, raw)) ok = false;
                in[q] = v;
                // the Parker-Youngs gradient of the raw fill levels
                if (q != 13) {
                    const float w = nnz(q) == 1 ? 4.f : (nnz(q) == 2 ? 2.f : 1.f);
                    gx += w * cx(q) * raw;
                    gy += w * cy(q) * raw;
                    gz += w * cz(q) * raw;
                }
            }
            const float gl = sqrtf(gx * gx + gy * gy + gz * gz);
            if (!(gl > 0.f)) ok = false;
            if (ok) {
                pyn = make_float4(-gx / gl, -gy / gl, -gz / gl, 0.f);
                // the dominant axis from the gradient itself (ties: the lower axis)
                const float g[3] = {gx, gy, gz};
                const int a = (fabsf(gx) >= fabsf(gy) && fabsf(gx) >= fabsf(gz)) ? 0 : (fabsf(gy) >= fabsf(gz) ? 1 : 2);
                const int u = a == 0 ? 1 : 0, v = a == 2 ? 1 : 2;
                const int sg = g[a] < 0.f ? 1 : -1;   // the normal -grad points to the gas
                float eta[3][3];
                for (int iu = -1; iu <= 1 && ok; ++iu)
                    for (int iv = -1; iv <= 1 && ok; ++iv) {
                        float sum = 0.f;
                        for (int t = -3; t <= 3 && ok; ++t) {
                            int d[3] = {0, 0, 0};
                            d[u] = iu;
                            d[v] = iv;
                            d[a] = sg * t;
                            float f = 0.f, fr = 0.f;
                            int ty = 0;
                            if (!fill_at(s, x, y, z, d[0], d[1], d[2], f, ty, fr)) ok = false;
                            else if ((t == -3 && ty != T_LIQ) || (t == 3 && ty != T_GAS)) ok = false;
                            sum += f;
                        }
                        eta[iu + 1][iv + 1] = sum - 3.5f;
                    }
                if (ok) {
                    const float eu = 0.5f * (eta[2][1] - eta[0][1]), ev = 0.5f * (eta[1][2] - eta[1][0]);
                    const float euu = eta[2][1] - 2.f * eta[1][1] + eta[0][1];
                    const float evv = eta[1][2] - 2.f * eta[1][1] + eta[1][0];
                    const float euv = 0.25f * (eta[2][2] - eta[2][0] - eta[0][2] + eta[0][0]);
                    const float g2 = 1.f + eu * eu + ev * ev;
                    const float inv = rsqrtf(g2);
                    float m[3];
                    m[a] = sg * inv;
                    m[u] = -eu * inv;
                    m[v] = -ev * inv;
                    const float kap = -(euu * (1.f + ev * ev) + evv * (1.f + eu * eu) - 2.f * eu * ev * euv) /
                                      (2.f * g2 * sqrtf(g2));
                    lab = make_float4(m[0], m[1], m[2], kap);
                }
            }
        }
        // warp-aggregated slots
        const unsigned bal = __ballot_sync(full, ok);
        unsigned long long slot0 = 0;
        if (bal) {
            const int leader = __ffs(bal) - 1;
            if (lane == leader) slot0 = atomicAdd(found, (unsigned long long)__popc(bal));
            slot0 = __shfl_sync(full, slot0, leader);
        }
        if (ok) {
            const unsigned long long k = slot0 + __popc(bal & ((1u << lane) - 1u));
            if ((long long)k < cap) {
#pragma unroll
                for (int q = 0; q < 27; ++q) fill[k * 27 + q] = in[q];
                target[k] = lab;
                if (fd) fd[k] = pyn;
                if (cells) cells[k] = c;
            }
        }
    }
}

void launch_log_stencils(const Dev& s, long long cap, float* fill, float* target, float* fd, int* cells,
                         unsigned long long* found, cudaStream_t st) {
    cudaMemsetAsync(found, 0, sizeof(unsigned long long), st);
    k_log_stencils<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(s, cap, fill, reinterpret_cast<float4*>(target),
                                                          reinterpret_cast<float4*>(fd), cells, found);
}

int launch_normals(const Dev& s, float4* out, cudaStream_t st) { return normals_into(s, out, s.wl, s.wl_count, st); }

int launch_conversion(const Dev& s, int last_parity, cudaStream_t st) {
    k_update_phi<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(s);
    k_candidates<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(s);
    cudaMemsetAsync(s.cl_count, 0, sizeof(int), st);
    k_conflict<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(s);
    // the excess-mass weights need the normals of the converting cells only;
    // fill levels and types are those k_update_phi left
    normals_into(s, s.nrm1, s.cl, s.cl_count, st);
    cudaMemsetAsync(s.nl_count, 0, sizeof(int), st);
    k_mark<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(s);
    k_init_new<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(s, last_parity);
    k_excess_prep<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(s);
    k_excess_gather<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(s);
    k_finalize_old<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(s);
    k_finalize_new<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(s);
    k_clear_conv<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(s);
    return 12;
}

// ------------------------------------------------------------ work lists
// Block-aggregated append of the cells c0 + k for the set bits k of a
// thread's two 32-bit masks, ma to list la and mb to list lb: one scan of
// both counts (list a in the low 16 bits, list b in the high ones; a block
// holds at most 32 x 32 bits per warp), one atomic per list and block. The
// cells of a block keep their order in each list. Every thread of the block
// must call it.
__device__ __forceinline__ void block_append_masks(const Dev& s, int c0, unsigned ma, int* la, int* ca, int capa,
                                                   unsigned mb, int* lb, int* cb, int capb) {
    __shared__ int warp_tot[32];
    __shared__ int base_a, base_b;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int na = __popc(ma), nb = __popc(mb);
    int incl = na | (nb << 16);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(full, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ta = 0, tb = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int c = warp_tot[w];
            warp_tot[w] = ta | (tb << 16);
            ta += c & 0xffff;
            tb += c >> 16;
        }
        base_a = ta ? atomicAdd(ca, ta) : 0;
        base_b = tb ? atomicAdd(cb, tb) : 0;
    }
    __syncthreads();
    const int pre = warp_tot[wid];
    int ka = base_a + (pre & 0xffff) + (incl & 0xffff) - na;
    int kb = base_b + (pre >> 16) + (incl >> 16) - nb;
    for (unsigned m = ma; m; m &= m - 1, ++ka) {
        if (ka < capa) la[ka] = c0 + __ffs(m) - 1;
        else set_error(s, ERR_CAPACITY);
    }
    for (unsigned m = mb; m; m &= m - 1, ++kb) {
        if (kb < capb) lb[kb] = c0 + __ffs(m) - 1;
        else set_error(s, ERR_CAPACITY);
    }
    __syncthreads();
}

// Lists the interface cells and the solid cells with a liquid or interface
// cell among their 26 neighbours, for lattices whose x extent is a multiple of
// 32. First pass, a thread per 32 consecutive cells of a row: their fluid,
// interface and solid bits from two 16-byte loads. Second pass, a thread per
// 32-cell word:
// the fluid words of the 3x3 rows around it, each widened by the halo bits of
// its x-neighbour words, are ORed, then ORed along x.
// four type bytes (gas 0, liquid 1, interface 2, solid 3 in the low two
// bits) to three 4-bit masks: fluid (1 or 2), interface, solid; the multiply
// gathers the bits at positions 0, 8, 16, 24 into bits 21..24
__device__ __forceinline__ void type_nibbles(unsigned v, unsigned& f, unsigned& i, unsigned& sl) {
    const unsigned a = v & 0x03030303u;
    const unsigned hi = a >> 1;
    auto pack = [](unsigned x) { return ((x * 0x00204081u) >> 21) & 0xFu; };
    f = pack((a ^ hi) & 0x01010101u);
    i = pack(hi & ~a & 0x01010101u);
    sl = pack(hi & a & 0x01010101u);
}

__global__ void k_type_bits(Dev s) {
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= (s.n >> 5)) return;
    const uint4* src = reinterpret_cast<const uint4*>(s.flags + (w << 5));
    const uint4 a = src[0], b = src[1];
    const unsigned words[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    unsigned fm = 0, im = 0, sm = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        unsigned f, i, sl;
        type_nibbles(words[k], f, i, sl);
        fm |= f << (4 * k);
        im |= i << (4 * k);
        sm |= sl << (4 * k);
    }
    s.fbits[w] = fm;
    s.ibits[w] = im;
    s.sbits[w] = sm;
}

__global__ void k_classify_bits(Dev s) {
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nxw = s.nx >> 5;                      // words per row
    const long long nw = s.n >> 5;
    unsigned ifc_mask = 0, sol_mask = 0;
    if (w < nw) {
        const int xw = (int)(w % nxw);
        const long long row = w / nxw;
        const int y = (int)(row % s.ny), z = (int)(row / s.ny);
        // x-neighbour words (periodic wrap, or none beyond a wall face)
        const int xl = xw > 0 ? xw - 1 : (s.per_x ? nxw - 1 : -1);
        const int xr = xw < nxw - 1 ? xw + 1 : (s.per_x ? 0 : -1);
        unsigned long long orr = 0;   // bit 1 + k <-> x0 + k, bit 0 <-> x0 - 1, bit 33 <-> x0 + 32
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            const int zz = shift(z, dz, s.nz, s.per_z);
            if (zz < 0) continue;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const int yy = shift(y, dy, s.ny, s.per_y);
                if (yy < 0) continue;
                const long long rbase = ((long long)zz * s.ny + yy) * nxw;
                const unsigned cw = s.fbits[rbase + xw];
                const unsigned lw = xl >= 0 ? s.fbits[rbase + xl] : 0u;
                const unsigned rw = xr >= 0 ? s.fbits[rbase + xr] : 0u;
                orr |= ((unsigned long long)cw << 1) | (unsigned long long)(lw >> 31) |
                       ((unsigned long long)(rw & 1u) << 33);
            }
        }
        const unsigned long long nb = orr | (orr >> 1) | (orr << 1);   // bit 1 + k: fluid in the 3x3x3 block
        sol_mask = s.sbits[w] & (unsigned)(nb >> 1);
        ifc_mask = s.ibits[w];
    }
    const int c0 = (int)(w << 5);
    block_append_masks(s, c0, ifc_mask, s.wl, s.wl_count, s.wl_cap, sol_mask, s.sl, s.sl_count, s.sl_cap);
}

// Bed segments, for particle links taken from the fluid side: a thread per
// BED_SEG-cell x-segment of a row flags it when one of its liquid cells has a
// solid cell among its 26 neighbours (the solid words of the 3x3 rows around
// it, dilated by one cell along x, ANDed with its liquid words) and lists it.
// Rows at or above zmax_cell hold no such cell (no particle reaches them).
__global__ void k_bed_segments(Dev s) {
    constexpr int WPS = BED_SEG / 32;                // words per segment
    const long long sg = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nxw = s.nx >> 5;
    const long long nseg = (long long)s.nsegx * s.ny * s.nz;
    bool bed = false;
    if (sg < nseg) {
        const long long row = sg / s.nsegx;
        const int xs = (int)(sg - row * s.nsegx);
        const int y = (int)(row % s.ny), z = (int)(row / s.ny);
        const int w0 = xs * WPS;
        const int nw = min(WPS, nxw - w0);
        unsigned liq[WPS];
        unsigned any = 0;
#pragma unroll
        for (int k = 0; k < WPS; ++k) {
            liq[k] = k < nw ? s.fbits[row * nxw + w0 + k] & ~s.ibits[row * nxw + w0 + k] : 0u;
            any |= liq[k];
        }
        if (any && (s.per_z || z < *s.zmax_cell)) {
            unsigned dil[WPS];
#pragma unroll
            for (int k = 0; k < WPS; ++k) dil[k] = 0u;
            for (int dz = -1; dz <= 1; ++dz) {
                const int zz = shift(z, dz, s.nz, s.per_z);
                if (zz < 0) continue;
                for (int dy = -1; dy <= 1; ++dy) {
                    const int yy = shift(y, dy, s.ny, s.per_y);
                    if (yy < 0) continue;
                    const long long rb = ((long long)zz * s.ny + yy) * nxw;
                    // word w0 + k for k in [-1, nw]: the x-halo wraps on a
                    // periodic x axis and is empty beyond a wall face
                    unsigned wv[WPS + 2];
#pragma unroll
                    for (int k = -1; k <= WPS; ++k) {
                        int xw = w0 + k;
                        if (k > nw) { wv[k + 1] = 0u; continue; }
                        if (xw < 0) xw = s.per_x ? nxw - 1 : -1;
                        else if (xw >= nxw) xw = s.per_x ? 0 : -1;
                        wv[k + 1] = xw >= 0 ? s.sbits[rb + xw] : 0u;
                    }
#pragma unroll
                    for (int k = 0; k < WPS; ++k)
                        dil[k] |= wv[k + 1] | (wv[k + 1] << 1) | (wv[k + 1] >> 1) | (wv[k] >> 31) | (wv[k + 2] << 31);
                }
            }
#pragma unroll
            for (int k = 0; k < WPS; ++k) bed |= (liq[k] & dil[k]) != 0u;
        }
        s.segflag[sg] = bed ? 1 : 0;
    }
    block_append(s, bed, (int)sg, s.bseg, s.bseg_count, (int)nseg);
}

// Fallback for lattices whose x extent is not a multiple of 32: one thread
// per cell, 26 neighbour reads for solid cells.
__global__ void k_classify(Dev s) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = c < s.n;
    int t = 0;
    bool surf = false;
    if (in) {
        t = s.flags[c] & TYPE_MASK;
        if (t == T_SOL) {
            int x, y, z;
            coords(s, c, x, y, z);
            const int xs[3] = {shift(x, -1, s.nx, s.per_x), x, shift(x, 1, s.nx, s.per_x)};
            const int ys[3] = {shift(y, -1, s.ny, s.per_y), y, shift(y, 1, s.ny, s.per_y)};
            const int zs[3] = {shift(z, -1, s.nz, s.per_z), z, shift(z, 1, s.nz, s.per_z)};
            unsigned any = 0;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                if (q == 13) continue;
                const int a = xs[1 + cx(q)], b = ys[1 + cy(q)], d = zs[1 + cz(q)];
                if (a < 0 || b < 0 || d < 0) continue;
                const int tn = s.flags[a + (long long)s.nx * (b + (long long)s.ny * d)] & TYPE_MASK;
                any |= (tn == T_LIQ || tn == T_IFC) ? 1u : 0u;
            }
            surf = any != 0;
        }
    }
    block_append(s, in && t == T_IFC, (int)c, s.wl, s.wl_count, s.wl_cap);
    block_append(s, surf, (int)c, s.sl, s.sl_count, s.sl_cap);
}

// liquid cells with a gas neighbour (the separation the conversion rules keep)
__global__ void k_check_invariant(Dev s) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.n || (s.flags[c] & TYPE_MASK) != T_LIQ) return;
    int x, y, z;
    coords(s, c, x, y, z);
    for (int q = 0; q < 27; ++q) {
        if (q == 13) continue;
        const long long nb = nbr(s, x, y, z, cx(q), cy(q), cz(q));
        if (nb >= 0 && (s.flags[nb] & TYPE_MASK) == T_GAS) {
            atomicAdd(s.viol, 1ull);
            return;
        }
    }
}

void launch_check_invariant(const Dev& s, cudaStream_t st) {
    k_check_invariant<<<blocks_for(s.n, 256), 256, 0, st>>>(s);
}

__global__ void k_clamp_count(Dev s) {
    if (*s.wl_count > s.wl_cap) *s.wl_count = s.wl_cap;
    if (*s.sl_count > s.sl_cap) *s.sl_count = s.sl_cap;
}

int launch_classify(const Dev& s, cudaStream_t st) {
    cudaMemsetAsync(s.wl_count, 0, sizeof(int), st);
    cudaMemsetAsync(s.sl_count, 0, sizeof(int), st);
    int k = 2;
    if (s.nx % 32 == 0) {
        k_type_bits<<<blocks_for(s.n / 32, 256), 256, 0, st>>>(s);
        k_classify_bits<<<blocks_for(s.n / 32, 128), 128, 0, st>>>(s);
        ++k;
        if (s.links_fused) {
            cudaMemsetAsync(s.bseg_count, 0, sizeof(int), st);
            k_bed_segments<<<blocks_for((long long)s.nsegx * s.ny * s.nz, 128), 128, 0, st>>>(s);
            ++k;
        }
    } else {
        k_classify<<<blocks_for(s.n, 256), 256, 0, st>>>(s);
    }
    k_clamp_count<<<1, 1, 0, st>>>(s);
    return k;
}

__global__ void k_cell_counts(Dev s, unsigned long long* out) {
    __shared__ unsigned long long sh[4];
    if (threadIdx.x < 4) sh[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long loc[4] = {0, 0, 0, 0};
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < s.n;
         c += (long long)gridDim.x * blockDim.x)
        loc[s.flags[c] & TYPE_MASK]++;
    for (int k = 0; k < 4; ++k) atomicAdd(&sh[k], loc[k]);
    __syncthreads();
    if (threadIdx.x < 4) atomicAdd(&out[threadIdx.x], sh[threadIdx.x]);
}

void launch_cell_counts(const Dev& s, unsigned long long* out, cudaStream_t st) {
    cudaMemsetAsync(out, 0, 4 * sizeof(unsigned long long), st);
    k_cell_counts<<<152 * 4, 256, 0, st>>>(s, out);
}

// ------------------------------------------------------------ mass pool
__global__ void k_pool_prepare(Dev s) {
    int cnt = *s.wl_count;
    double p = *s.pool;
    if (cnt > 0 && p != 0.0) {
        *s.pool_share = p / (double)cnt;
        *s.pool = 0.0;
    } else {
        *s.pool_share = 0.0;
    }
}
__global__ void k_pool_spread(Dev s) {
    const double share = *s.pool_share;
    if (share == 0.0) return;
    FOR_LIST(i, s.wl_count) {
        int c = s.wl[i];
        float m = (float)((double)s.mass[c] + share);
        s.mass[c] = m;
        s.phi[c] = m / s.ru[c].x;
    }
}

int launch_pool_spread(const Dev& s, cudaStream_t st) {
    k_pool_prepare<<<1, 1, 0, st>>>(s);
    k_pool_spread<<<LIST_BLOCKS, LIST_THREADS, 0, st>>>(s);
    return 2;
}

// ------------------------------------------------------------ initial state
__device__ __forceinline__ float clamp01(double v) { return (float)(v < 0 ? 0 : (v > 1 ? 1 : v)); }

__device__ void init_cell(const Dev& s, long long c, int t, double H, double fill) {
    int x, y, z;
    coords(s, c, x, y, z);
    s.flags[c] = (uint8_t)t;
    s.owner[c] = -1;
    s.conv[c] = 0;
    s.mass[c] = 0.f;
    s.phi[c] = 0.f;
    s.ru[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    s.nrm[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t == T_GAS) return;
    double rho = (double)s.rho_gas * exp(3.0 * fabs((double)s.gzd) * (H - (z + 0.5)));
    float f[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) f[q] = (float)(wqd(q) * (rho - 1.0));
    store_fstar(s, c, 1, f);
    if (t == T_IFC)
        for (int q = 0; q < 27; ++q) st_any(s, s.fs, (long long)q * s.n + c, f[q]);
    s.ru[c] = make_float4((float)rho, 0.f, 0.f, 0.f);
    double m = rho * fill;
    s.mass[c] = (float)m;
    s.phi[c] = (float)(m / rho);
}

// flat surface at height H: fill(k) = clamp(H - k, 0, 1); interface where
// 0 < fill < 1 or where a full cell has gas directly above
__global__ void k_init_flat(Dev s, double H) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.n) return;
    int x, y, z;
    coords(s, c, x, y, z);
    double fk = H - z;
    fk = fk < 0 ? 0 : (fk > 1 ? 1 : fk);
    int t;
    if (fk == 0.0) t = T_GAS;
    else {
        bool above_gas;
        if (z + 1 < s.nz) {
            double fa = H - (z + 1);
            above_gas = fa <= 0.0;
        } else {
            above_gas = s.per_z ? (H <= 0.0) : false;
        }
        t = (fk < 1.0 || above_gas) ? T_IFC : T_LIQ;
    }
    init_cell(s, c, t, H, fk);
}

// surface height per column: gas where the fill is 0, liquid where it is 1
// and no 26-neighbour is gas, interface otherwise; solid cells are kept
__global__ void k_init_surface(Dev s, const double* Hxy) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.n) return;
    if ((s.flags[c] & TYPE_MASK) == T_SOL) return;
    int x, y, z;
    coords(s, c, x, y, z);
    const double H = Hxy[(long long)y * s.nx + x];
    double fk = H - z;
    fk = fk < 0 ? 0 : (fk > 1 ? 1 : fk);
    int t;
    if (fk == 0.0) t = T_GAS;
    else {
        bool gas_nb = false;
        for (int q = 0; q < 27; ++q) {
            if (q == 13) continue;
            long long nb = nbr(s, x, y, z, cx(q), cy(q), cz(q));
            if (nb < 0 || (s.flags[nb] & TYPE_MASK) == T_SOL) continue;
            int bx, by, bz;
            coords(s, nb, bx, by, bz);
            if (Hxy[(long long)by * s.nx + bx] - bz <= 0.0) gas_nb = true;
        }
        t = (fk < 1.0 || gas_nb) ? T_IFC : T_LIQ;
    }
    init_cell(s, c, t, H, fk);
}

// The flat start's values depend on z alone: the hydrostatic density of each
// z and its 27 stored deviations, by the expressions of init_cell, once per z.
__global__ void k_init_flat_table(Dev s, double H, double* rho_z, float* f_z) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= s.nz) return;
    const double rho = (double)s.rho_gas * exp(3.0 * fabs((double)s.gzd) * (H - (z + 0.5)));
    rho_z[z] = rho;
#pragma unroll
    for (int q = 0; q < 27; ++q) f_z[27 * z + q] = (float)(wqd(q) * (rho - 1.0));
}

// k_init_flat from the per-z table, with 32-bit cell coordinates (n < 2^31):
// the same cell types and values without an FP64 exponential and 64-bit
// divisions per cell
__global__ void k_init_flat_tab(Dev s, double H, const double* rho_z, const float* f_z) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.n) return;
    int x, y, z;
    coords32(s, (int)c, x, y, z);
    double fk = H - z;
    fk = fk < 0 ? 0 : (fk > 1 ? 1 : fk);
    int t;
    if (fk == 0.0) t = T_GAS;
    else {
        bool above_gas;
        if (z + 1 < s.nz) {
            double fa = H - (z + 1);
            above_gas = fa <= 0.0;
        } else {
            above_gas = s.per_z ? (H <= 0.0) : false;
        }
        t = (fk < 1.0 || above_gas) ? T_IFC : T_LIQ;
    }
    s.flags[c] = (uint8_t)t;
    s.owner[c] = -1;
    s.conv[c] = 0;
    s.mass[c] = 0.f;
    s.phi[c] = 0.f;
    s.ru[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    s.nrm[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t == T_GAS) return;
    const double rho = rho_z[z];
    float f[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) f[q] = f_z[27 * z + q];
#pragma unroll
    for (int q = 0; q < 27; ++q) st_any(s, s.f, fstar_slot(s, q, x, y, z, c, 1), f[q]);
    if (t == T_IFC)
        for (int q = 0; q < 27; ++q) st_any(s, s.fs, (long long)q * s.n + c, f[q]);
    s.ru[c] = make_float4((float)rho, 0.f, 0.f, 0.f);
    const double m = rho * fk;
    s.mass[c] = (float)m;
    s.phi[c] = (float)(m / rho);
}

void launch_init_flat(const Dev& s, double H, cudaStream_t st) {
    // the table lives for the two launches in the excess-mass normal field
    // (scratch between steps), which is zeroed again after them
    const size_t need = (size_t)s.nz * (sizeof(double) + 27 * sizeof(float));
    if (s.n < (1LL << 31) && need <= (size_t)s.n * sizeof(float4)) {
        double* rho_z = reinterpret_cast<double*>(s.nrm1);
        float* f_z = reinterpret_cast<float*>(rho_z + s.nz);
        k_init_flat_table<<<(s.nz + 127) / 128, 128, 0, st>>>(s, H, rho_z, f_z);
        k_init_flat_tab<<<blocks_for(s.n, 256), 256, 0, st>>>(s, H, rho_z, f_z);
        cudaMemsetAsync(s.nrm1, 0, need, st);
    } else {
        k_init_flat<<<blocks_for(s.n, 256), 256, 0, st>>>(s, H);
    }
}
void launch_init_surface(const Dev& s, const double* H, cudaStream_t st) {
    k_init_surface<<<blocks_for(s.n, 256), 256, 0, st>>>(s, H);
}

}  // namespace fsl
