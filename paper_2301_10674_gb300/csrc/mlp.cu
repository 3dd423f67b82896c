// Learned interface normal: training data, training and inference of the
// 27-64-64-4 perceptron (layout and fragment conventions in mlp_dev.cuh).
//
// Training data: analytic surfaces (planes, liquid and gas spheres, sine
// waves) through a point P near the centre of a 3x3x3 block; the fill level
// of each cell is its liquid volume fraction, the labels are the unit normal
// toward the gas and the mean curvature at P. Training: Adam on the loss
// 1 - cos(n, n_true) + lam (k - k_true)^2 + mu (|n| - 1)^2, averaged over a
// batch drawn by SplitMix64 from a seed, each stencil mapped by one of the 48
// cube symmetries. Every product runs on the tensor cores with BF16 operands
// and FP32 accumulation; master weights and Adam moments are FP32.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "fslbm.h"
#include "fslbm_dev.cuh"
#include "mlp_dev.cuh"

namespace fsl {

// ------------------------------------------------------------ surfaces
constexpr int GEN_THREADS = 256;
constexpr int SUBS = 64;                 // sub-samples per cell edge
constexpr int ROWS = SUBS * SUBS;        // sample rows along x per cell

// Volume of {xi in [0,1]^3 : m.xi <= alpha}, m >= 0, as the divided
// difference of G3(b) = max(b, 0)^3 / 6 over the three steps m_i. A step
// below 1e-3 is replaced by the derivative at the midpoint (G_k' = G_{k-1}),
// whose error is below m_i^2 / 24 times a bounded third derivative.
__device__ double box_volume_below(const double (&m)[3], double alpha) {
    double e[3];
    int ne = 0;
    double b0 = alpha;
    for (int i = 0; i < 3; ++i) {
        if (m[i] >= 1e-3) e[ne++] = m[i];
        else b0 -= 0.5 * m[i];
    }
    double sum = 0.0;
    for (int v = 0; v < (1 << ne); ++v) {
        double b = b0;
        int sgn = 1;
        for (int i = 0; i < ne; ++i)
            if (v >> i & 1) { b -= e[i]; sgn = -sgn; }
        double gk;
        if (b <= 0.0) gk = 0.0;
        else if (ne == 0) gk = 1.0;
        else if (ne == 1) gk = b;
        else if (ne == 2) gk = 0.5 * b * b;
        else gk = b * b * b / 6.0;
        sum += sgn * gk;
    }
    double den = 1.0;
    for (int i = 0; i < ne; ++i) den *= e[i];
    const double V = sum / den;
    return V < 0.0 ? 0.0 : (V > 1.0 ? 1.0 : V);
}

// liquid fraction of cell q below the plane (x - P).n <= 0: with
// x = c - 1/2 + xi and the negative components reflected (xi_i -> 1 - xi_i)
__device__ double plane_cell(const double (&n)[3], const double (&P)[3], int q) {
    const double c[3] = {(double)cx(q), (double)cy(q), (double)cz(q)};
    double beta = 0.0, shift = 0.0;
    double m[3];
    for (int i = 0; i < 3; ++i) {
        beta += n[i] * (P[i] - (c[i] - 0.5));
        if (n[i] < 0.0) shift += n[i];
        m[i] = fabs(n[i]);
    }
    return box_volume_below(m, beta - shift);
}

// sum over the block, the same order on every call
__device__ float block_sum(float v, float* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    float s = 0.f;
    for (int i = 0; i < GEN_THREADS / 32; ++i) s += sh[i];
    return s;
}

// One block per surface. params: n x 12 FP64 rows (kind, n0, s, r, A, k,
// phase, e1; P = s n0); fill: n x 27 FP32; target: n x 4 FP32.
__global__ void __launch_bounds__(GEN_THREADS) k_make_stencils(const double* __restrict__ params, long long n,
                                                               float* fill, float* target) {
    __shared__ float sh[GEN_THREADS / 32];
    const long long i = blockIdx.x;
    if (i >= n) return;
    const double* p = params + i * 12;
    const int kind = (int)p[0];
    const double n0[3] = {p[1], p[2], p[3]};
    const double s = p[4], r = p[5], A = p[6], kw = p[7], ph = p[8];
    const double e1[3] = {p[9], p[10], p[11]};
    const double P[3] = {s * n0[0], s * n0[1], s * n0[2]};
    const int tid = threadIdx.x;
    if (kind == 0) {
        if (tid < 27) fill[i * 27 + tid] = (float)plane_cell(n0, P, tid);
    } else if (kind == 1 || kind == 2) {
        // exact chord along x of each of the 64 x 64 rows
        const double sg = kind == 1 ? -1.0 : 1.0;       // centre P -/+ r n0
        const double C[3] = {P[0] + sg * r * n0[0], P[1] + sg * r * n0[1], P[2] + sg * r * n0[2]};
        const float rr = (float)(r * r);
        for (int q = 0; q < 27; ++q) {
            const float ox = (float)(C[0] - cx(q)), oy = (float)(C[1] - cy(q)), oz = (float)(C[2] - cz(q));
            float acc = 0.f;
            for (int j = tid; j < ROWS; j += GEN_THREADS) {
                const float y = ((j % SUBS) + 0.5f) / SUBS - 0.5f, z = ((j / SUBS) + 0.5f) / SUBS - 0.5f;
                const float dy = y - oy, dz = z - oz;
                const float h2 = rr - dy * dy - dz * dz;
                if (h2 > 0.f) {
                    const float h = sqrtf(h2);
                    acc += fmaxf(fminf(ox + h, 0.5f) - fmaxf(ox - h, -0.5f), 0.f);
                }
            }
            const float tot = block_sum(acc, sh) / ROWS;
            if (tid == 0) fill[i * 27 + q] = kind == 1 ? tot : 1.f - tot;
        }
    } else {
        // w <= A (sin(k u + phase) - sin(phase)) at 64^3 midpoints, u = d.e1,
        // w = d.n0, d = x - P. Per cell the corner offset is formed in FP64,
        // the sub-cell offsets in FP32; along a row the phase advances by
        // k e1.x / 64 per sample (a rotation), restarted from sincosf every
        // 16 samples.
        float sd, cd;
        sincosf((float)(kw * e1[0] / SUBS), &sd, &cd);
        const float Af = (float)A, As = (float)(A * sin(ph)), kf = (float)kw, pf = (float)ph;
        const float fe[3] = {(float)e1[0], (float)e1[1], (float)e1[2]};
        const float fn[3] = {(float)n0[0], (float)n0[1], (float)n0[2]};
        for (int q = 0; q < 27; ++q) {
            const double b[3] = {cx(q) - 0.5 - P[0], cy(q) - 0.5 - P[1], cz(q) - 0.5 - P[2]};
            const float bu = (float)(b[0] * e1[0] + b[1] * e1[1] + b[2] * e1[2]);
            const float bw = (float)(b[0] * n0[0] + b[1] * n0[1] + b[2] * n0[2]);
            int cnt = 0;
            for (int j = tid; j < ROWS; j += GEN_THREADS) {
                const float yo = ((j % SUBS) + 0.5f) / SUBS, zo = ((j / SUBS) + 0.5f) / SUBS;
                const float x0 = 0.5f / SUBS;
                const float u0 = bu + (x0 * fe[0] + yo * fe[1] + zo * fe[2]);
                const float w0 = bw + (x0 * fn[0] + yo * fn[1] + zo * fn[2]);
                for (int seg = 0; seg < SUBS; seg += 16) {
                    float sn, cs;
                    sincosf(kf * (u0 + seg * (fe[0] / SUBS)) + pf, &sn, &cs);
                    float w = w0 + seg * (fn[0] / SUBS);
                    for (int k = 0; k < 16; ++k) {
                        cnt += w <= Af * sn - As ? 1 : 0;
                        const float sn2 = sn * cd + cs * sd;
                        cs = cs * cd - sn * sd;
                        sn = sn2;
                        w += fn[0] / SUBS;
                    }
                }
            }
            const float tot = block_sum((float)cnt, sh);      // integer counts: exact in FP32
            if (tid == 0) fill[i * 27 + q] = tot / (float)(ROWS * SUBS);
        }
    }
    if (tid == 0) {
        double nt[3] = {n0[0], n0[1], n0[2]}, kap = 0.0;
        if (kind == 1) kap = 1.0 / r;
        else if (kind == 2) kap = -1.0 / r;
        else if (kind == 3) {
            // graph w = f(u): normal (n0 - f' e1) / sqrt(1 + f'^2), mean
            // curvature of the cylinder -f'' / (2 (1 + f'^2)^(3/2))
            const double fp = A * kw * cos(ph), fpp = -A * kw * kw * sin(ph);
            const double qn = sqrt(1.0 + fp * fp);
            for (int k = 0; k < 3; ++k) nt[k] = (n0[k] - fp * e1[k]) / qn;
            kap = -fpp / (2.0 * qn * qn * qn);
        }
        for (int k = 0; k < 3; ++k) target[i * 4 + k] = (float)nt[k];
        target[i * 4 + 3] = (float)kap;
    }
}

// ------------------------------------------------------------ sampling
// output `counter` (from 0) of SplitMix64 seeded with `seed`
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t counter) {
    uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// cube symmetry k: (T v)_i = s_i v_perm(i), perm the (k / 8)-th permutation
// of (0, 1, 2) in lexicographic order, s_i = -1 where bit i of k % 8 is set
__device__ __forceinline__ int sym_perm(int k, int i) {
    constexpr int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    return P[k >> 3][i];
}
__device__ __forceinline__ int sym_sign(int k, int i) { return ((k & 7) >> i & 1) ? -1 : 1; }

// the cell whose fill lands in cell qd under symmetry k: c = T^-1 c', i.e.
// c[perm(i)] = s_i c'[i]
__device__ __forceinline__ int sym_source(int k, int qd) {
    const int cdst[3] = {qd % 3 - 1, (qd / 3) % 3 - 1, qd / 9 - 1};
    int c[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < 3; ++i) c[sym_perm(k, i)] = sym_sign(k, i) * cdst[i];
    return (c[0] + 1) + 3 * (c[1] + 1) + 9 * (c[2] + 1);
}

// ------------------------------------------------------------ training
constexpr int TR_WARPS = 8;
constexpr int TR_ROWS = 16 * TR_WARPS;   // samples per block
constexpr int LDS = TR_ROWS + 8;         // padded row: rows g = 0..7 fall in distinct banks
constexpr int PSTRIDE = 6216;            // floats per block in the partial buffer
constexpr int LOSS_SLOT = MLP_NPARAM;

struct TrainSmem {
    __nv_bfloat16 XT[32][LDS];           // inputs, transposed (column, sample)
    __nv_bfloat16 H1T[MLP_H][LDS];       // relu(z1)
    __nv_bfloat16 H2T[MLP_H][LDS];       // relu(z2)
    __nv_bfloat16 D1T[MLP_H][LDS];       // dL/dz1
    __nv_bfloat16 D2T[MLP_H][LDS];       // dL/dz2
    __nv_bfloat16 DYT[16][LDS];          // dL/dy (outputs 4..15 zero)
    float bsum[TR_WARPS][132];           // per-warp column sums of dz1, dz2, dy
    float lsum[TR_WARPS];
};

enum : int { TR_FIXED = 0, TR_DRAW_SYM = 1, TR_DRAW = 2 };

struct TrainArgs {
    const MlpBf16* W;
    const float* fill;
    const float* target;
    long long n;            // stencils in the set
    int B;                  // samples in the batch
    int mode;               // TR_FIXED: sample j is stencil j; TR_DRAW(_SYM): drawn (and mapped)
    uint64_t seed;
    long long step;
    float lam, mu;
    float* part;            // [blocks][PSTRIDE]
};

__device__ __forceinline__ float sum_over_groups(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

// One block per 128 samples: per-warp forward and backward of 16 samples,
// then the block's share of the weight gradients dW = dZ^T H as 56
// tensor-core tiles over K = 128 samples, written with the bias and loss
// sums to the block's row of the partial buffer.
__global__ void __launch_bounds__(256) k_mlp_train_block(TrainArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const MlpBf16& W = *a.W;
    const float invB = 1.f / (float)a.B;

    // -------- per-warp forward and backward
    long long src[2];
    int sym[2];
    bool valid[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const long long j = (long long)blockIdx.x * TR_ROWS + warp * 16 + g + 8 * r;
        valid[r] = j < a.B;
        src[r] = 0;
        sym[r] = 0;
        if (valid[r]) {
            if (a.mode == TR_FIXED) {
                src[r] = j;
            } else {
                const uint64_t v = splitmix64(a.seed, (uint64_t)a.step * (uint64_t)a.B + (uint64_t)j);
                src[r] = (long long)(v % (uint64_t)a.n);
                sym[r] = a.mode == TR_DRAW_SYM ? (int)((v >> 32) % 48ull) : 0;
            }
        }
    }
    float xv[2][8];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = frag_col(j >> 2, j & 3, t);
            xv[r][j] = (valid[r] && col < 27) ? a.fill[src[r] * 27 + sym_source(sym[r], col)] : 0.f;
        }
    uint32_t xf[2][4];
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        xf[kk][0] = pack_bf16(xv[0][4 * kk + 0], xv[0][4 * kk + 1]);
        xf[kk][1] = pack_bf16(xv[1][4 * kk + 0], xv[1][4 * kk + 1]);
        xf[kk][2] = pack_bf16(xv[0][4 * kk + 2], xv[0][4 * kk + 3]);
        xf[kk][3] = pack_bf16(xv[1][4 * kk + 2], xv[1][4 * kk + 3]);
    }
    MlpAct act;
    mlp_forward(W, xf, act);
    float y[2][4];
    mlp_outputs(act, y[0], y[1]);

    // loss (already divided by the batch size) and dL/dy of both rows,
    // identical in the four lanes of a group
    float dy[2][4], L[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        float tg[4] = {0.f, 0.f, 0.f, 0.f};
        if (valid[r]) {
            const float* tp = a.target + src[r] * 4;
            const int k = sym[r];
#pragma unroll
            for (int i = 0; i < 3; ++i) tg[i] = sym_sign(k, i) * tp[sym_perm(k, i)];
            tg[3] = tp[3];
        }
        const float n2 = y[r][0] * y[r][0] + y[r][1] * y[r][1] + y[r][2] * y[r][2];
        const float nrm = sqrtf(fmaxf(n2, 1e-30f));
        const float dot = y[r][0] * tg[0] + y[r][1] * tg[1] + y[r][2] * tg[2];
        const float dk = y[r][3] - tg[3];
        const float pen = 2.f * a.mu * (nrm - 1.f) / nrm;
#pragma unroll
        for (int i = 0; i < 3; ++i)
            dy[r][i] = valid[r] ? (-(tg[i] / nrm - dot / (nrm * nrm * nrm) * y[r][i]) + pen * y[r][i]) * invB : 0.f;
        dy[r][3] = valid[r] ? 2.f * a.lam * dk * invB : 0.f;
        L[r] = valid[r] ? (1.f - dot / nrm + a.lam * dk * dk + a.mu * (nrm - 1.f) * (nrm - 1.f)) * invB : 0.f;
    }

    // dZ2 = (dY W3) masked by z2 > 0, dY as A operand (k = output)
    const uint32_t ay0 = t == 0 ? pack_bf16(dy[0][0], dy[0][1]) : (t == 1 ? pack_bf16(dy[0][2], dy[0][3]) : 0u);
    const uint32_t ay1 = t == 0 ? pack_bf16(dy[1][0], dy[1][1]) : (t == 1 ? pack_bf16(dy[1][2], dy[1][3]) : 0u);
    float dz2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        const __nv_bfloat16* col = W.w3t + (8 * nt + g) * 16 + 2 * t;
        mma_bf16(d, ay0, ay1, 0u, 0u, ld_pair(col), ld_pair(col + 8));
#pragma unroll
        for (int k = 0; k < 4; ++k) dz2[nt][k] = act.z2[nt][k] > 0.f ? d[k] : 0.f;
    }
    // dZ1 = (dZ2 W2) masked by z1 > 0
    float dz1[8][4];
    {
        uint32_t af[4][4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const float* p = dz2[2 * kk];
            const float* q = dz2[2 * kk + 1];
            af[kk][0] = pack_bf16(p[0], p[1]);
            af[kk][1] = pack_bf16(p[2], p[3]);
            af[kk][2] = pack_bf16(q[0], q[1]);
            af[kk][3] = pack_bf16(q[2], q[3]);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const __nv_bfloat16* col = W.w2t + (8 * nt + g) * MLP_H + 16 * kk + 2 * t;
                mma_bf16(d, af[kk][0], af[kk][1], af[kk][2], af[kk][3], ld_pair(col), ld_pair(col + 8));
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) dz1[nt][k] = act.z1[nt][k] > 0.f ? d[k] : 0.f;
        }
    }

    // operands of the weight-gradient products, transposed into shared memory
    const int rl = warp * 16 + g, rl8 = rl + 8;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int col = frag_col(j >> 2, j & 3, t);
        S.XT[col][rl] = __float2bfloat16_rn(xv[0][j]);
        S.XT[col][rl8] = __float2bfloat16_rn(xv[1][j]);
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int u = 8 * nt + 2 * t;
        S.H1T[u][rl] = __float2bfloat16_rn(fmaxf(act.z1[nt][0], 0.f));
        S.H1T[u + 1][rl] = __float2bfloat16_rn(fmaxf(act.z1[nt][1], 0.f));
        S.H1T[u][rl8] = __float2bfloat16_rn(fmaxf(act.z1[nt][2], 0.f));
        S.H1T[u + 1][rl8] = __float2bfloat16_rn(fmaxf(act.z1[nt][3], 0.f));
        S.H2T[u][rl] = __float2bfloat16_rn(fmaxf(act.z2[nt][0], 0.f));
        S.H2T[u + 1][rl] = __float2bfloat16_rn(fmaxf(act.z2[nt][1], 0.f));
        S.H2T[u][rl8] = __float2bfloat16_rn(fmaxf(act.z2[nt][2], 0.f));
        S.H2T[u + 1][rl8] = __float2bfloat16_rn(fmaxf(act.z2[nt][3], 0.f));
        S.D1T[u][rl] = __float2bfloat16_rn(dz1[nt][0]);
        S.D1T[u + 1][rl] = __float2bfloat16_rn(dz1[nt][1]);
        S.D1T[u][rl8] = __float2bfloat16_rn(dz1[nt][2]);
        S.D1T[u + 1][rl8] = __float2bfloat16_rn(dz1[nt][3]);
        S.D2T[u][rl] = __float2bfloat16_rn(dz2[nt][0]);
        S.D2T[u + 1][rl] = __float2bfloat16_rn(dz2[nt][1]);
        S.D2T[u][rl8] = __float2bfloat16_rn(dz2[nt][2]);
        S.D2T[u + 1][rl8] = __float2bfloat16_rn(dz2[nt][3]);
    }
    S.DYT[t][rl] = __float2bfloat16_rn(dy[0][t]);
    S.DYT[t][rl8] = __float2bfloat16_rn(dy[1][t]);
    for (int o = 4 + t; o < 16; o += 4) {
        S.DYT[o][rl] = __float2bfloat16_rn(0.f);
        S.DYT[o][rl8] = __float2bfloat16_rn(0.f);
    }
    // bias gradients and loss in FP32: sums over the warp's 16 samples
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float s10 = sum_over_groups(dz1[nt][0] + dz1[nt][2]);
        const float s11 = sum_over_groups(dz1[nt][1] + dz1[nt][3]);
        const float s20 = sum_over_groups(dz2[nt][0] + dz2[nt][2]);
        const float s21 = sum_over_groups(dz2[nt][1] + dz2[nt][3]);
        if (g == 0) {
            S.bsum[warp][8 * nt + 2 * t] = s10;
            S.bsum[warp][8 * nt + 2 * t + 1] = s11;
            S.bsum[warp][64 + 8 * nt + 2 * t] = s20;
            S.bsum[warp][64 + 8 * nt + 2 * t + 1] = s21;
        }
    }
    {
        const float sy = sum_over_groups(dy[0][t] + dy[1][t]);
        const float sl = sum_over_groups(L[0] + L[1]);
        if (g == 0) S.bsum[warp][128 + t] = sy;
        if (lane == 0) S.lsum[warp] = sl;
    }
    __syncthreads();

    // -------- the block's share of the weight gradients: 56 tiles of 16 x 8
    float* part = a.part + (long long)blockIdx.x * PSTRIDE;
    for (int tile = warp; tile < 56; tile += TR_WARPS) {
        const __nv_bfloat16 *Am, *Bm;
        int mt, nt, which;
        if (tile < 16) { which = 1; mt = tile >> 2; nt = tile & 3; Am = &S.D1T[0][0]; Bm = &S.XT[0][0]; }
        else if (tile < 48) { which = 2; mt = (tile - 16) >> 3; nt = (tile - 16) & 7; Am = &S.D2T[0][0]; Bm = &S.H1T[0][0]; }
        else { which = 3; mt = 0; nt = tile - 48; Am = &S.DYT[0][0]; Bm = &S.H2T[0][0]; }
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < TR_ROWS / 16; ++ks) {
            const __nv_bfloat16* ar = Am + (16 * mt + g) * LDS + 16 * ks + 2 * t;
            const __nv_bfloat16* br = Bm + (8 * nt + g) * LDS + 16 * ks + 2 * t;
            mma_bf16(d, ld_pair(ar), ld_pair(ar + 8 * LDS), ld_pair(ar + 8), ld_pair(ar + 8 * LDS + 8), ld_pair(br),
                     ld_pair(br + 8));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int row = 16 * mt + g + 8 * (k >> 1), col = 8 * nt + 2 * t + (k & 1);
            if (which == 1) { if (col < MLP_IN) part[OFF_W1 + row * MLP_IN + col] = d[k]; }
            else if (which == 2) part[OFF_W2 + row * MLP_H + col] = d[k];
            else if (row < MLP_OUT) part[OFF_W3 + row * MLP_H + col] = d[k];
        }
    }
    const int j = threadIdx.x;
    if (j < 132) {
        float s = 0.f;
        for (int w = 0; w < TR_WARPS; ++w) s += S.bsum[w][j];
        const int off = j < 64 ? OFF_B1 + j : (j < 128 ? OFF_B2 + j - 64 : OFF_B3 + j - 128);
        part[off] = s;
    }
    if (j == 132) {
        float s = 0.f;
        for (int w = 0; w < TR_WARPS; ++w) s += S.lsum[w];
        part[LOSS_SLOT] = s;
    }
}

// writes the operand copies of parameter i
__device__ __forceinline__ void emit_bf16(MlpBf16* W, int i, float v) {
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    if (i < OFF_B1) {
        W->w1[(i / MLP_IN) * 32 + i % MLP_IN] = b;
    } else if (i < OFF_W2) {
        W->b1[i - OFF_B1] = v;
    } else if (i < OFF_B2) {
        const int r = (i - OFF_W2) / MLP_H, c = (i - OFF_W2) % MLP_H;
        W->w2[r * MLP_H + c] = b;
        W->w2t[c * MLP_H + r] = b;
    } else if (i < OFF_W3) {
        W->b2[i - OFF_B2] = v;
    } else if (i < OFF_B3) {
        const int r = (i - OFF_W3) / MLP_H, c = (i - OFF_W3) % MLP_H;
        W->w3[r * MLP_H + c] = b;
        W->w3t[c * 16 + r] = b;
    } else {
        W->b3[i - OFF_B3] = v;
    }
}

// zero padding (first launch), then the copies of every parameter (second)
__global__ void k_mlp_pad(MlpBf16* W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MLP_H * 32) W->w1[i] = __float2bfloat16_rn(0.f);
    if (i < 16 * MLP_H) {
        W->w3[i] = __float2bfloat16_rn(0.f);
        W->w3t[i] = __float2bfloat16_rn(0.f);
    }
    if (i < 16) W->b3[i] = 0.f;
}
__global__ void k_mlp_emit(const float* __restrict__ theta, MlpBf16* W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MLP_NPARAM) emit_bf16(W, i, theta[i]);
}

struct AdamArgs {
    float lr, b1, b2, eps, c1, c2;
};

// Sum of the blocks' partials in block order (deterministic). mode 0:
// gradient and loss out; mode 1: Adam update of theta and its operand
// copies, loss out.
__global__ void k_mlp_reduce(const float* __restrict__ part, int nblocks, int mode, float* grad, float* loss,
                             float* theta, float* m, float* v, MlpBf16* W, AdamArgs ad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > MLP_NPARAM) return;
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += part[(long long)b * PSTRIDE + i];
    if (i == LOSS_SLOT) {
        if (loss) *loss = s;
        return;
    }
    if (mode == 0) {
        grad[i] = s;
        return;
    }
    const float mi = ad.b1 * m[i] + (1.f - ad.b1) * s;
    const float vi = ad.b2 * v[i] + (1.f - ad.b2) * s * s;
    m[i] = mi;
    v[i] = vi;
    const float p = theta[i] - ad.lr * (mi / ad.c1) / (sqrtf(vi / ad.c2) + ad.eps);
    theta[i] = p;
    emit_bf16(W, i, p);
}

// Raw outputs (n, curvature) of n stencils, a warp per 16
__global__ void __launch_bounds__(128) k_mlp_infer(const MlpBf16* __restrict__ Wp, const float* __restrict__ fill,
                                                   long long n, float4* out) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 16; base < n;
         base += nwarps * 16) {
        const long long r0 = base + g, r1 = base + g + 8;
        auto val = [&](int r, int col) -> float {
            const long long row = r ? r1 : r0;
            return (row < n && col < 27) ? fill[row * 27 + col] : 0.f;
        };
        uint32_t xf[2][4];
        input_frags(val, xf);
        MlpAct act;
        mlp_forward(*Wp, xf, act);
        float y[2][4];
        mlp_outputs(act, y[0], y[1]);
        if (t < 2) {
            const long long row = t ? r1 : r0;
            if (row < n) out[row] = make_float4(y[t][0], y[t][1], y[t][2], y[t][3]);
        }
    }
}

// First-layer operands of the mirror images of R-17g, built on the host from
// BF16 bit patterns: block m - 1 (m = 1 mirrors x, 2 mirrors y, 3 both) is W1
// with input column q taken from the mirrored column, so that it applied to
// a stencil gives W1 applied to the mirrored stencil.
void mlp_mirror_w1_host(const uint16_t* w, __nv_bfloat16* out) {
    for (int m = 1; m < 4; ++m)
        for (int r = 0; r < MLP_H; ++r)
            for (int c = 0; c < 32; ++c) {
                __nv_bfloat16_raw v;
                v.x = 0;   // +0.0: the padding columns 27..31
                if (c < MLP_IN) {
                    int a = c % 3, b = (c / 3) % 3;
                    const int z = c / 9;
                    if (m & 1) a = 2 - a;
                    if (m & 2) b = 2 - b;
                    v.x = w[OFF_W1 + r * MLP_IN + a + 3 * b + 9 * z];
                }
                out[(m - 1) * MLP_H * 32 + r * 32 + c] = __nv_bfloat16(v);
            }
}

// The in-step weights in fragment order (MlpFrag), from the operand copies
// h and the mirrored first layers w1m: lane (g, t) of an mma over n-tile nt
// and k-tile kk takes row 8 nt + g (g for the output layer) and the column
// pairs 16 kk + 2t and 16 kk + 2t + 8, packed low element first.
void mlp_frag_host(const MlpBf16& h, const __nv_bfloat16* w1m, MlpFrag& G) {
    auto pair = [](const __nv_bfloat16* p) {
        __nv_bfloat16_raw lo = p[0], hi = p[1];
        return (uint32_t)lo.x | ((uint32_t)hi.x << 16);
    };
    for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, t = lane & 3;
        for (int m = 0; m < 4; ++m) {
            const __nv_bfloat16* w1 = m == 0 ? h.w1 : w1m + (m - 1) * MLP_H * 32;
            for (int nt = 0; nt < 8; ++nt)
                for (int kk = 0; kk < 2; ++kk) {
                    const __nv_bfloat16* r = w1 + (8 * nt + g) * 32 + 16 * kk + 2 * t;
                    G.w1[m][nt][kk][lane] = make_uint2(pair(r), pair(r + 8));
                }
        }
        for (int nt = 0; nt < 8; ++nt)
            for (int kk = 0; kk < 4; ++kk) {
                const __nv_bfloat16* r = h.w2 + (8 * nt + g) * MLP_H + 16 * kk + 2 * t;
                G.w2[nt][kk][lane] = make_uint2(pair(r), pair(r + 8));
            }
        for (int kk = 0; kk < 4; ++kk) {
            const __nv_bfloat16* r = h.w3 + g * MLP_H + 16 * kk + 2 * t;
            G.w3[kk][lane] = make_uint2(pair(r), pair(r + 8));
        }
    }
}

// operand copies built on the host from BF16 bit patterns
void mlp_from_bf16_host(const uint16_t* w, MlpBf16& h) {
    auto f = [](uint16_t b) {
        const uint32_t u = (uint32_t)b << 16;
        float x;
        memcpy(&x, &u, 4);
        return x;
    };
    auto bf = [](uint16_t b) {
        __nv_bfloat16_raw r;
        r.x = b;
        return __nv_bfloat16(r);
    };
    memset(&h, 0, sizeof(h));   // +0.0 in BF16 and FP32 is all-zero bits
    for (int r = 0; r < MLP_H; ++r)
        for (int c = 0; c < MLP_IN; ++c) h.w1[r * 32 + c] = bf(w[OFF_W1 + r * MLP_IN + c]);
    for (int r = 0; r < MLP_H; ++r)
        for (int c = 0; c < MLP_H; ++c) {
            h.w2[r * MLP_H + c] = bf(w[OFF_W2 + r * MLP_H + c]);
            h.w2t[c * MLP_H + r] = bf(w[OFF_W2 + r * MLP_H + c]);
        }
    for (int r = 0; r < MLP_OUT; ++r)
        for (int c = 0; c < MLP_H; ++c) {
            h.w3[r * MLP_H + c] = bf(w[OFF_W3 + r * MLP_H + c]);
            h.w3t[c * 16 + r] = bf(w[OFF_W3 + r * MLP_H + c]);
        }
    for (int i = 0; i < MLP_H; ++i) {
        h.b1[i] = f(w[OFF_B1 + i]);
        h.b2[i] = f(w[OFF_B2 + i]);
    }
    for (int i = 0; i < MLP_OUT; ++i) h.b3[i] = f(w[OFF_B3 + i]);
}

}  // namespace fsl

// ------------------------------------------------------------ C ABI
using namespace fsl;

namespace {

struct Scratch {
    std::vector<void*> ptrs;
    bool ok = true;
    template <class T>
    T* get(size_t count) {
        void* p = nullptr;
        if (!ok || cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
            ok = false;
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~Scratch() {
        for (void* p : ptrs) cudaFree(p);
    }
};

int finish(cudaStream_t st) {
    if (cudaGetLastError() != cudaSuccess) return FSLBM_EDEVICE;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FSLBM_EDEVICE;
    return FSLBM_OK;
}

void emit(const float* theta, MlpBf16* W, cudaStream_t st) {
    k_mlp_pad<<<(MLP_H * 32 + 255) / 256, 256, 0, st>>>(W);
    k_mlp_emit<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(theta, W);
}

bool train_smem_ready() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    static int done_mask = 0;
    if (dev < 31 && (done_mask >> dev & 1)) return true;
    if (cudaFuncSetAttribute(k_mlp_train_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(TrainSmem)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (dev < 31) done_mask |= 1 << dev;
    return true;
}

}  // namespace

extern "C" {

int fslbm_mlp_stencils(const double* params, int64_t n, float* fill, float* target, void* cuda_stream) {
    if (!params || !fill || !target || n <= 0 || n > ((int64_t)1 << 31) - 1) return FSLBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    k_make_stencils<<<(unsigned)n, GEN_THREADS, 0, st>>>(params, (long long)n, fill, target);
    return finish(st);
}

int fslbm_mlp_gradient(const float* theta, const float* fill, const float* target, int64_t n, double lam,
                       double mu, float* grad, float* loss, void* cuda_stream) {
    if (!theta || !fill || !target || !grad || !loss || n <= 0 || n > ((int64_t)1 << 24)) return FSLBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (!train_smem_ready()) return FSLBM_EDEVICE;
    const int blocks = (int)((n + TR_ROWS - 1) / TR_ROWS);
    Scratch sc;
    MlpBf16* W = sc.get<MlpBf16>(1);
    float* part = sc.get<float>((size_t)blocks * PSTRIDE);
    if (!sc.ok) return FSLBM_ENOMEM;
    emit(theta, W, st);
    TrainArgs a{W, fill, target, (long long)n, (int)n, TR_FIXED, 0, 0, (float)lam, (float)mu, part};
    k_mlp_train_block<<<blocks, 256, sizeof(TrainSmem), st>>>(a);
    k_mlp_reduce<<<(MLP_NPARAM + 256) / 256, 256, 0, st>>>(part, blocks, 0, grad, loss, nullptr, nullptr,
                                                           nullptr, nullptr, AdamArgs{});
    return finish(st);
}

int fslbm_mlp_train(float* theta, const float* fill, const float* target, int64_t n, int64_t steps, int batch,
                    double lr, double lr_end, double lam, double mu, uint64_t seed, int augment, float* loss_curve,
                    void* cuda_stream) {
    if (!theta || !fill || !target || n <= 0 || n > ((int64_t)1 << 31) - 1 || steps < 0 || batch <= 0 ||
        batch > (1 << 20) || !(lr >= 0.0) || !(lr_end >= 0.0))
        return FSLBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (!train_smem_ready()) return FSLBM_EDEVICE;
    const int blocks = (batch + TR_ROWS - 1) / TR_ROWS;
    Scratch sc;
    MlpBf16* W = sc.get<MlpBf16>(1);
    float* part = sc.get<float>((size_t)blocks * PSTRIDE);
    float* m = sc.get<float>(MLP_NPARAM);
    float* v = sc.get<float>(MLP_NPARAM);
    if (!sc.ok) return FSLBM_ENOMEM;
    cudaMemsetAsync(m, 0, MLP_NPARAM * sizeof(float), st);
    cudaMemsetAsync(v, 0, MLP_NPARAM * sizeof(float), st);
    emit(theta, W, st);
    const double b1 = 0.9, b2 = 0.999;
    double p1 = 1.0, p2 = 1.0;
    for (int64_t k = 0; k < steps; ++k) {
        TrainArgs a{W, fill, target, (long long)n, batch, augment ? TR_DRAW_SYM : TR_DRAW, seed, (long long)k,
                    (float)lam, (float)mu, part};
        k_mlp_train_block<<<blocks, 256, sizeof(TrainSmem), st>>>(a);
        p1 *= b1;
        p2 *= b2;
        // learning rate: geometric from lr to lr_end over the run (constant
        // when lr_end is 0 or equal to lr)
        const double frac = steps > 1 ? (double)k / (double)(steps - 1) : 0.0;
        const double lr_k = (lr_end > 0.0 && lr > 0.0) ? lr * std::pow(lr_end / lr, frac) : lr;
        const AdamArgs ad{(float)lr_k, (float)b1, (float)b2, 1e-8f, (float)(1.0 - p1), (float)(1.0 - p2)};
        k_mlp_reduce<<<(MLP_NPARAM + 256) / 256, 256, 0, st>>>(part, blocks, 1, nullptr,
                                                               loss_curve ? loss_curve + k : nullptr, theta, m,
                                                               v, W, ad);
        if ((k & 255) == 255 && cudaGetLastError() != cudaSuccess) return FSLBM_EDEVICE;
    }
    return finish(st);
}

int fslbm_mlp_infer(const float* theta, const float* fill, int64_t n, float* out, void* cuda_stream) {
    if (!theta || !fill || !out || n <= 0) return FSLBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    Scratch sc;
    MlpBf16* W = sc.get<MlpBf16>(1);
    if (!sc.ok) return FSLBM_ENOMEM;
    emit(theta, W, st);
    const long long blocks_needed = ((n + 15) / 16 * 32 + 127) / 128;
    const int blocks = (int)(blocks_needed < 152 * 16 ? blocks_needed : 152 * 16);
    k_mlp_infer<<<blocks, 128, 0, st>>>(W, fill, (long long)n, reinterpret_cast<float4*>(out));
    return finish(st);
}

}  // extern "C"
