// The cumulant collision of two cells at once (Section 2.1), on the packed
// FP32 instructions of sm_100 and later: every add, multiply and fused
// multiply-add acts on a float2 that holds the same quantity of both cells
// (one FADD2 / FMUL2 / FFMA2 for the pair). It computes what collide_scaled
// computes, term for term, except that the known zeros among the
// post-collision moments (the third-order moments with two equal indices,
// k111, and the fifth-order ones) are left out of the backward transform by
// hand; each cell's results are FP32 operations on that cell's values alone.
#pragma once
#include "fslbm_dev.cuh"

namespace fsl {

__device__ __forceinline__ float2 p_set(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b: the product b (-1) is exact, so the one rounding is the subtraction's
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, p_set(-1.f), a); }

// per-axis coefficients of the backward transform (as AxisCoef) for two cells
struct AxisCoef2 {
    float2 A, B, C, D;
};
__device__ __forceinline__ AxisCoef2 axis_coef2(float2 u) {
    const float2 h = p_mul(p_set(0.5f), u);
    const float2 hu = p_mul(h, u);
    return {p_sub(hu, h), p_add(u, p_set(-0.5f)), p_add(hu, h), p_add(u, p_set(0.5f))};
}
// one line (k0, k1, k2) -> (f_-1, f_0, f_+1) with rest value R of the zeroth
// moment; K0, K1, K2 false mark inputs that are known zeros (not read)
template <bool K0, bool K1, bool K2>
__device__ __forceinline__ void bwd_line2(float2& a, float2& b, float2& c, const AxisCoef2& w, float R) {
    const float2 k0 = a, k1 = b, k2 = c;
    const bool hasK = K0 || R != 0.f;
    float2 K = p_set(R);
    if (K0) K = R != 0.f ? p_add(p_set(R), k0) : k0;
    float2 lo, hi;
    if (K2) {
        const float2 h = p_mul(p_set(0.5f), k2);
        lo = K1 ? p_fma(w.B, k1, h) : h;
        hi = K1 ? p_fma(w.D, k1, h) : h;
        if (hasK) {
            lo = p_fma(w.A, K, lo);
            hi = p_fma(w.C, K, hi);
        }
    } else if (hasK) {
        lo = K1 ? p_fma(w.A, K, p_mul(w.B, k1)) : p_mul(w.A, K);
        hi = K1 ? p_fma(w.C, K, p_mul(w.D, k1)) : p_mul(w.C, K);
    } else {
        lo = p_mul(w.B, k1);
        hi = p_mul(w.D, k1);
    }
    a = lo;
    c = hi;
    b = K0 ? p_sub(p_sub(k0, lo), hi) : p_sub(p_mul(lo, p_set(-1.f)), hi);
}

// Reference of the 16-bit stored values (Section 2.1 hydrostatic start of the
// liquid): a stored value is (f - w_q (1 + r)) 2^SCALE_LOG2, r the reference
// deviation delta(z) of the z of the slot it sits in. rd[c_z + 1] is r of the
// slots the pair's directions with c_z = -1, 0, +1 were read from. The
// collision works on deviations from w: the read reference enters the
// moments (its zeroth, z and second diagonal moments; the D3Q27 weights
// factor into per-axis weights 1/6, 2/3, 1/6, so nothing else). The outputs
// come out relative to w; the caller takes the reference of the slot each
// one is written to off at its store (keeping the rest values of the
// backward transform compile-time constants keeps the registers free).
struct PairRef {
    float rd[3];
};

// f: the stored values (deviations times 2^SCALE_LOG2) of two cells, in place;
// with HREF the stored values are relative to the reference `ref` (16-bit
// storage), without it relative to w
template <int SCALE_LOG2, bool HREF>
__device__ __forceinline__ void collide_pair(float2 (&f)[27], float omega, float gx, float gy, float gz,
                                             const PairRef& ref) {
    constexpr float scale = (float)(1u << SCALE_LOG2);
    constexpr bool scaled = SCALE_LOG2 != 0;

    // forward, x: per (b, c) line the sum, first and second raw moments
    float2 X0[9], X1[9], X2[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const float2 t = p_add(f[3 * l], f[3 * l + 2]);
        X0[l] = p_add(t, f[3 * l + 1]);
        X1[l] = p_sub(f[3 * l + 2], f[3 * l]);
        X2[l] = t;
    }
    // y: only the combinations of total order <= 2
    float2 Y00[3], Y01[3], Y02[3], Y10[3], Y11[3], Y20[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 t0 = p_add(X0[3 * c], X0[3 * c + 2]);
        Y00[c] = p_add(t0, X0[3 * c + 1]);
        Y01[c] = p_sub(X0[3 * c + 2], X0[3 * c]);
        Y02[c] = t0;
        Y10[c] = p_add(p_add(X1[3 * c], X1[3 * c + 1]), X1[3 * c + 2]);
        Y11[c] = p_sub(X1[3 * c + 2], X1[3 * c]);
        Y20[c] = p_add(p_add(X2[3 * c], X2[3 * c + 1]), X2[3 * c + 2]);
    }
    // z, and the unscaled raw moments
    const float2 tz = p_add(Y00[0], Y00[2]);
    float2 drho = p_add(tz, Y00[1]);
    float2 jz = p_sub(Y00[2], Y00[0]);
    float2 pzz = tz;
    float2 jy = p_add(p_add(Y01[0], Y01[1]), Y01[2]);
    float2 pyz = p_sub(Y01[2], Y01[0]);
    float2 jx = p_add(p_add(Y10[0], Y10[1]), Y10[2]);
    float2 pxz = p_sub(Y10[2], Y10[0]);
    float2 pyy = p_add(p_add(Y02[0], Y02[1]), Y02[2]);
    float2 pxy = p_add(p_add(Y11[0], Y11[1]), Y11[2]);
    float2 pxx = p_add(p_add(Y20[0], Y20[1]), Y20[2]);
    if (scaled) {
        const float2 is = p_set(1.f / scale);
        drho = p_mul(drho, is); jz = p_mul(jz, is); pzz = p_mul(pzz, is);
        jy = p_mul(jy, is); pyz = p_mul(pyz, is); jx = p_mul(jx, is);
        pxz = p_mul(pxz, is); pyy = p_mul(pyy, is); pxy = p_mul(pxy, is);
        pxx = p_mul(pxx, is);
    }
    if (HREF) {
        // moments of sum_q w_q r(c_qz) (1, c, c c): per-axis weights (1/6, 2/3, 1/6)
        const float r0 = (ref.rd[0] + ref.rd[2]) * (1.f / 6.f);
        const float rr = fmaf(ref.rd[1], 2.f / 3.f, r0);
        drho = p_add(drho, p_set(rr));
        jz = p_add(jz, p_set((ref.rd[2] - ref.rd[0]) * (1.f / 6.f)));
        pzz = p_add(pzz, p_set(r0));
        pxx = p_add(pxx, p_set(rr * (1.f / 3.f)));
        pyy = p_add(pyy, p_set(rr * (1.f / 3.f)));
    }
    const float2 rho = p_add(p_set(1.f), drho);
    const float2 inv = make_float2(1.f / rho.x, 1.f / rho.y);
    const float2 Fx = p_mul(rho, p_set(gx)), Fy = p_mul(rho, p_set(gy)), Fz = p_mul(rho, p_set(gz));
    const float2 half = p_set(0.5f);
    const float2 ux = p_mul(p_fma(half, Fx, jx), inv);
    const float2 uy = p_mul(p_fma(half, Fy, jy), inv);
    const float2 uz = p_mul(p_fma(half, Fz, jz), inv);
    // central second-order moments: k_ab = P_ab - u_a j_b - u_b j_a + rho u_a u_b
    const float2 m1 = p_set(-1.f), m2 = p_set(-2.f);
    const float2 njx = p_mul(jx, m1), njy = p_mul(jy, m1), njz = p_mul(jz, m1);
    const float2 kxx = p_fma(ux, p_fma(rho, ux, p_mul(jx, m2)), pxx);
    const float2 kyy = p_fma(uy, p_fma(rho, uy, p_mul(jy, m2)), pyy);
    const float2 kzz = p_fma(uz, p_fma(rho, uz, p_mul(jz, m2)), pzz);
    const float2 kxy = p_fma(uy, njx, p_fma(ux, p_fma(rho, uy, njy), pxy));
    const float2 kxz = p_fma(uz, njx, p_fma(ux, p_fma(rho, uz, njz), pxz));
    const float2 kyz = p_fma(uz, njy, p_fma(uy, p_fma(rho, uz, njz), pyz));
    // relaxation: shear parts with omega, the trace to rho
    const float2 om1 = p_set(1.f - omega);
    const float2 third = p_set(1.f / 3.f);
    const float2 Dxy = p_mul(om1, p_sub(kxx, kyy));
    const float2 Dxz = p_mul(om1, p_sub(kxx, kzz));
    const float2 a200 = p_mul(p_add(Dxy, Dxz), third);
    const float2 a020 = p_mul(p_fma(Dxy, m2, Dxz), third);
    const float2 a002 = p_mul(p_fma(Dxz, m2, Dxy), third);
    const float2 drho3 = p_mul(drho, third);
    const float2 k110 = p_mul(om1, kxy), k101 = p_mul(om1, kxz), k011 = p_mul(om1, kyz);
    // normalised post-collision second-order cumulants
    const float2 sxx = p_mul(a200, inv), syy = p_mul(a020, inv), szz = p_mul(a002, inv);
    const float2 Sxy = p_mul(k110, inv), Sxz = p_mul(k101, inv), Syz = p_mul(k011, inv);
    const float2 rs = scaled ? p_mul(rho, p_set(scale)) : rho;
    const float2 sc = p_set(scale);
    auto scl = [&](float2 v) { return scaled ? p_mul(v, sc) : v; };
    // post-collision central moments m[a + 3b + 9c] (times the scale)
    f[0] = scl(drho);
    f[1] = p_mul(Fx, p_set(0.5f * scale));
    f[3] = p_mul(Fy, p_set(0.5f * scale));
    f[9] = p_mul(Fz, p_set(0.5f * scale));
    f[2] = scl(p_add(a200, drho3));
    f[6] = scl(p_add(a020, drho3));
    f[18] = scl(p_add(a002, drho3));
    f[4] = scl(k110);
    f[10] = scl(k101);
    f[12] = scl(k011);
    const float2 two = p_set(2.f);
    const float2 S2xy = p_mul(two, Sxy), S2xz = p_mul(two, Sxz), S2yz = p_mul(two, Syz);
    const float2 d9 = p_mul(drho, p_set(scale / 9.f));
    // fourth order: rest + rho ((s_a + s_b)/3 + s_a s_b + 2 S_ab^2)
    f[8] = p_fma(rs, p_fma(S2xy, Sxy, p_fma(sxx, syy, p_mul(p_add(sxx, syy), third))), d9);
    f[20] = p_fma(rs, p_fma(S2xz, Sxz, p_fma(sxx, szz, p_mul(p_add(sxx, szz), third))), d9);
    f[24] = p_fma(rs, p_fma(S2yz, Syz, p_fma(syy, szz, p_mul(p_add(syy, szz), third))), d9);
    const float2 tx = p_add(third, sxx), ty = p_add(third, syy), tzz = p_add(third, szz);
    f[14] = p_mul(rs, p_fma(S2xy, Sxz, p_mul(tx, Syz)));
    f[16] = p_mul(rs, p_fma(S2xy, Syz, p_mul(ty, Sxz)));
    f[22] = p_mul(rs, p_fma(S2xz, Syz, p_mul(tzz, Sxy)));
    {
        // sixth order
        const float2 sum = p_add(p_add(sxx, syy), szz);
        const float2 pairs = p_fma(sxx, syy, p_fma(sxx, szz, p_mul(syy, szz)));
        const float2 trip = p_mul(p_mul(sxx, syy), szz);
        const float2 sq = p_fma(tx, p_mul(Syz, Syz), p_fma(ty, p_mul(Sxz, Sxz), p_mul(tzz, p_mul(Sxy, Sxy))));
        const float2 cyc = p_mul(p_mul(Sxy, Sxz), Syz);
        float2 t = p_fma(sum, p_set(1.f / 9.f), p_mul(pairs, third));
        t = p_add(t, trip);
        t = p_fma(two, sq, t);
        t = p_fma(p_set(8.f), cyc, t);
        f[26] = p_fma(rs, t, p_mul(drho, p_set(scale / 27.f)));
    }
    // backward, x (lines (b, c); rest value scale mrest(b) mrest(c)); known
    // zeros: k210, k120, k201, k021, k102, k012, k111, k221, k212, k122
    const AxisCoef2 wx = axis_coef2(ux), wy = axis_coef2(uy), wz = axis_coef2(uz);
    constexpr float s1 = scale, s3 = scale / 3.f, s9 = scale / 9.f;
    bwd_line2<true, true, true>(f[0], f[1], f[2], wx, s1);       // (0,0)
    bwd_line2<true, true, false>(f[3], f[4], f[5], wx, 0.f);     // (1,0)
    bwd_line2<true, false, true>(f[6], f[7], f[8], wx, s3);      // (2,0)
    bwd_line2<true, true, false>(f[9], f[10], f[11], wx, 0.f);   // (0,1)
    bwd_line2<true, false, true>(f[12], f[13], f[14], wx, 0.f);  // (1,1)
    bwd_line2<false, true, false>(f[15], f[16], f[17], wx, 0.f); // (2,1)
    bwd_line2<true, false, true>(f[18], f[19], f[20], wx, s3);   // (0,2)
    bwd_line2<false, true, false>(f[21], f[22], f[23], wx, 0.f); // (1,2)
    bwd_line2<true, false, true>(f[24], f[25], f[26], wx, s9);   // (2,2)
    // y (lines (a, c); rest value scale w1(a) mrest(c)), then z (lines (a, b);
    // rest value scale w1(a) w1(b)): no known zeros left
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            bwd_line2<true, true, true>(f[a + 9 * c], f[a + 3 + 9 * c], f[a + 6 + 9 * c], wy,
                                        scale * w1(a) * mrest(c));
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            bwd_line2<true, true, true>(f[a + 3 * b], f[a + 3 * b + 9], f[a + 3 * b + 18], wz,
                                        scale * w1(a) * w1(b));
}

// loads and stores of two x-adjacent stored values; the pair starts on an
// even element, so the wide access is aligned
template <typename S> struct Pair;
template <> struct Pair<float> {
    static constexpr int SCALE_LOG2 = 0;
    __device__ static __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
    __device__ static __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
};
template <> struct Pair<__half> {
    static constexpr int SCALE_LOG2 = 12;
    __device__ static __forceinline__ float2 ld2(const __half* p) {
        return __half22float2(*reinterpret_cast<const __half2*>(p));
    }
    __device__ static __forceinline__ void st2(__half* p, float2 v) {
        *reinterpret_cast<__half2*>(p) = __float22half2_rn(v);
    }
};
template <> struct Pair<__nv_bfloat16> {
    static constexpr int SCALE_LOG2 = 0;
    __device__ static __forceinline__ float2 ld2(const __nv_bfloat16* p) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    }
    __device__ static __forceinline__ void st2(__nv_bfloat16* p, float2 v) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v);
    }
};
static_assert((float)(1u << Pair<__half>::SCALE_LOG2) == Store<__half>::scale, "FP16 storage scale");

}  // namespace fsl
