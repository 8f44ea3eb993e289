// lb_pair.cuh -- packed FP32 pair arithmetic (Blackwell f32x2 FMA, ADD, MUL)
// and the collision data of two cells at once, shared by the paired FV and
// ST kernels.
#pragma once

#include "lb_internal.cuh"

namespace lbgb {
namespace pairmath {

struct V2 {
    float2 v;
};
__device__ __forceinline__ V2 mk(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ V2 bc(float s) { return {make_float2(s, s)}; }
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 fma2(V2 a, V2 b, V2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return fma2(b, bc(-1.0f), a); }

// Pair loads/stores of the deviation storage (see Store<> for the scales).
template <typename S> struct PairIO;
template <> struct PairIO<float> {
    __device__ static V2 ld(const float* p) { return {__ldg(reinterpret_cast<const float2*>(p))}; }
    __device__ static void st(float* p, V2 v) { *reinterpret_cast<float2*>(p) = v.v; }
};
template <> struct PairIO<__half> {
    __device__ static V2 ld(const __half* p) {
        float2 f = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
        return {make_float2(f.x * (1.0f / kF16Scale), f.y * (1.0f / kF16Scale))};
    }
    __device__ static void st(__half* p, V2 v) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v.v.x * kF16Scale, v.v.y * kF16Scale);
    }
};
template <> struct PairIO<__nv_bfloat16> {
    __device__ static V2 ld(const __nv_bfloat16* p) {
        return {__bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)))};
    }
    __device__ static void st(__nv_bfloat16* p, V2 v) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.v.x, v.v.y);
    }
};

// Collision data of a pair of cells on one row (base-state frame, see
// lb_internal.cuh): moments, then per population the deviation of f_eq, the
// Guo force and (thermal) the deviation of g_eq.
template <bool TH>
struct PairCell {
    V2 rp, rho, ux, uy, Td, T, ay, uuneg, ua3neg;
    V2 feqd[Q], F[Q], geqd[Q];

    __device__ __forceinline__ void build(const V2* d, const V2* e, const StepArgs<float>& A, float ro, float to) {
        V2 r = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
        V2 jx = (d[1] + d[5] + d[8]) - (d[3] + d[6] + d[7]);
        V2 jy = (d[2] + d[5] + d[6]) - (d[4] + d[7] + d[8]);
        rp = r;
        rho = r + bc(1.0f + ro);
        V2 ir = mk(__fdividef(1.0f, rho.v.x), __fdividef(1.0f, rho.v.y));
        if (TH) {
            Td = ((e[0] + e[1]) + (e[2] + e[3])) + ((e[4] + e[5]) + (e[6] + e[7])) + e[8];
            const V2 dT0 = Td + bc(to);
            T = dT0 + bc(A.T0);
            ay = fma2(bc(A.bg), dT0, bc(A.ay));
        } else {
            ay = bc(A.ay);
        }
        ux = fma2(jx, ir, bc(A.hf * A.ax));
        uy = fma2(ay, bc(A.hf), jy * ir);
        uuneg = (ux * ux + uy * uy) * bc(-1.5f);
        ua3neg = fma2(uy, ay, ux * bc(A.ax)) * bc(-3.0f);
        // rest population: c = 0
        const float w0 = wgt<float>(0);
        const V2 wr0 = rho * bc(w0);
        feqd[0] = fma2(wr0, uuneg, rp * bc(w0));
        F[0] = wr0 * ua3neg;
        if (TH) geqd[0] = fma2(T * bc(w0), uuneg, Td * bc(w0));
        pair<1>(A);
        pair<2>(A);
        pair<5>(A);
        pair<6>(A);
    }

    // populations a and inv(a): c.u and c.a flip sign, squares do not.
    template <int a>
    __device__ __forceinline__ void pair(const StepArgs<float>& A) {
        constexpr int b = inv(a);
        const float w = wgt<float>(a);
        V2 cu, ca;
        if constexpr (a == 1) { cu = ux; ca = bc(A.ax); }
        else if constexpr (a == 2) { cu = uy; ca = ay; }
        else if constexpr (a == 5) { cu = ux + uy; ca = ay + bc(A.ax); }
        else { cu = uy - ux; ca = ay - bc(A.ax); }  // a == 6: c = (-1, 1)
        const V2 q = fma2(cu * bc(4.5f), cu, uuneg);  // 4.5 (c.u)^2 - 1.5 u.u
        const V2 pa = fma2(bc(3.0f), cu, q), pb = fma2(bc(-3.0f), cu, q);
        const V2 wr = rho * bc(w), wrp = rp * bc(w);
        feqd[a] = fma2(wr, pa, wrp);
        feqd[b] = fma2(wr, pb, wrp);
        const V2 t = ca * bc(3.0f);
        const V2 m = fma2(cu * bc(3.0f), t, ua3neg);  // 9 (c.u)(c.a) - 3 u.a
        F[a] = wr * (m + t);
        F[b] = wr * (m - t);
        if (TH) {
            const V2 wT = T * bc(w), wTd = Td * bc(w);
            geqd[a] = fma2(wT, pa, wTd);
            geqd[b] = fma2(wT, pb, wTd);
        }
    }
};

// Collision of a pair of cells in storage units (deviations times K: the
// FP16 scale 2^12, or 1 for BF16 and FP32) on a flow grid, whose base state is
// rho_r = 1 on every row.  The BGK relaxation with the Guo force,
//   post_a = d_a + om (feq_a - f_a) + cf F_a,
// is regrouped per pair of opposite populations a, b = inv(a): with
// cu3 = 3 c_a.u, t = 3 c_a.a (a uniform constant), w = w_a and
//   C0 = om (-1.5 u.u) + cf (-3 u.a),
//   g  = (om/2) cu3 + cf t,   S = cu3 g + C0,   D = g + (om/2) cu3,
// the two results are
//   post_a = (1 - om) d_a + om w K (rho - 1) + w K rho (S + D),
//   post_b = (1 - om) d_b + om w K (rho - 1) + w K rho (S - D),
// which is the same polynomial as f_eq = w rho (1 + 3 c.u + 4.5 (c.u)^2
// - 1.5 u.u) and F = w rho (3 (c - u).a + 9 (c.u)(c.a)) (Sec. II A), with
// the even part S and the odd part D shared by a and b.  Moments come from
// the sums divided by K once; no population is rescaled on load or store.
template <int K_>
__device__ __forceinline__ void collide_units(const V2* d, const StepArgs<float>& A, V2* post) {
    constexpr float K = float(K_), iK = 1.0f / K;
    const float om = A.om, om1 = 1.0f - A.om, omh = 0.5f * A.om;
    const V2 e1 = d[1] - d[3], e2 = d[2] - d[4], e57 = d[5] - d[7], e68 = d[6] - d[8];
    const V2 rK = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    const V2 jx = ((e1 + e57) - e68) * bc(iK), jy = ((e2 + e57) + e68) * bc(iK);
    const V2 rho = fma2(rK, bc(iK), bc(1.0f));
    const V2 ir = mk(__fdividef(1.0f, rho.v.x), __fdividef(1.0f, rho.v.y));
    const V2 ux = fma2(jx, ir, bc(A.hf * A.ax));
    const V2 uy = fma2(bc(A.ay), bc(A.hf), jy * ir);
    const V2 ux3 = ux * bc(3.0f), uy3 = uy * bc(3.0f);
    const V2 uuneg = fma2(ux, ux, uy * uy) * bc(-1.5f);
    const V2 ua3neg = fma2(uy3, bc(-A.ay), ux3 * bc(-A.ax));
    const V2 C0 = fma2(bc(om), uuneg, bc(A.cf) * ua3neg);
    post[0] = fma2(rho * bc(K * wgt<float>(0)), C0, fma2(bc(om1), d[0], rK * bc(om * wgt<float>(0))));
    const V2 wrA = rho * bc(K * wgt<float>(1)), wrD = rho * bc(K * wgt<float>(5));
    const V2 bA = rK * bc(om * wgt<float>(1)), bD = rK * bc(om * wgt<float>(5));
#pragma unroll
    for (int a : {1, 2, 5, 6}) {
        const int b = inv(a);
        V2 cu3;
        float ct;  // cf t
        if (a == 1) { cu3 = ux3; ct = 3.0f * A.cf * A.ax; }
        else if (a == 2) { cu3 = uy3; ct = 3.0f * A.cf * A.ay; }
        else if (a == 5) { cu3 = ux3 + uy3; ct = 3.0f * A.cf * (A.ay + A.ax); }
        else { cu3 = uy3 - ux3; ct = 3.0f * A.cf * (A.ay - A.ax); }  // a == 6: c = (-1, 1)
        const V2 g = fma2(cu3, bc(omh), bc(ct));
        const V2 Sv = fma2(cu3, g, C0), Dv = fma2(cu3, bc(omh), g);
        const V2 wr = a < 5 ? wrA : wrD, bb = a < 5 ? bA : bD;
        post[a] = fma2(wr, Sv + Dv, fma2(bc(om1), d[a], bb));
        post[b] = fma2(wr, Sv - Dv, fma2(bc(om1), d[b], bb));
    }
}

// Moments of a pair of cells and the relaxations the FV stages build from
// them: stage A needs two of one cell (the advected field h and f~ + Coll),
// stage B one (h*).  In the base-state frame (d = f - w rho_r, rp = sum d =
// rho - rho_r, e = g - w T_r, Td = sum e = T - T_r)
//   relax_f: out_a = d_a + k1 (feqd_a - d_a) + k2 F_a
//          = (1 - k1) d_a + k1 w rp + w rho (S +- D)   (a and b = inv(a)),
//     with cu3 = 3 c_a.u, t = 3 c_a.a, C0 = k1 (-1.5 u.u) + k2 (-3 u.a),
//     g = (k1/2) cu3 + k2 t, S = cu3 g + C0, D = g + (k1/2) cu3: the even
//     part S and the odd part D of f_eq and F (Sec. II A) shared by the pair;
//   relax_g: out_a = e_a + k (geqd_a - e_a), geqd_a = w (Td + T (3 c.u +
//     4.5 (c.u)^2 - 1.5 u.u)).
// The thermal buoyancy makes a_y a per-cell value: a_y + beta g (T - T0).
template <bool TH>
struct PairMom {
    V2 rp, rho, ux3, uy3, ay, uuneg, ua3neg, Td, T;

    __device__ __forceinline__ void build(const V2* d, const V2* e, const StepArgs<float>& A, float ro, float to) {
        const V2 e1 = d[1] - d[3], e2 = d[2] - d[4], e57 = d[5] - d[7], e68 = d[6] - d[8];
        rp = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
        const V2 jx = (e1 + e57) - e68, jy = (e2 + e57) + e68;
        rho = rp + bc(1.0f + ro);
        const V2 ir = mk(__fdividef(1.0f, rho.v.x), __fdividef(1.0f, rho.v.y));
        if constexpr (TH) {
            Td = ((e[0] + e[1]) + (e[2] + e[3])) + ((e[4] + e[5]) + (e[6] + e[7])) + e[8];
            const V2 dT0 = Td + bc(to);
            T = dT0 + bc(A.T0);
            ay = fma2(bc(A.bg), dT0, bc(A.ay));
        } else {
            ay = bc(A.ay);
        }
        const V2 ux = fma2(jx, ir, bc(A.hf * A.ax));
        const V2 uy = fma2(ay, bc(A.hf), jy * ir);
        ux3 = ux * bc(3.0f);
        uy3 = uy * bc(3.0f);
        uuneg = fma2(ux, ux, uy * uy) * bc(-1.5f);
        ua3neg = fma2(uy3, ay, ux3 * bc(A.ax)) * bc(-1.0f);
    }

    template <int a>
    __device__ __forceinline__ V2 cu3_of() const {
        if constexpr (a == 1) return ux3;
        else if constexpr (a == 2) return uy3;
        else if constexpr (a == 5) return ux3 + uy3;
        else return uy3 - ux3;  // a == 6: c = (-1, 1)
    }

    __device__ __forceinline__ void relax_f(const V2* d, const StepArgs<float>& A, float k1, float k2, V2* out) const {
        const float k1h = 0.5f * k1, k1c = 1.0f - k1;
        const V2 C0 = fma2(bc(k1), uuneg, bc(k2) * ua3neg);
        const V2 cty = ay * bc(3.0f * k2);
        const float ctx = 3.0f * k2 * A.ax;
        out[0] = fma2(rho * bc(wgt<float>(0)), C0, fma2(bc(k1c), d[0], rp * bc(k1 * wgt<float>(0))));
        const V2 wrA = rho * bc(wgt<float>(1)), wrD = rho * bc(wgt<float>(5));
        const V2 bA = rp * bc(k1 * wgt<float>(1)), bD = rp * bc(k1 * wgt<float>(5));
        pair_f<1>(d, k1h, k1c, C0, bc(ctx), wrA, bA, out);
        pair_f<2>(d, k1h, k1c, C0, cty, wrA, bA, out);
        pair_f<5>(d, k1h, k1c, C0, cty + bc(ctx), wrD, bD, out);
        pair_f<6>(d, k1h, k1c, C0, cty - bc(ctx), wrD, bD, out);
    }

    template <int a>
    __device__ __forceinline__ void pair_f(const V2* d, float k1h, float k1c, V2 C0, V2 ct, V2 wr, V2 bb,
                                           V2* out) const {
        constexpr int b = inv(a);
        const V2 cu3 = cu3_of<a>();
        const V2 g = fma2(cu3, bc(k1h), ct);
        const V2 Sv = fma2(cu3, g, C0), Dv = fma2(cu3, bc(k1h), g);
        out[a] = fma2(wr, Sv + Dv, fma2(bc(k1c), d[a], bb));
        out[b] = fma2(wr, Sv - Dv, fma2(bc(k1c), d[b], bb));
    }

    __device__ __forceinline__ void relax_g(const V2* e, float k, V2* out) const {
        const float w0 = wgt<float>(0);
        out[0] = fma2(bc(k), fma2(T * bc(w0), uuneg, Td * bc(w0)) - e[0], e[0]);
        pair_g<1>(e, k, out);
        pair_g<2>(e, k, out);
        pair_g<5>(e, k, out);
        pair_g<6>(e, k, out);
    }

    template <int a>
    __device__ __forceinline__ void pair_g(const V2* e, float k, V2* out) const {
        constexpr int b = inv(a);
        const V2 cu3 = cu3_of<a>();
        const V2 q = fma2(cu3 * bc(0.5f), cu3, uuneg);  // 4.5 (c.u)^2 - 1.5 u.u
        const V2 wT = T * bc(wgt<float>(a)), wTd = Td * bc(wgt<float>(a));
        out[a] = fma2(bc(k), fma2(wT, cu3 + q, wTd) - e[a], e[a]);
        out[b] = fma2(bc(k), fma2(wT, q - cu3, wTd) - e[b], e[b]);
    }
};

}  // namespace pairmath
}  // namespace lbgb
