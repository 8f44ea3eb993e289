// lb3_pair.cuh -- moments and equilibria of two adjacent x cells of the
// D3Q19 lattice at once, in packed FP32 pairs (Blackwell f32x2), shared by
// the paired 3-D ST kernel and the paired 3-D FV collision and star passes.
//
// Storage holds deviations from a constant reference (d = f - w, e = g -
// w T0), so rho = 1 + sum d and T = T0 + sum e; the buoyancy makes a_z a
// per-cell value, a_z + beta g (T - T0); u = sum c d / rho + hf a (hf = dt/2
// for tilded populations, Appendix A).
#pragma once

#include "lb3.cuh"
#include "lb_pair.cuh"

namespace lbgb {
namespace pairmath {

template <bool TH>
struct Cell3P {
    V2 rp, rho, ux, uy, uz, Td, T, az, uu, ua;

    __device__ __forceinline__ void moments(const V2* d, const V2* e, const Args3<float>& A) {
        V2 r = bc(0.0f), jx = bc(0.0f), jy = bc(0.0f), jz = bc(0.0f);
#pragma unroll
        for (int a = 0; a < Q3; ++a) {
            r = r + d[a];
            if (c3x(a) != 0) jx = c3x(a) > 0 ? jx + d[a] : jx - d[a];
            if (c3y(a) != 0) jy = c3y(a) > 0 ? jy + d[a] : jy - d[a];
            if (c3z(a) != 0) jz = c3z(a) > 0 ? jz + d[a] : jz - d[a];
        }
        V2 td = bc(0.0f);
        if constexpr (TH) {
#pragma unroll
            for (int a = 0; a < Q3; ++a) td = td + e[a];
        }
        from_sums(r, jx, jy, jz, td, A);
    }

    // the same from the sums sum d, sum c d (3) and sum e
    __device__ __forceinline__ void from_sums(V2 r, V2 jx, V2 jy, V2 jz, V2 td, const Args3<float>& A) {
        Td = TH ? td : bc(0.0f);
        rp = r;
        rho = r + bc(1.0f);
        T = Td + bc(A.T0);
        az = TH ? fma2(bc(A.bg), Td, bc(A.az)) : bc(A.az);
        const V2 ir = mk(__fdividef(1.0f, rho.v.x), __fdividef(1.0f, rho.v.y));
        ux = fma2(jx, ir, bc(A.hf * A.ax));
        uy = fma2(jy, ir, bc(A.hf * A.ay));
        uz = fma2(az, bc(A.hf), jz * ir);
        uu = fma2(ux, ux, fma2(uy, uy, uz * uz));
        ua = fma2(ux, bc(A.ax), fma2(uy, bc(A.ay), uz * az));
    }

    // population a: f_eq - w (feqd), the Guo force F (Eq. (F2)) and, if
    // thermal, g_eq - w T0 (geqd)
    template <int a>
    __device__ __forceinline__ void eq(const Args3<float>& A, V2& feqd, V2& F, V2& geqd) const {
        const float w = w3<float>(a);
        V2 cu = bc(0.0f), ca = bc(0.0f);
        if constexpr (c3x(a) != 0) {
            cu = ux * bc(float(c3x(a)));
            ca = bc(float(c3x(a)) * A.ax);
        }
        if constexpr (c3y(a) != 0) {
            cu = fma2(uy, bc(float(c3y(a))), cu);
            ca = ca + bc(float(c3y(a)) * A.ay);
        }
        if constexpr (c3z(a) != 0) {
            cu = fma2(uz, bc(float(c3z(a))), cu);
            ca = fma2(az, bc(float(c3z(a))), ca);
        }
        // 3 c.u + 4.5 (c.u)^2 - 1.5 u.u
        const V2 poly = fma2(cu, fma2(cu, bc(4.5f), bc(3.0f)), uu * bc(-1.5f));
        feqd = (rp + rho * poly) * bc(w);
        F = (rho * bc(w)) * fma2(bc(9.0f), cu * ca, (ca - ua) * bc(3.0f));
        geqd = TH ? (Td + T * poly) * bc(w) : bc(0.0f);
    }
};

}  // namespace pairmath
}  // namespace lbgb
