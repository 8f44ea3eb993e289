// k_fv_warp.cu -- the FV time step (Sec. II B: Eqs. (semi) and (semi-heun),
// QUICK faces of Sec. II B 3, double-reflection walls of Sec. II B 5) as a
// warp march: every strip of 32 column pairs is marched up a chunk of rows by
// one or two warps of its own, with no block-wide barrier.
//
//   stage A, row t:     moments, equilibrium and force of f~^n; h^n and
//                       f~ + Coll^n of the row;
//   stage B, row t - 2: A[h^n] -> f~*, f~ + Coll - dt/2 A[h^n], h*;
//   stage C, row t - 4: A[h*] -> f~^(n+1), stored.
//
// Where the stencils' data lives:
//   - y: every moving population keeps, in registers, its last two rows of h
//     (and of h*) and the face values still to be differenced: the QUICK
//     value of a face between two rows is formed once, when its last node
//     arrives, and carried to the one or two rows it bounds;
//   - x: the neighbouring column pairs are the neighbouring lanes, read by
//     warp shuffles; lanes 0 and 31 only feed their neighbours, so a strip
//     of 64 columns writes the 56 in its middle (stage B is valid on lanes
//     1..30, stage C on 2..29);
//   - f~ + Coll waits four rows between stages A and C in a private
//     shared-memory ring (five rows).
// A strip's populations may be split over two warps ("roles"): the nine f
// and the nine g of a thermal grid, or, for flow, {0, 1, 3, 5, 7} and
// {2, 4, 6, 8} (each set closed under inv, so a wall's ghosts stay within
// it).  The two warps add their moment sums through shared memory at a
// two-warp named barrier, twice per row.
//
// Walls on y: ghost rows are formed in the carried registers from the rows
// they mirror (h'_a = h'_inv(a) for f, -h'_inv(a) for g, in the base-state
// frame of lb_internal.cuh).  The face between the bottom wall and row 0
// needs row 1's mirror, so it is formed one row late, before its first use.
#include "lb_pair.cuh"

namespace lbgb {

namespace {

using namespace pairmath;

constexpr int kPairs = 32;              // column pairs per strip (one warp)
constexpr int kOut = 2 * (kPairs - 4);  // output columns per strip

// Populations a warp of role ROLE steps (SPW warps per strip).
template <bool TH, int SPW, int ROLE>
__host__ __device__ constexpr bool owns(int a) {
    if (TH || SPW == 1) return true;
    return ROLE == 0 ? (a == 0 || a == 1 || a == 3 || a == 5 || a == 7) : !(a == 0 || a == 1 || a == 3 || a == 5 || a == 7);
}
template <bool TH, int ROLE>
__host__ __device__ constexpr bool is_g() {
    return TH && ROLE == 1;
}
// Position of population a among the role's own populations (ring index).
template <bool TH, int SPW, int ROLE>
__host__ __device__ constexpr int own_index(int a) {
    int k = 0;
    for (int b = 0; b < a; ++b) k += owns<TH, SPW, ROLE>(b) ? 1 : 0;
    return k;
}
// Ring rows per thread: the most populations one role owns.
template <bool TH, int SPW>
__host__ __device__ constexpr int ring_pops() {
    return (TH || SPW == 1) ? Q : 5;
}

// x metric of the pair whose left column is c (the per-column table).
struct XW {
    float wp[3], mp[3], ep[3];
    float wm[3], mm[3], em[3];
    V2 inv;
};
__device__ __forceinline__ void load_xw(const float* tab, int c, XW& X) {
    const float4* p = reinterpret_cast<const float4*>(tab + 20 * c);
    const float4 a = __ldg(p), b = __ldg(p + 1), cc = __ldg(p + 2), d = __ldg(p + 3), e = __ldg(p + 4);
    X.wp[0] = a.x; X.wp[1] = a.y; X.wp[2] = a.z;
    X.mp[0] = a.w; X.mp[1] = b.x; X.mp[2] = b.y;
    X.ep[0] = b.z; X.ep[1] = b.w; X.ep[2] = cc.x;
    X.wm[0] = cc.y; X.wm[1] = cc.z; X.wm[2] = cc.w;
    X.mm[0] = d.x; X.mm[1] = d.y; X.mm[2] = d.z;
    X.em[0] = d.w; X.em[1] = e.x; X.em[2] = e.y;
    X.inv = mk(e.z, e.w);
}

// x flux divergence of a population with c_x = C (+1 or -1) at the lane's
// two columns; P is the lane's pair of the row, its neighbours' pairs come by
// shuffle.  Every lane of the warp must call it.
template <int C>
__device__ __forceinline__ V2 xdiv(V2 P, const XW& X) {
    const unsigned full = 0xffffffffu;
    float fw, fm, fe;
    if constexpr (C > 0) {
        const float l0 = __shfl_up_sync(full, P.v.x, 1), l1 = __shfl_up_sync(full, P.v.y, 1);
        const float r0 = __shfl_down_sync(full, P.v.x, 1);
        fw = X.wp[0] * l0 + X.wp[1] * l1 + X.wp[2] * P.v.x;
        fm = X.mp[0] * l1 + X.mp[1] * P.v.x + X.mp[2] * P.v.y;
        fe = X.ep[0] * P.v.x + X.ep[1] * P.v.y + X.ep[2] * r0;
        return (mk(fm, fe) - mk(fw, fm)) * X.inv;
    } else {
        const float l1 = __shfl_up_sync(full, P.v.y, 1);
        const float r0 = __shfl_down_sync(full, P.v.x, 1), r1 = __shfl_down_sync(full, P.v.y, 1);
        fw = X.wm[0] * l1 + X.wm[1] * P.v.x + X.wm[2] * P.v.y;
        fm = X.mm[0] * P.v.x + X.mm[1] * P.v.y + X.mm[2] * r0;
        fe = X.em[0] * P.v.y + X.em[1] * r0 + X.em[2] * r1;
        return bc(0.0f) - (mk(fm, fe) - mk(fw, fm)) * X.inv;
    }
}

// Weights of the face below row j (between rows j-1 and j): c > 0 from nodes
// j-2, j-1, j; c < 0 from nodes j-1, j, j+1.  They are row j's south face in
// the per-row table; the top wall face (j = ny) is row ny-1's north face;
// periodic rows wrap.  Faces beyond a wall are never used.
struct FW {
    V2 p[3], m[3];
};
// The table is the chunk's copy in shared memory: entry i is row base + i
// (wrapped on a periodic axis).  Indices outside the copy are clamped; only
// faces that no written row uses fall outside it.
struct ChunkTab {
    const float* t;
    int base, rows;
    __device__ __forceinline__ const float* entry(int r) const {
        int i = r - base;
        i = i < 0 ? 0 : (i >= rows ? rows - 1 : i);
        return t + 20 * i;
    }
};
__device__ __forceinline__ void load_fw(const ChunkTab& T, int j, int ny, bool wall, FW& F) {
    int r = j, op = 0, om = 6;
    if (wall && j >= ny) {
        r = ny - 1;
        op = 3;
        om = 9;
    }
    const float* e = T.entry(r);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        F.p[i] = bc(e[op + i]);
        F.m[i] = bc(e[om + i]);
    }
}

// Per-row data: 1/dy, base-state offsets, the base state's y flux divergences.
struct RW {
    float inv, ro, to, dref[4];
};
__device__ __forceinline__ void load_rw(const ChunkTab& T, int r, RW& R) {
    const float* e = T.entry(r);
    R.inv = e[12];
    R.ro = e[13];
    R.to = e[14];
#pragma unroll
    for (int i = 0; i < 4; ++i) R.dref[i] = e[15 + i];
}
__device__ __forceinline__ RW zero_rw() { return RW{0.f, 0.f, 0.f, {0.f, 0.f, 0.f, 0.f}}; }

// y flux divergence of the base state of population a (g if G), one row.
template <int a, bool G>
__device__ __forceinline__ float ref_y(const RW& R) {
    if constexpr (cy(a) == 0) return 0.0f;
    else return float(cy(a)) * wgt<float>(a) * R.dref[(G ? 2 : 0) + (cy(a) > 0 ? 0 : 1)];
}

// The carried state of the warp's populations for one advected field (h or
// h*): rows t-2 and t-1 of every moving population (hA, hB), and the face
// values still pending: below rows t-2 (FA) and t-1 (FB) for c_y > 0, below
// row t-2 (FA) for c_y < 0.
template <bool TH, int SPW, int ROLE>
struct Carry {
    V2 hA[Q], hB[Q], FA[Q], FB[Q];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int a = 0; a < Q; ++a) hA[a] = hB[a] = FA[a] = FB[a] = bc(0.0f);
    }
    // Takes row t (h), forms the faces below row t (c > 0, weights Ft.p) and
    // below row t-1 (c < 0, weights Fm.m), writes the y flux divergence of
    // row t-2 into dy (scaled by inv = 1/dy of row t-2) and shifts by a row.
    __device__ __forceinline__ void advance(const V2* h, const FW& Ft, const FW& Fm, V2 inv, V2* dy) {
#pragma unroll
        for (int a = 1; a < Q; ++a) {
            if (!owns<TH, SPW, ROLE>(a)) continue;
            if (cy(a) > 0) {
                const V2 Fn = fma2(Ft.p[0], hA[a], fma2(Ft.p[1], hB[a], Ft.p[2] * h[a]));
                dy[a] = (FB[a] - FA[a]) * inv;
                FA[a] = FB[a];
                FB[a] = Fn;
            } else if (cy(a) < 0) {
                const V2 Fn = fma2(Fm.m[0], hA[a], fma2(Fm.m[1], hB[a], Fm.m[2] * h[a]));
                dy[a] = bc(0.0f) - (Fn - FA[a]) * inv;
                FA[a] = Fn;
            }
            hA[a] = hB[a];
            hB[a] = h[a];
        }
    }
    // Bottom wall, before advancing row 1 (hB = row 0, h = row 1): ghost row
    // -1 replaces hA, and the wall face (below row 0, c_y > 0) is formed from
    // ghosts -2, -1 and row 0 into FB, so that the advance leaves it in FA.
    __device__ __forceinline__ void bottom_wall(const V2* h, const FW& F0, V2 sgn) {
#pragma unroll
        for (int a = 1; a < Q; ++a) {
            if (!owns<TH, SPW, ROLE>(a) || cy(a) == 0) continue;
            const V2 g1 = hB[inv(a)] * sgn, g2 = h[inv(a)] * sgn;
            if (cy(a) > 0) FB[a] = fma2(F0.p[0], g2, fma2(F0.p[1], g1, F0.p[2] * hB[a]));
            hA[a] = g1;
        }
    }
};

// Moments of a pair of cells from the moment sums (f: rho - rho_r, j_x, j_y;
// g: T - T_r), base-state frame, with the arithmetic of PairCell.
struct Mom {
    V2 rp, rho, ux, uy, Td, T, ay, uuneg, ua3neg;
    __device__ __forceinline__ void set(V2 r, V2 jx, V2 jy, V2 td, bool TH, const StepArgs<float>& A, float ro,
                                        float to) {
        rp = r;
        rho = r + bc(1.0f + ro);
        const V2 ir = mk(__fdividef(1.0f, rho.v.x), __fdividef(1.0f, rho.v.y));
        if (TH) {
            Td = td;
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
    }
    // f_eq - w rho_r and the Guo force F (G false), or g_eq - w T_r (G true).
    template <int a, bool G>
    __device__ __forceinline__ void eq(const StepArgs<float>& A, V2& e, V2& F) const {
        const float w = wgt<float>(a);
        V2 cu, ca;
        if constexpr (cx(a) == 0 && cy(a) == 0) {
            cu = bc(0.0f);
            ca = bc(0.0f);
        } else if constexpr (cy(a) == 0) {
            cu = ux * bc(float(cx(a)));
            ca = bc(float(cx(a)) * A.ax);
        } else if constexpr (cx(a) == 0) {
            cu = uy * bc(float(cy(a)));
            ca = ay * bc(float(cy(a)));
        } else {
            cu = fma2(uy, bc(float(cy(a))), ux * bc(float(cx(a))));
            ca = fma2(ay, bc(float(cy(a))), bc(float(cx(a)) * A.ax));
        }
        if constexpr (cx(a) == 0 && cy(a) == 0) {
            if constexpr (!G) {
                const V2 wr = rho * bc(w);
                e = fma2(wr, uuneg, rp * bc(w));
                F = wr * ua3neg;
            } else {
                e = fma2(T * bc(w), uuneg, Td * bc(w));
                F = bc(0.0f);
            }
        } else {
            const V2 q = fma2(cu * bc(4.5f), cu, uuneg);
            const V2 pa = fma2(bc(3.0f), cu, q);
            if constexpr (!G) {
                const V2 wr = rho * bc(w);
                e = fma2(wr, pa, rp * bc(w));
                const V2 t = ca * bc(3.0f);
                F = wr * (fma2(cu * bc(3.0f), t, ua3neg) + t);
            } else {
                e = fma2(T * bc(w), pa, Td * bc(w));
                F = bc(0.0f);
            }
        }
    }
};

__device__ __forceinline__ void pair_barrier(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// The moment sums of the warp's populations of a row pair-cell.
template <bool TH, int SPW, int ROLE>
__device__ __forceinline__ void partial_sums(const V2* d, V2& r, V2& jx, V2& jy, V2& td) {
    r = jx = jy = td = bc(0.0f);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        if (!owns<TH, SPW, ROLE>(a)) continue;
        if (is_g<TH, ROLE>()) {
            td = td + d[a];
        } else {
            r = r + d[a];
            if (cx(a) != 0) jx = cx(a) > 0 ? jx + d[a] : jx - d[a];
            if (cy(a) != 0) jy = cy(a) > 0 ? jy + d[a] : jy - d[a];
        }
    }
}

// The whole march of one warp of role ROLE.
template <typename S, bool TH, int SPW, int ROLE, int NW>
__device__ __forceinline__ void march(const StepArgs<float>& A, const int CH, V2* ring, V2* xch, V2* ghost,
                                      const ChunkTab& T) {
    constexpr int NTH = 32 * NW;
    constexpr int RP = ring_pops<TH, SPW>();
    constexpr bool G = is_g<TH, ROLE>();
    const V2 sgn = bc(G ? -1.0f : 1.0f);  // wall rule in the base-state frame
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int strip = blockIdx.x * (NW / SPW) + warp / SPW;
    const int xu = strip * kOut - 4 + 2 * lane;  // unwrapped left column of the lane's pair
    const int nx = A.nx, ny = A.ny;
    const int gxl = ((xu % nx) + nx) % nx, gxr = ((xu + 1) % nx + nx) % nx;
    const bool contiguous = xu >= 0 && xu + 1 < nx;
    const bool laneC = lane >= 2 && lane < 30 && xu < nx;
    const bool both = xu + 1 < nx;
    const int ys = blockIdx.y * CH;
    const int ye = min(ys + CH, ny);
    const bool wall = A.bcy == LB_BC_WALLS;
    const int bar = 1 + warp / SPW;  // two-warp barrier of the strip (SPW == 2)
    V2* xs = xch + (warp / SPW) * 2 * 2 * 4 * 32;  // [2 stages][2 roles][4 sums][32 lanes]

    XW X;
    load_xw(A.coltab, gxl, X);
    const S* in = static_cast<const S*>(G ? A.gin : A.fin);
    S* out = static_cast<S*>(G ? A.gout : A.fout);
    const float omh = G ? A.omgh : A.omh, om = G ? A.omg : A.om;

    auto fluid = [&](int r, int& g) { return map_axis(r, ny, A.bcy, g); };
    auto load_pops = [&](int r, V2* b) {
        int gy;
        if (r < ye + 4 && fluid(r, gy)) {
            const long long row = (long long)gy * A.pitch;
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                if (!owns<TH, SPW, ROLE>(a)) continue;
                const S* base = in + a * A.plane + row;
                b[a] = contiguous ? PairIO<S>::ld(base + xu) : mk(Store<S>::ld(base + gxl), Store<S>::ld(base + gxr));
            }
        }
    };
    // Full moment sums of a pair-cell: the warp's own plus its partner's
    // (two-warp strips).  Each role writes its sums to its own slot of the
    // stage, both meet at the strip's barrier and both add role 0's sums to
    // role 1's, in that order, so both hold the same bits.  A slot is
    // rewritten one stage later, after the partner has passed the next
    // barrier, so one barrier per exchange suffices.
    auto full_sums = [&](int stage, V2& r, V2& jx, V2& jy, V2& td) {
        if constexpr (SPW == 2) {
            V2* mine = xs + (stage * 2 + ROLE) * 4 * 32;
            V2* other = xs + (stage * 2 + (1 - ROLE)) * 4 * 32;
            mine[lane] = r;
            mine[32 + lane] = jx;
            mine[64 + lane] = jy;
            mine[96 + lane] = td;
            pair_barrier(bar);
            const V2 r1 = other[lane], jx1 = other[32 + lane], jy1 = other[64 + lane], td1 = other[96 + lane];
            if (ROLE == 0) {
                r = r + r1;
                jx = jx + jx1;
                jy = jy + jy1;
                td = td + td1;
            } else {
                r = r1 + r;
                jx = jx1 + jx;
                jy = jy1 + jy;
                td = td1 + td;
            }
        }
    };
    auto slot = [](int r) { return ((r % 5) + 5) % 5; };

    V2 b0[Q], b1[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) b0[a] = b1[a] = bc(0.0f);
    load_pops(ys - 4, b0);
    load_pops(ys - 3, b1);
    Carry<TH, SPW, ROLE> Ch, Cs;  // the carries of h^n and of h*
    Ch.zero();
    Cs.zero();
    V2* gh = ghost + threadIdx.x;  // [2 fields][RP][NTH]: the top wall's second ghost rows

    for (int t = ys - 4; t < ye + 4; ++t) {
        // ---- stage A: row t ----
        V2 d[Q], h[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            d[a] = b0[a];
            b0[a] = b1[a];
            h[a] = bc(0.0f);
        }
        load_pops(t + 2, b1);
        int gA;
        const bool fA = fluid(t, gA);
        RW RA = zero_rw();
        if (fA) load_rw(T, t, RA);  // the copy is indexed by the unwrapped row
        {
            V2 r, jx, jy, td;
            partial_sums<TH, SPW, ROLE>(d, r, jx, jy, td);
            full_sums(0, r, jx, jy, td);
            if (fA) {
                Mom m;
                m.set(r, jx, jy, td, TH, A, RA.ro, TH ? RA.to : 0.0f);
                V2* rs = ring + slot(t) * RP * NTH + threadIdx.x;
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    if (!owns<TH, SPW, ROLE>(a)) continue;
                    V2 e, F;
                    switch (a) {
                        case 0: m.template eq<0, G>(A, e, F); break;
                        case 1: m.template eq<1, G>(A, e, F); break;
                        case 2: m.template eq<2, G>(A, e, F); break;
                        case 3: m.template eq<3, G>(A, e, F); break;
                        case 4: m.template eq<4, G>(A, e, F); break;
                        case 5: m.template eq<5, G>(A, e, F); break;
                        case 6: m.template eq<6, G>(A, e, F); break;
                        case 7: m.template eq<7, G>(A, e, F); break;
                        default: m.template eq<8, G>(A, e, F); break;
                    }
                    const V2 neq = e - d[a];
                    if (G) {
                        h[a] = fma2(bc(omh), neq, d[a]);
                        rs[own_index<TH, SPW, ROLE>(a) * NTH] = fma2(bc(om), neq, d[a]);
                    } else {
                        h[a] = fma2(bc(omh), neq, fma2(bc(A.hf), F, d[a]));
                        rs[own_index<TH, SPW, ROLE>(a) * NTH] = fma2(bc(om), neq, fma2(bc(A.cf), F, d[a]));
                    }
                }
            } else if (wall && t == ny) {
                // rows ny and ny+1 mirror rows ny-1 and ny-2
#pragma unroll
                for (int a = 1; a < Q; ++a) {
                    if (!owns<TH, SPW, ROLE>(a)) continue;
                    h[a] = Ch.hB[inv(a)] * sgn;
                    gh[own_index<TH, SPW, ROLE>(a) * NTH] = Ch.hA[inv(a)] * sgn;
                }
            } else if (wall && t == ny + 1) {
#pragma unroll
                for (int a = 1; a < Q; ++a)
                    if (owns<TH, SPW, ROLE>(a)) h[a] = gh[own_index<TH, SPW, ROLE>(a) * NTH];
            }
        }
        if (wall && t == 1 && ys == 0) {
            FW F0;
            load_fw(T, 0, ny, wall, F0);
            Ch.bottom_wall(h, F0, sgn);
        }

        // ---- stage B: row t - 2 ----
        const int rB = t - 2;
        int gB;
        const bool fB = fluid(rB, gB);
        RW RB = zero_rw();
        if (fB) load_rw(T, rB, RB);
        V2 adv[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) adv[a] = bc(0.0f);
        // x divergences of row t - 2 (its h is the carry's hA before advancing)
#pragma unroll
        for (int a = 1; a < Q; ++a) {
            if (!owns<TH, SPW, ROLE>(a) || cx(a) == 0) continue;
            adv[a] = cx(a) > 0 ? xdiv<1>(Ch.hA[a], X) : xdiv<-1>(Ch.hA[a], X);
        }
        {
            FW Ft, Fm;
            load_fw(T, t, ny, wall, Ft);
            load_fw(T, t - 1, ny, wall, Fm);
            V2 dy[Q];
            Ch.advance(h, Ft, Fm, bc(RB.inv), dy);
#pragma unroll
            for (int a = 1; a < Q; ++a)
                if (owns<TH, SPW, ROLE>(a) && cy(a) != 0) adv[a] = adv[a] + dy[a];
        }
        V2 hs[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) hs[a] = bc(0.0f);
        {
            const bool doB = fB && rB >= ys - 2 && rB < ye + 2;
            V2 fs[Q];
            V2* rs = ring + slot(rB) * RP * NTH + threadIdx.x;
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                fs[a] = bc(0.0f);
                if (!owns<TH, SPW, ROLE>(a) || !doB) continue;
                V2 ref;
                switch (a) {
                    case 1: ref = bc(ref_y<1, G>(RB)); break;
                    case 2: ref = bc(ref_y<2, G>(RB)); break;
                    case 3: ref = bc(ref_y<3, G>(RB)); break;
                    case 4: ref = bc(ref_y<4, G>(RB)); break;
                    case 5: ref = bc(ref_y<5, G>(RB)); break;
                    case 6: ref = bc(ref_y<6, G>(RB)); break;
                    case 7: ref = bc(ref_y<7, G>(RB)); break;
                    case 8: ref = bc(ref_y<8, G>(RB)); break;
                    default: ref = bc(0.0f); break;
                }
                const V2 av = adv[a] + ref;
                const V2 fc = rs[own_index<TH, SPW, ROLE>(a) * NTH];
                fs[a] = fma2(bc(-A.dt), av, fc);
                rs[own_index<TH, SPW, ROLE>(a) * NTH] = fma2(bc(-A.hf), av, fc);
            }
            V2 r, jx, jy, td;
            partial_sums<TH, SPW, ROLE>(fs, r, jx, jy, td);
            full_sums(1, r, jx, jy, td);
            if (doB) {
                Mom m;
                m.set(r, jx, jy, td, TH, A, RB.ro, TH ? RB.to : 0.0f);
#pragma unroll
                for (int a = 1; a < Q; ++a) {
                    if (!owns<TH, SPW, ROLE>(a)) continue;
                    V2 e, F;
                    switch (a) {
                        case 1: m.template eq<1, G>(A, e, F); break;
                        case 2: m.template eq<2, G>(A, e, F); break;
                        case 3: m.template eq<3, G>(A, e, F); break;
                        case 4: m.template eq<4, G>(A, e, F); break;
                        case 5: m.template eq<5, G>(A, e, F); break;
                        case 6: m.template eq<6, G>(A, e, F); break;
                        case 7: m.template eq<7, G>(A, e, F); break;
                        default: m.template eq<8, G>(A, e, F); break;
                    }
                    if (G) hs[a] = fma2(bc(omh), e - fs[a], fs[a]);
                    else hs[a] = fma2(bc(omh), e - fs[a], fma2(bc(A.hf), F, fs[a]));
                }
            } else if (wall && rB == ny) {
#pragma unroll
                for (int a = 1; a < Q; ++a) {
                    if (!owns<TH, SPW, ROLE>(a)) continue;
                    hs[a] = Cs.hB[inv(a)] * sgn;
                    gh[(RP + own_index<TH, SPW, ROLE>(a)) * NTH] = Cs.hA[inv(a)] * sgn;
                }
            } else if (wall && rB == ny + 1) {
#pragma unroll
                for (int a = 1; a < Q; ++a)
                    if (owns<TH, SPW, ROLE>(a)) hs[a] = gh[(RP + own_index<TH, SPW, ROLE>(a)) * NTH];
            }
        }
        if (wall && rB == 1 && ys == 0) {
            FW F0;
            load_fw(T, 0, ny, wall, F0);
            Cs.bottom_wall(hs, F0, sgn);
        }

        // ---- stage C: row t - 4 ----
        const int rC = t - 4;
        RW RC = zero_rw();
        const bool doC = rC >= ys && rC < ye;
        if (doC) load_rw(T, rC, RC);
        V2 advs[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) advs[a] = bc(0.0f);
#pragma unroll
        for (int a = 1; a < Q; ++a) {
            if (!owns<TH, SPW, ROLE>(a) || cx(a) == 0) continue;
            advs[a] = cx(a) > 0 ? xdiv<1>(Cs.hA[a], X) : xdiv<-1>(Cs.hA[a], X);
        }
        {
            FW Ft, Fm;
            load_fw(T, rB, ny, wall, Ft);
            load_fw(T, rB - 1, ny, wall, Fm);
            V2 dy[Q];
            Cs.advance(hs, Ft, Fm, bc(RC.inv), dy);
#pragma unroll
            for (int a = 1; a < Q; ++a)
                if (owns<TH, SPW, ROLE>(a) && cy(a) != 0) advs[a] = advs[a] + dy[a];
        }
        if (doC && laneC) {
            const long long row = (long long)rC * A.pitch;
            const V2* rs = ring + slot(rC) * RP * NTH + threadIdx.x;
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                if (!owns<TH, SPW, ROLE>(a)) continue;
                V2 ref;
                switch (a) {
                    case 1: ref = bc(ref_y<1, G>(RC)); break;
                    case 2: ref = bc(ref_y<2, G>(RC)); break;
                    case 3: ref = bc(ref_y<3, G>(RC)); break;
                    case 4: ref = bc(ref_y<4, G>(RC)); break;
                    case 5: ref = bc(ref_y<5, G>(RC)); break;
                    case 6: ref = bc(ref_y<6, G>(RC)); break;
                    case 7: ref = bc(ref_y<7, G>(RC)); break;
                    case 8: ref = bc(ref_y<8, G>(RC)); break;
                    default: ref = bc(0.0f); break;
                }
                const V2 o = fma2(bc(-A.hf), advs[a] + ref, rs[own_index<TH, SPW, ROLE>(a) * NTH]);
                S* base = out + a * A.plane + row;
                if (both) PairIO<S>::st(base + xu, o);
                else Store<S>::st(base + xu, o.v.x);
            }
        }
    }
}

}  // namespace

// NW warps per CTA; SPW warps per strip (2: the strip's populations split
// into two roles).  blockIdx.x picks NW / SPW strips, blockIdx.y the chunk.
template <typename S, bool TH, int SPW, int NW>
__global__ void __launch_bounds__(32 * NW) k_fv_warp(const StepArgs<float> A, const int CH) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NTH = 32 * NW;
    constexpr int RP = ring_pops<TH, SPW>();
    V2* ring = reinterpret_cast<V2*>(smem_raw);  // [5][RP][NTH]
    V2* ghost = ring + 5 * RP * NTH;             // [2][RP][NTH]
    V2* xch = ghost + 2 * RP * NTH;              // [NW / SPW][2][2][4][32]
    float* tab = reinterpret_cast<float*>(xch + (NW / SPW) * 2 * 2 * 4 * 32);  // [CH + 8][20]
    // the chunk's rows ys-4 .. ye+3 of the per-row table, copied once
    const int ys = blockIdx.y * CH, ye = min(ys + CH, A.ny);
    const ChunkTab T{tab, ys - 4, ye - ys + 8};
    for (int k = threadIdx.x; k < 5 * T.rows; k += NTH) {
        int gy;
        const float4 v = map_axis(T.base + k / 5, A.ny, A.bcy, gy)
                             ? __ldg(reinterpret_cast<const float4*>(A.rowtab) + 5 * gy + k % 5)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<float4*>(tab)[k] = v;
    }
    __syncthreads();
    const int role = (threadIdx.x >> 5) % SPW;
    if (role == 0) march<S, TH, SPW, 0, NW>(A, CH, ring, xch, ghost, T);
    else if constexpr (SPW == 2) march<S, TH, SPW, 1, NW>(A, CH, ring, xch, ghost, T);
}

template <typename S, bool TH, int SPW>
static cudaError_t run_warp(const StepArgs<float>& A, int chunk, cudaStream_t s) {
    constexpr int NW = 4;
    constexpr int NTH = 32 * NW;
    const int ch = chunk < 8 ? 8 : (chunk > 1024 ? 1024 : chunk);
    const size_t smem = sizeof(V2) * ((5 + 2) * ring_pops<TH, SPW>() * NTH + (NW / SPW) * 2 * 2 * 4 * 32) +
                        sizeof(float) * 20 * (size_t)(ch + 8);
    {
        cudaError_t e = set_max_smem((const void*)k_fv_warp<S, TH, SPW, NW>, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int strips = (A.nx + kOut - 1) / kOut;
    constexpr int per_cta = NW / SPW;
    dim3 grid((strips + per_cta - 1) / per_cta, (A.ny + ch - 1) / ch);
    k_fv_warp<S, TH, SPW, NW><<<grid, NTH, smem, s>>>(A, ch);
    count_launch();
    return cudaGetLastError();
}

// Flow grids march each strip with one warp; thermal grids step f and g in
// the strip's two warps.
cudaError_t launch_fv_warp(Prec p, bool th, const void* args, int chunk, cudaStream_t s) {
    const StepArgs<float>& A = *static_cast<const StepArgs<float>*>(args);
    switch (p) {
        case Prec::F32:
            return th ? run_warp<float, true, 2>(A, chunk, s) : run_warp<float, false, 1>(A, chunk, s);
        case Prec::F16:
            return th ? run_warp<__half, true, 2>(A, chunk, s) : run_warp<__half, false, 1>(A, chunk, s);
        case Prec::BF16:
            return th ? run_warp<__nv_bfloat16, true, 2>(A, chunk, s) : run_warp<__nv_bfloat16, false, 1>(A, chunk, s);
        default:
            return cudaErrorInvalidValue;
    }
}

int warp_width() { return kOut; }
// Strips per CTA and shared memory per CTA of launch_fv_warp's kernels.
int warp_strips_per_cta(bool th) { return th ? 2 : 4; }

}  // namespace lbgb
