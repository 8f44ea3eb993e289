// k_fv_pair.cu -- the FV time step (Sec. II B: Eqs. (semi), (semi-heun),
// QUICK faces of Sec. II B 3, double-reflection walls of Sec. II B 5) in
// kernels where every thread owns two adjacent columns and all arithmetic
// runs on packed FP32 pairs (Blackwell's f32x2 FMA, ADD and MUL: one
// instruction for both columns):
//   k_fv_pair             y-marching strips (below);
//   k_fv_ptile            the tile step of k_fv.cu on column pairs;
//   k_fv_split_a / _c     the tile step in two launches;
//   k_fv_ptile_batched    the paired tile over the server's request table.
//
// March structure as in k_fv_march.cu: stage A forms h^n and f~ + Coll^n of
// row t, stage B forms f~* and h* of row t - 2, stage C writes f~^(n+1) of
// row t - 4; rows live in 5-slot shared-memory rings, one barrier per row.
// Pairing adds:
//   - populations are loaded and stored two columns at a time (8-byte FP32,
//     4-byte half2 / bfloat162), so 16-bit storage also halves instructions;
//   - equilibrium and Guo force are formed for each pair of opposite
//     velocities together (they share c.u squared and the force terms);
//   - the two columns share their middle x face, so an x flux needs three
//     face values for two cells instead of four.
// The kernel serves x-periodic grids (every workload here); grids with walls
// on x use the scalar kernels.
#include "lb_pair.cuh"

namespace lbgb {

namespace {

using namespace pairmath;

__device__ __forceinline__ int slot5(int r) {
    const int s = r % 5;
    return s < 0 ? s + 5 : s;
}

// x metric of the thread's two columns: faces W (west of the left column),
// M (between them) and E (east of the right one), both upwind directions.
struct XPair {
    float wp[3], mp[3], ep[3];  // c > 0: nodes (k-2, k-1, k) of face k
    float wm[3], mm[3], em[3];  // c < 0: nodes (k-1, k, k+1)
    V2 inv;
};

// One row of the per-row table (20 floats, 80 bytes): QUICK weights of the
// row's south and north faces for both upwind directions, 1/dy, the base
// state offsets and the base state's y flux divergences.
struct YPair {
    V2 ps[3], pn[3], ms[3], mn[3], inv;
    float ro, to, dref[4];
};

// The raw 80 bytes of a row entry, so that a row's entry can be loaded one
// row ahead of its use and unpacked when it is needed.
struct RowRaw {
    float4 a, b, c, d, e;
};
__device__ __forceinline__ void load_raw(const float* tab, int g, RowRaw& R) {
    const float4* p = reinterpret_cast<const float4*>(tab + 20 * g);
    R.a = __ldg(p); R.b = __ldg(p + 1); R.c = __ldg(p + 2); R.d = __ldg(p + 3); R.e = __ldg(p + 4);
}
__device__ __forceinline__ void unpack_row(const RowRaw& R, YPair& Y) {
    const float4 a = R.a, b = R.b, c = R.c, d = R.d, e = R.e;
    Y.ps[0] = bc(a.x); Y.ps[1] = bc(a.y); Y.ps[2] = bc(a.z);
    Y.pn[0] = bc(a.w); Y.pn[1] = bc(b.x); Y.pn[2] = bc(b.y);
    Y.ms[0] = bc(b.z); Y.ms[1] = bc(b.w); Y.ms[2] = bc(c.x);
    Y.mn[0] = bc(c.y); Y.mn[1] = bc(c.z); Y.mn[2] = bc(c.w);
    Y.inv = bc(d.x);
    Y.ro = d.y;
    Y.to = d.z;
    Y.dref[0] = d.w; Y.dref[1] = e.x; Y.dref[2] = e.y; Y.dref[3] = e.z;
}

__device__ __forceinline__ void load_row(const float* tab, int g, YPair& Y) {
    const float4* p = reinterpret_cast<const float4*>(tab + 20 * g);
    const float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3), e = __ldg(p + 4);
    Y.ps[0] = bc(a.x); Y.ps[1] = bc(a.y); Y.ps[2] = bc(a.z);
    Y.pn[0] = bc(a.w); Y.pn[1] = bc(b.x); Y.pn[2] = bc(b.y);
    Y.ms[0] = bc(b.z); Y.ms[1] = bc(b.w); Y.ms[2] = bc(c.x);
    Y.mn[0] = bc(c.y); Y.mn[1] = bc(c.z); Y.mn[2] = bc(c.w);
    Y.inv = bc(d.x);
    Y.ro = d.y;
    Y.to = d.z;
    Y.dref[0] = d.w; Y.dref[1] = e.x; Y.dref[2] = e.y; Y.dref[3] = e.z;
}

// y flux divergence of the base state for population a (row data).
template <int a>
__device__ __forceinline__ float row_ref_flux(const YPair& Y, bool thermal) {
    if constexpr (cy(a) == 0) {
        return 0.0f;
    } else {
        return float(cy(a)) * wgt<float>(a) * Y.dref[(thermal ? 2 : 0) + (cy(a) > 0 ? 0 : 1)];
    }
}

// Rows each population's advected field keeps in the marching rings: five
// for c_y != 0 (the y stencil spans rows r-2..r+2), three for the x-only
// populations (their row is read two iterations after it is written, by
// the x stencil), none for the rest population, whose field never moves.
// Population p >= Q is the thermal population p - Q.
__host__ __device__ constexpr int ring_depth(int p) {
    return cy(p % Q) != 0 ? 5 : (cx(p % Q) != 0 ? 3 : 0);
}
// First ring row of population p: the depths of the D2Q9 order (0, 3, 5, 3,
// 5, 5, 5, 5, 5; 36 rows) in closed form, so that every index folds to a
// constant (a recursive sum is not folded when called with a loop index).
__host__ __device__ constexpr int ring_off(int p) {
    const int a = p % Q;
    return 36 * (p / Q) + (a <= 1 ? 0 : a == 2 ? 3 : a == 3 ? 8 : a == 4 ? 11 : 16 + 5 * (a - 5));
}
constexpr int ring_sum(int p) { return p == 0 ? 0 : ring_sum(p - 1) + ring_depth(p - 1); }
static_assert(ring_off(1) == ring_sum(1) && ring_off(2) == ring_sum(2) && ring_off(3) == ring_sum(3) &&
                  ring_off(4) == ring_sum(4) && ring_off(5) == ring_sum(5) && ring_off(8) == ring_sum(8) &&
                  ring_off(9) == ring_sum(9) && ring_off(13) == ring_sum(13) && ring_off(18) == ring_sum(18),
              "ring offsets");

// Flux divergence of population p (velocity a) for the thread's two
// columns.  Its ring holds rows r-2..r+2 in slots sl[0..4] (depth 5) or row
// r in slot c3 (depth 3); x neighbours are the pairs of threads k-1, k+1.
template <int NQ, int NT, int a>
__device__ __forceinline__ V2 advect_pair(const V2* ring, const int* sl, int c3, int p, int k, const XPair& X,
                                          const YPair& Y) {
    V2 v = bc(0.0f);
    const V2* base = ring + ring_off(p) * NT;
    if constexpr (cx(a) != 0) {
        const V2* row = base + (ring_depth(p) == 5 ? sl[2] : c3) * NT;
        const float2 P0 = row[k - 1].v, P1 = row[k].v, P2 = row[k + 1].v;  // columns 2k-2 .. 2k+3
        float fw, fm, fe;
        if constexpr (cx(a) > 0) {
            fw = X.wp[0] * P0.x + X.wp[1] * P0.y + X.wp[2] * P1.x;
            fm = X.mp[0] * P0.y + X.mp[1] * P1.x + X.mp[2] * P1.y;
            fe = X.ep[0] * P1.x + X.ep[1] * P1.y + X.ep[2] * P2.x;
        } else {
            fw = X.wm[0] * P0.y + X.wm[1] * P1.x + X.wm[2] * P1.y;
            fm = X.mm[0] * P1.x + X.mm[1] * P1.y + X.mm[2] * P2.x;
            fe = X.em[0] * P1.y + X.em[1] * P2.x + X.em[2] * P2.y;
        }
        const V2 dx = (mk(fm, fe) - mk(fw, fm)) * X.inv;
        v = cx(a) > 0 ? dx : v - dx;
    }
    if constexpr (cy(a) != 0) {
        V2 c[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) c[i] = base[sl[i] * NT + k];
        V2 fn, fs;
        if constexpr (cy(a) > 0) {
            fn = fma2(Y.pn[0], c[1], fma2(Y.pn[1], c[2], Y.pn[2] * c[3]));
            fs = fma2(Y.ps[0], c[0], fma2(Y.ps[1], c[1], Y.ps[2] * c[2]));
            v = fma2(fn - fs, Y.inv, v);
        } else {
            fn = fma2(Y.mn[0], c[2], fma2(Y.mn[1], c[3], Y.mn[2] * c[4]));
            fs = fma2(Y.ms[0], c[1], fma2(Y.ms[1], c[2], Y.ms[2] * c[3]));
            v = v - (fn - fs) * Y.inv;
        }
    }
    return v;
}

template <bool TH, int NQ, int NT, int a>
__device__ __forceinline__ void advect_all(const V2* ring, const int* sl, int c3, int k, const XPair& X,
                                           const YPair& Y, const StepArgs<float>& A, int gy, V2* out) {
    out[a] = advect_pair<NQ, NT, a>(ring, sl, c3, a, k, X, Y) + bc(row_ref_flux<a>(Y, false));
    if constexpr (TH)
        out[Q + a] = advect_pair<NQ, NT, a>(ring, sl, c3, Q + a, k, X, Y) + bc(row_ref_flux<a>(Y, true));
    if constexpr (a + 1 < Q) advect_all<TH, NQ, NT, a + 1>(ring, sl, c3, k, X, Y, A, gy, out);
}

// Ghost row of a wall on y (own columns), base-state deviations: h'_a =
// h'_inv(a) for f and -h'_inv(a) for g.  Only the populations with c_y != 0
// read ghost rows (the x stencil runs on fluid rows); a and inv(a) share
// their ring depth.
template <bool TH, int NQ, int NT>
__device__ __forceinline__ void ghost_row(V2* ring, int dst, int src, int k) {
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        if (ring_depth(a) != 5) continue;
        ring[(ring_off(a) + dst) * NT + k] = ring[(ring_off(inv(a)) + src) * NT + k];
        if constexpr (TH)
            ring[(ring_off(Q + a) + dst) * NT + k] = bc(0.0f) - ring[(ring_off(Q + inv(a)) + src) * NT + k];
    }
}

}  // namespace

template <typename S, bool TH, int NT>
__global__ void __launch_bounds__(NT) k_fv_pair(const StepArgs<float> A, const int CH) {
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr int W = 2 * NT - 8;  // output columns per strip
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int HR = ring_off(NQ);            // rows of the h and h* rings (all populations)
    V2* sH = reinterpret_cast<V2*>(smem_raw);  // [HR][NT] h^n, ring_depth(p) rows of population p
    V2* sP = sH + HR * NT;                     // [5][NQ][NT] f~ + Coll, then - dt/2 A[h^n] (own)
    V2* sS = sP + 5 * NQ * NT;                 // [HR][NT] h*
    const int k = threadIdx.x;
    const int xu = blockIdx.x * W - 4 + 2 * k;  // unwrapped left column of the pair
    const int ys = blockIdx.y * CH;
    const int ye = min(ys + CH, A.ny);
    const int nx = A.nx;
    const int gxl = ((xu % nx) + nx) % nx;
    const int gxr = ((xu + 1) % nx + nx) % nx;
    const bool contiguous = xu >= 0 && xu + 1 < nx;  // pair stored side by side
    const bool colB = k >= 1 && k < NT - 1;
    const bool colC = k >= 2 && k < NT - 2 && xu < nx;
    const bool wally = A.bcy == LB_BC_WALLS;

    XPair X;
    if (colB) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            X.wp[r] = A.mx.wp(r, gxl);
            X.mp[r] = A.mx.wp(r, gxl + 1);
            X.ep[r] = A.mx.wp(r, gxr + 1);
            X.wm[r] = A.mx.wm(r, gxl);
            X.mm[r] = A.mx.wm(r, gxl + 1);
            X.em[r] = A.mx.wm(r, gxr + 1);
        }
        X.inv = mk(A.mx.invd(gxl), A.mx.invd(gxr));
    }

    const S* fin = static_cast<const S*>(A.fin);
    const S* gin = static_cast<const S*>(A.gin);
    S* fout = static_cast<S*>(A.fout);
    S* gout = static_cast<S*>(A.gout);

    auto fluid_row = [&](int r, int& gy) { return map_axis(r, A.ny, A.bcy, gy); };
    auto load_pair = [&](const S* base, int gy, V2& out) {
        const long long row = (long long)gy * A.pitch;
        if (contiguous) {
            out = PairIO<S>::ld(base + row + xu);
        } else {
            out = mk(Store<S>::ld(base + row + gxl), Store<S>::ld(base + row + gxr));
        }
    };
    // populations of row r into (bd, be), and the row's base-state offsets
    // into bo; rows are loaded two iterations before stage A needs them, so
    // the DRAM latency overlaps two rows of work
    auto prefetch = [&](int r, V2* bd, V2* be, float4& bo) {
        int gy;
        if (r < ye + 4 && fluid_row(r, gy)) {
            bo = __ldg(reinterpret_cast<const float4*>(A.rowtab + 20 * gy) + 3);
#pragma unroll
            for (int a = 0; a < Q; ++a) load_pair(fin + a * A.plane, gy, bd[a]);
            if constexpr (TH) {
#pragma unroll
                for (int a = 0; a < Q; ++a) load_pair(gin + a * A.plane, gy, be[a]);
            }
        }
    };

    // register buffers: (b0, e0, o0) hold row t, (b1, e1, o1) row t + 1 (in flight)
    V2 b0[Q], e0[Q], b1[Q], e1[Q];
    float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0;
    prefetch(ys - 4, b0, e0, o0);
    prefetch(ys - 3, b1, e1, o1);
    // row tables of stages B (row t - 2) and C (row t - 4), loaded one
    // iteration before their use
    RowRaw rb{}, rc{};
    auto next_tables = [&](int t) {
        int gy;
        const int r = t - 2;
        if (r >= ys - 2 && r < ye + 2 && fluid_row(r, gy) && colB) load_raw(A.rowtab, gy, rb);
        if (t - 4 >= ys && t - 4 < ye && colC) load_raw(A.rowtab, t - 4, rc);
    };
    next_tables(ys - 4);
    int s0 = slot5(ys - 4);  // slot of row t
    int t3 = ((ys - 4) % 3 + 3) % 3;  // slot of row t in the 3-row rings
    for (int t = ys - 4; t < ye + 4; ++t) {
        // 3-row ring slots of rows t - 2 and t - 4 (rows three apart share one)
        const int c3b = t3 == 2 ? 0 : t3 + 1, c3c = t3 == 0 ? 2 : t3 - 1;
        // m[i] = slot of row t - 4 + i (rows t - 4 .. t; m[4] = s0), since
        // rows five apart share a slot
        int m[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const int v = s0 + 1 + i;
            m[i] = v >= 5 ? v - 5 : v;
        }
        // ---- stage A on row t ----
        {
            int gy;
            const int s = s0;
            V2 d[Q], e[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                d[a] = b0[a];
                b0[a] = b1[a];
                if constexpr (TH) {
                    e[a] = e0[a];
                    e0[a] = e1[a];
                }
            }
            const float4 o = o0;
            o0 = o1;
            prefetch(t + 2, b1, e1, o1);
            if (fluid_row(t, gy)) {
                PairMom<TH> c;
                c.build(d, e, A, o.y, TH ? o.z : 0.0f);
                V2 hv[Q], pv[Q], hg[Q], pg[Q];
                c.relax_f(d, A, A.omh, A.hF, hv);
                c.relax_f(d, A, A.om, A.cf, pv);
                if constexpr (TH) {
                    c.relax_g(e, A.omgh, hg);
                    c.relax_g(e, A.omg, pg);
                }
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    if (ring_depth(a) > 0) sH[(ring_off(a) + (ring_depth(a) == 5 ? s : t3)) * NT + k] = hv[a];
                    sP[(s * NQ + a) * NT + k] = pv[a];
                    if constexpr (TH) {
                        if (ring_depth(a) > 0)
                            sH[(ring_off(Q + a) + (ring_depth(a) == 5 ? s : t3)) * NT + k] = hg[a];
                        sP[(s * NQ + Q + a) * NT + k] = pg[a];
                    }
                }
            } else if (wally && (t == A.ny || t == A.ny + 1)) {
                ghost_row<TH, NQ, NT>(sH, s, slot5(2 * A.ny - 1 - t), k);
            }
            if (wally && t == 1 && ys == 0) {
                ghost_row<TH, NQ, NT>(sH, slot5(-1), slot5(0), k);
                ghost_row<TH, NQ, NT>(sH, slot5(-2), slot5(1), k);
            }
        }
        // ---- stage B on row t - 2: rows t-4 .. t are slots m[0] .. m[4] ----
        {
            const int r = t - 2;
            int gy;
            if (r >= ys - 2 && r < ye + 2) {
                const int s = m[2];
                if (fluid_row(r, gy)) {
                    if (colB) {
                        YPair Y;
                        unpack_row(rb, Y);
                        const int sl[5] = {m[0], m[1], m[2], m[3], m[4]};
                        V2 adv[NQ];
                        advect_all<TH, NQ, NT, 0>(sH, sl, c3b, k, X, Y, A, gy, adv);
                        V2 fs[Q], es[Q];
#pragma unroll
                        for (int a = 0; a < Q; ++a) {
                            const V2 fc = sP[(s * NQ + a) * NT + k];
                            fs[a] = fma2(bc(-A.dt), adv[a], fc);
                            sP[(s * NQ + a) * NT + k] = fma2(bc(-A.hf), adv[a], fc);
                            if constexpr (TH) {
                                const V2 gc = sP[(s * NQ + Q + a) * NT + k];
                                es[a] = fma2(bc(-A.dt), adv[Q + a], gc);
                                sP[(s * NQ + Q + a) * NT + k] = fma2(bc(-A.hf), adv[Q + a], gc);
                            }
                        }
                        PairMom<TH> c;
                        c.build(fs, es, A, Y.ro, TH ? Y.to : 0.0f);
                        V2 hv[Q], hg[Q];
                        c.relax_f(fs, A, A.omh, A.hF, hv);
                        if constexpr (TH) c.relax_g(es, A.omgh, hg);
#pragma unroll
                        for (int a = 0; a < Q; ++a) {
                            if (ring_depth(a) == 0) continue;
                            const int sa = ring_depth(a) == 5 ? s : c3b;
                            sS[(ring_off(a) + sa) * NT + k] = hv[a];
                            if constexpr (TH) sS[(ring_off(Q + a) + sa) * NT + k] = hg[a];
                        }
                    }
                } else if (wally && (r == A.ny || r == A.ny + 1)) {
                    ghost_row<TH, NQ, NT>(sS, s, slot5(2 * A.ny - 1 - r), k);
                }
                if (wally && r == 1 && ys == 0) {
                    ghost_row<TH, NQ, NT>(sS, slot5(-1), slot5(0), k);
                    ghost_row<TH, NQ, NT>(sS, slot5(-2), slot5(1), k);
                }
            }
        }
        // ---- stage C on row t - 4: rows t-6 .. t-2 are slots m[3], m[4], m[0], m[1], m[2] ----
        {
            const int r = t - 4;
            if (r >= ys && r < ye && colC) {
                const int s = m[0];
                YPair Y;
                unpack_row(rc, Y);
                const int sl[5] = {m[3], m[4], m[0], m[1], m[2]};
                V2 adv[NQ];
                advect_all<TH, NQ, NT, 0>(sS, sl, c3c, k, X, Y, A, r, adv);
                const long long row = (long long)r * A.pitch;
                const bool both = xu + 1 < nx;
#pragma unroll
                for (int a = 0; a < NQ; ++a) {
                    const V2 o = fma2(bc(-A.hf), adv[a], sP[(s * NQ + a) * NT + k]);
                    S* base = (a < Q ? fout + a * A.plane : gout + (a - Q) * A.plane) + row;
                    if (both) PairIO<S>::st(base + xu, o);
                    else Store<S>::st(base + xu, o.v.x);
                }
            }
        }
        next_tables(t + 1);
        __syncthreads();
        s0 = m[0];  // slot of row t + 1 (= slot of row t - 4)
        t3 = t3 == 2 ? 0 : t3 + 1;
    }
}

// ---------------------------------------------------------------------------
// Paired tile kernel: the tile decomposition of k_fv.cu (TX x TY outputs,
// regions E4 = tile + 4 and E2 = tile + 2 in shared memory) with two columns
// per thread-cell and packed FP32 pair arithmetic.  For grids too small to
// fill the GPU with marching strips, and for the 18-population thermal case.

// x metric of the pair whose left column is g: from the per-column table
// (20 floats: wp at faces g, g+1, g_r+1; wm at the same faces; 1/dx of both).
__device__ __forceinline__ void load_col(const float* tab, int g, XPair& X) {
    const float4* p = reinterpret_cast<const float4*>(tab + 20 * g);
    const float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3), e = __ldg(p + 4);
    X.wp[0] = a.x; X.wp[1] = a.y; X.wp[2] = a.z;
    X.mp[0] = a.w; X.mp[1] = b.x; X.mp[2] = b.y;
    X.ep[0] = b.z; X.ep[1] = b.w; X.ep[2] = c.x;
    X.wm[0] = c.y; X.wm[1] = c.z; X.wm[2] = c.w;
    X.mm[0] = d.x; X.mm[1] = d.y; X.mm[2] = d.z;
    X.em[0] = d.w; X.em[1] = e.x; X.em[2] = e.y;
    X.inv = mk(e.z, e.w);
}

// The same entries from a shared-memory copy of the tables.
__device__ __forceinline__ void load_col_s(const float4* p, XPair& X) {
    const float4 a = p[0], b = p[1], c = p[2], d = p[3], e = p[4];
    X.wp[0] = a.x; X.wp[1] = a.y; X.wp[2] = a.z;
    X.mp[0] = a.w; X.mp[1] = b.x; X.mp[2] = b.y;
    X.ep[0] = b.z; X.ep[1] = b.w; X.ep[2] = c.x;
    X.wm[0] = c.y; X.wm[1] = c.z; X.wm[2] = c.w;
    X.mm[0] = d.x; X.mm[1] = d.y; X.mm[2] = d.z;
    X.em[0] = d.w; X.em[1] = e.x; X.em[2] = e.y;
    X.inv = mk(e.z, e.w);
}
__device__ __forceinline__ void load_row_s(const float4* p, YPair& Y) {
    RowRaw R{p[0], p[1], p[2], p[3], p[4]};
    unpack_row(R, Y);
}

// Floats of the per-tile copy of the row and column tables: the rows and
// pair-columns of region E2 (tile + 2).
__host__ __device__ constexpr int ptile_tab_floats(int TX, int TY) { return 20 * ((TY + 4) + (TX + 4) / 2); }

// Flux divergence of population a at pair-cell (px, y) of a region plane
// with row stride W pairs.
template <int a>
__device__ __forceinline__ V2 advect_region(const V2* plane, int W, int px, int y, const XPair& X, const YPair& Y) {
    V2 v = bc(0.0f);
    if constexpr (cx(a) != 0) {
        const V2* row = plane + y * W;
        const float2 P0 = row[px - 1].v, P1 = row[px].v, P2 = row[px + 1].v;
        float fw, fm, fe;
        if constexpr (cx(a) > 0) {
            fw = X.wp[0] * P0.x + X.wp[1] * P0.y + X.wp[2] * P1.x;
            fm = X.mp[0] * P0.y + X.mp[1] * P1.x + X.mp[2] * P1.y;
            fe = X.ep[0] * P1.x + X.ep[1] * P1.y + X.ep[2] * P2.x;
        } else {
            fw = X.wm[0] * P0.y + X.wm[1] * P1.x + X.wm[2] * P1.y;
            fm = X.mm[0] * P1.x + X.mm[1] * P1.y + X.mm[2] * P2.x;
            fe = X.em[0] * P1.y + X.em[1] * P2.x + X.em[2] * P2.y;
        }
        const V2 dx = (mk(fm, fe) - mk(fw, fm)) * X.inv;
        v = cx(a) > 0 ? dx : v - dx;
    }
    if constexpr (cy(a) != 0) {
        V2 c[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) c[i] = plane[(y - 2 + i) * W + px];
        if constexpr (cy(a) > 0) {
            const V2 fn = fma2(Y.pn[0], c[1], fma2(Y.pn[1], c[2], Y.pn[2] * c[3]));
            const V2 fs = fma2(Y.ps[0], c[0], fma2(Y.ps[1], c[1], Y.ps[2] * c[2]));
            v = fma2(fn - fs, Y.inv, v);
        } else {
            const V2 fn = fma2(Y.mn[0], c[2], fma2(Y.mn[1], c[3], Y.mn[2] * c[4]));
            const V2 fs = fma2(Y.ms[0], c[1], fma2(Y.ms[1], c[2], Y.ms[2] * c[3]));
            v = v - (fn - fs) * Y.inv;
        }
    }
    return v;
}

template <bool TH, int NQ, int H, int W, int a>
__device__ __forceinline__ void advect_region_all(const V2* P, int px, int y, const XPair& X, const YPair& Y,
                                                  V2* out) {
    out[a] = advect_region<a>(P + a * H * W, W, px, y, X, Y) + bc(row_ref_flux<a>(Y, false));
    if constexpr (TH) out[Q + a] = advect_region<a>(P + (Q + a) * H * W, W, px, y, X, Y) + bc(row_ref_flux<a>(Y, true));
    if constexpr (a + 1 < Q) advect_region_all<TH, NQ, H, W, a + 1>(P, px, y, X, Y, out);
}

// The populations i (0..NQ-1; i >= Q are thermal) whose bit is set in M,
// for a corrector split over two threads per pair-cell.
template <bool TH, int H, int W, unsigned M, int i>
__device__ __forceinline__ void advect_region_mask(const V2* P, int px, int y, const XPair& X, const YPair& Y,
                                                   V2* out) {
    constexpr int NQ = TH ? 2 * Q : Q;
    if constexpr ((M >> i) & 1u) {
        constexpr int a = i < Q ? i : i - Q;
        out[i] = advect_region<a>(P + i * H * W, W, px, y, X, Y) + bc(row_ref_flux<a>(Y, i >= Q));
    }
    if constexpr (i + 1 < NQ) advect_region_mask<TH, H, W, M, i + 1>(P, px, y, X, Y, out);
}

// Ghost rows of a region (walls on y), own pair-columns: h'_a = h'_inv(a)
// for f, -h'_inv(a) for g.
template <bool TH, int NQ, int H, int W>
__device__ __forceinline__ void ghost_rows_region(V2* P, int gy0, const StepArgs<float>& A) {
    if (A.bcy != LB_BC_WALLS) return;
    for (int k = threadIdx.x; k < W * 4; k += blockDim.x) {
        const int px = k % W, which = k / W;
        const int kk = (which & 1) + 1;
        const bool bot = which < 2;
        const int gy = bot ? -kk : A.ny - 1 + kk;
        const int gys = bot ? kk - 1 : A.ny - kk;
        const int ey = gy - gy0, eys = gys - gy0;
        if (ey < 0 || ey >= H) continue;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            P[(a * H + ey) * W + px] = P[(inv(a) * H + eys) * W + px];
            if constexpr (TH) P[((Q + a) * H + ey) * W + px] = bc(0.0f) - P[((Q + inv(a)) * H + eys) * W + px];
        }
    }
}

// Corrector output of the populations in M at tile pair-cell (tx, ty):
// f~^(n+1) = (f~ + Coll - dt/2 A[h^n]) - dt/2 A[h*].
template <typename S, bool TH, int BH, int BW, unsigned M>
__device__ __forceinline__ void corrector_write(const V2* sHs, const V2* sFC, int tx, int ty, int gx, int gy,
                                                const XPair& X, const YPair& Y, const StepArgs<float>& A) {
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr int NB = BW * BH;
    V2 adv[NQ];
    advect_region_mask<TH, BH, BW, M, 0>(sHs, tx + 1, ty + 2, X, Y, adv);
    const int kb = (ty + 2) * BW + tx + 1;
    const long long row = (long long)gy * A.pitch;
    const bool both = gx + 1 < A.nx;
    S* fout = static_cast<S*>(A.fout);
    S* gout = static_cast<S*>(A.gout);
#pragma unroll
    for (int a = 0; a < NQ; ++a) {
        if (!((M >> a) & 1u)) continue;
        const V2 o = fma2(bc(-A.hf), adv[a], sFC[a * NB + kb]);
        S* base = (a < Q ? fout + a * A.plane : gout + (a - Q) * A.plane) + row;
        if (both) PairIO<S>::st(base + gx, o);
        else Store<S>::st(base + gx, o.v.x);
    }
}

template <typename S, bool TH, int TX, int TY, int NTH>
__device__ __forceinline__ void ptile_body(const StepArgs<float>& A, const int x0, const int y0) {
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr int EW = (TX + 8) / 2, EH = TY + 8, NE = EW * EH;
    constexpr int BW = (TX + 4) / 2, BH = TY + 4, NB = BW * BH;
    constexpr int TW = TX / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2* sH = reinterpret_cast<V2*>(smem_raw);  // [NQ][EH][EW] h^n
    V2* sFC = sH + NQ * NE;                    // [NQ][BH][BW] f~ + Coll, then - dt/2 A[h^n]
    V2* sHs = sFC + NQ * NB;                   // [NQ][BH][BW] h*
    static_assert((NQ * (NE + 2 * NB)) % 2 == 0, "table copy must start 16-byte aligned");
    float4* sRow = reinterpret_cast<float4*>(sHs + NQ * NB);  // [BH][5] row entries of E2's rows
    float4* sCol = sRow + 5 * BH;                              // [BW][5] entries of E2's pair-columns
    const int nx = A.nx;
    const S* fin = static_cast<const S*>(A.fin);
    const S* gin = static_cast<const S*>(A.gin);

    // The row and column tables of region E2, copied before stage A so that
    // their loads overlap it; the barrier after stage A publishes them.
    for (int k = threadIdx.x; k < 5 * (BH + BW); k += NTH) {
        const int e = k / 5, part = k % 5;
        if (e < BH) {
            int gy;
            if (map_axis(y0 - 2 + e, A.ny, A.bcy, gy))
                sRow[k] = __ldg(reinterpret_cast<const float4*>(A.rowtab) + 5 * gy + part);
        } else {
            const int xu = x0 - 2 + 2 * (e - BH);
            const int gxl = ((xu % nx) + nx) % nx;
            sCol[(e - BH) * 5 + part] = __ldg(reinterpret_cast<const float4*>(A.coltab) + 5 * gxl + part);
        }
    }

    // ---- time level n on E4 ----
    for (int k = threadIdx.x; k < NE; k += NTH) {
        const int px = k % EW, ey = k / EW;
        int gy;
        if (!map_axis(y0 - 4 + ey, A.ny, A.bcy, gy)) continue;
        const int xu = x0 - 4 + 2 * px;
        const int gxl = ((xu % nx) + nx) % nx, gxr = ((xu + 1) % nx + nx) % nx;
        const bool contiguous = xu >= 0 && xu + 1 < nx;
        const long long row = (long long)gy * A.pitch;
        V2 d[Q], e[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const S* b = fin + a * A.plane + row;
            d[a] = contiguous ? PairIO<S>::ld(b + xu) : mk(Store<S>::ld(b + gxl), Store<S>::ld(b + gxr));
            if constexpr (TH) {
                const S* bg = gin + a * A.plane + row;
                e[a] = contiguous ? PairIO<S>::ld(bg + xu) : mk(Store<S>::ld(bg + gxl), Store<S>::ld(bg + gxr));
            }
        }
        const float4 o = __ldg(reinterpret_cast<const float4*>(A.rowtab + 20 * gy) + 3);
        PairMom<TH> c;
        c.build(d, e, A, o.y, TH ? o.z : 0.0f);
        const bool inB = px >= 1 && px < EW - 1 && ey >= 2 && ey < EH - 2;
        const int kb = (ey - 2) * BW + (px - 1);
        V2 hv[Q], hg[Q];
        c.relax_f(d, A, A.omh, A.hF, hv);
        if constexpr (TH) c.relax_g(e, A.omgh, hg);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            sH[a * NE + k] = hv[a];
            if constexpr (TH) sH[(Q + a) * NE + k] = hg[a];
        }
        if (inB) {
            V2 pv[Q], pg[Q];
            c.relax_f(d, A, A.om, A.cf, pv);
            if constexpr (TH) c.relax_g(e, A.omg, pg);
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                sFC[a * NB + kb] = pv[a];
                if constexpr (TH) sFC[(Q + a) * NB + kb] = pg[a];
            }
        }
    }
    __syncthreads();
    ghost_rows_region<TH, NQ, EH, EW>(sH, y0 - 4, A);
    __syncthreads();

    // ---- predictor on E2 ----
    for (int k = threadIdx.x; k < NB; k += NTH) {
        const int bx = k % BW, by = k / BW;
        int gy;
        if (!map_axis(y0 - 2 + by, A.ny, A.bcy, gy)) continue;
        XPair X;
        load_col_s(sCol + 5 * bx, X);
        YPair Y;
        load_row_s(sRow + 5 * by, Y);
        V2 adv[NQ];
        advect_region_all<TH, NQ, EH, EW, 0>(sH, bx + 1, by + 2, X, Y, adv);
        const bool tile = bx >= 1 && bx < BW - 1 && by >= 2 && by < BH - 2;
        V2 fs[Q], es[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const V2 fc = sFC[a * NB + k];
            fs[a] = fma2(bc(-A.dt), adv[a], fc);
            if (tile) sFC[a * NB + k] = fma2(bc(-A.hf), adv[a], fc);
            if constexpr (TH) {
                const V2 gc = sFC[(Q + a) * NB + k];
                es[a] = fma2(bc(-A.dt), adv[Q + a], gc);
                if (tile) sFC[(Q + a) * NB + k] = fma2(bc(-A.hf), adv[Q + a], gc);
            }
        }
        PairMom<TH> c;
        c.build(fs, es, A, Y.ro, TH ? Y.to : 0.0f);
        V2 hv[Q], hg[Q];
        c.relax_f(fs, A, A.omh, A.hF, hv);
        if constexpr (TH) c.relax_g(es, A.omgh, hg);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            sHs[a * NB + k] = hv[a];
            if constexpr (TH) sHs[(Q + a) * NB + k] = hg[a];
        }
    }
    __syncthreads();
    ghost_rows_region<TH, NQ, BH, BW>(sHs, y0 - 2, A);
    __syncthreads();

    // ---- corrector on the tile ----
    // With at least two threads per tile pair-cell the populations are split
    // between them: every corrector population is independent of the others.
    // Flow: {0, 1, 2, 5, 6} and {3, 4, 7, 8} (two axis and two diagonal
    // fluxes each); thermal: the nine f and the nine g.
    constexpr bool SPLIT = NTH >= 2 * TW * TY;
    constexpr unsigned ALL = (1u << NQ) - 1u;
    constexpr unsigned HALF0 = TH ? 0x1FFu : 0x67u;
    for (int k = threadIdx.x; k < (SPLIT ? 2 : 1) * TW * TY; k += NTH) {
        const int kp = SPLIT ? k % (TW * TY) : k;
        const int tx = kp % TW, ty = kp / TW;
        const int gx = x0 + 2 * tx, gy = y0 + ty;
        if (gx >= nx || gy >= A.ny) continue;
        XPair X;
        load_col_s(sCol + 5 * (tx + 1), X);
        YPair Y;
        load_row_s(sRow + 5 * (ty + 2), Y);
        if (!SPLIT) {
            corrector_write<S, TH, BH, BW, ALL>(sHs, sFC, tx, ty, gx, gy, X, Y, A);
        } else if (k < TW * TY) {
            corrector_write<S, TH, BH, BW, HALF0>(sHs, sFC, tx, ty, gx, gy, X, Y, A);
        } else {
            corrector_write<S, TH, BH, BW, ALL & ~HALF0>(sHs, sFC, tx, ty, gx, gy, X, Y, A);
        }
    }
}

template <typename S, bool TH, int TX, int TY, int NTH, int MINB>
__global__ void __launch_bounds__(NTH, MINB) k_fv_ptile(const StepArgs<float> A) {
    ptile_body<S, TH, TX, TY, NTH>(A, blockIdx.x * TX, blockIdx.y * TY);
}

// ---- split schedule: two kernels per step ----
// The fused tile recomputes the collision on tile + 4 and the predictor on
// tile + 2.  Here the first kernel computes the collision on tile + 2 and the
// predictor on the tile only, and hands h* and f~ + Coll - dt/2 A[h^n] to
// the second kernel through global memory (L2 on small grids); the second
// reads h* on tile + 2 and applies the corrector.  Halo work drops from
// 1.875x and 1.41x to 1.41x and 1x, and shared memory from three regions
// to one per kernel, at the price of a second launch and 72 B (144 B with
// g) per cell through L2.
template <typename S, bool TH, int TX, int TY, int NTH>
__global__ void __launch_bounds__(NTH) k_fv_split_a(const StepArgs<float> A) {
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr int BW = (TX + 4) / 2, BH = TY + 4, NB = BW * BH;
    constexpr int TW = TX / 2, NT = TW * TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2* sH = reinterpret_cast<V2*>(smem_raw);  // [NQ][BH][BW] h^n on tile + 2
    V2* sFC = sH + NQ * NB;                    // [NQ][TY][TW] f~ + Coll on the tile
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, nx = A.nx;
    const S* fin = static_cast<const S*>(A.fin);
    const S* gin = static_cast<const S*>(A.gin);
    for (int k = threadIdx.x; k < NB; k += NTH) {
        const int px = k % BW, ey = k / BW;
        int gy;
        if (!map_axis(y0 - 2 + ey, A.ny, A.bcy, gy)) continue;
        const int xu = x0 - 2 + 2 * px;
        const int gxl = ((xu % nx) + nx) % nx, gxr = ((xu + 1) % nx + nx) % nx;
        const bool contiguous = xu >= 0 && xu + 1 < nx;
        const long long row = (long long)gy * A.pitch;
        V2 d[Q], e[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const S* b = fin + a * A.plane + row;
            d[a] = contiguous ? PairIO<S>::ld(b + xu) : mk(Store<S>::ld(b + gxl), Store<S>::ld(b + gxr));
            if constexpr (TH) {
                const S* bg = gin + a * A.plane + row;
                e[a] = contiguous ? PairIO<S>::ld(bg + xu) : mk(Store<S>::ld(bg + gxl), Store<S>::ld(bg + gxr));
            }
        }
        const float4 o = __ldg(reinterpret_cast<const float4*>(A.rowtab + 20 * gy) + 3);
        PairMom<TH> c;
        c.build(d, e, A, o.y, TH ? o.z : 0.0f);
        const bool inT = px >= 1 && px < BW - 1 && ey >= 2 && ey < BH - 2;
        const int kt = (ey - 2) * TW + (px - 1);
        V2 hv[Q], hg[Q];
        c.relax_f(d, A, A.omh, A.hF, hv);
        if constexpr (TH) c.relax_g(e, A.omgh, hg);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            sH[a * NB + k] = hv[a];
            if constexpr (TH) sH[(Q + a) * NB + k] = hg[a];
        }
        if (inT) {
            V2 pv[Q], pg[Q];
            c.relax_f(d, A, A.om, A.cf, pv);
            if constexpr (TH) c.relax_g(e, A.omg, pg);
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                sFC[a * NT + kt] = pv[a];
                if constexpr (TH) sFC[(Q + a) * NT + kt] = pg[a];
            }
        }
    }
    __syncthreads();
    ghost_rows_region<TH, NQ, BH, BW>(sH, y0 - 2, A);
    __syncthreads();
    for (int k = threadIdx.x; k < NT; k += NTH) {
        const int tx = k % TW, ty = k / TW;
        const int gx = x0 + 2 * tx, gy = y0 + ty;
        if (gx >= nx || gy >= A.ny) continue;
        XPair X;
        load_col(A.coltab, gx, X);
        YPair Y;
        load_row(A.rowtab, gy, Y);
        V2 adv[NQ];
        advect_region_all<TH, NQ, BH, BW, 0>(sH, tx + 1, ty + 2, X, Y, adv);
        const long long at = (long long)gy * A.pitch + gx;
        const bool both = gx + 1 < nx;
        V2 fs[Q], es[Q];
#pragma unroll
        for (int a = 0; a < NQ; ++a) {
            const V2 fc = sFC[a * NT + k];
            const V2 fcb = fma2(bc(-A.hf), adv[a], fc);
            float* p = A.xfc + a * A.plane + at;
            if (both) PairIO<float>::st(p, fcb);
            else *p = fcb.v.x;
            const V2 st = fma2(bc(-A.dt), adv[a], fc);
            if (a < Q) fs[a] = st;
            else if constexpr (TH) es[a - Q] = st;
        }
        PairMom<TH> c;
        c.build(fs, es, A, Y.ro, TH ? Y.to : 0.0f);
        V2 hv[Q], hgv[Q];
        c.relax_f(fs, A, A.omh, A.hF, hv);
        if constexpr (TH) c.relax_g(es, A.omgh, hgv);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            float* p = A.xh + a * A.plane + at;
            if (both) PairIO<float>::st(p, hv[a]);
            else *p = hv[a].v.x;
            if constexpr (TH) {
                float* q = A.xh + (Q + a) * A.plane + at;
                if (both) PairIO<float>::st(q, hgv[a]);
                else *q = hgv[a].v.x;
            }
        }
    }
}

template <typename S, bool TH, int TX, int TY, int NTH>
__global__ void __launch_bounds__(NTH) k_fv_split_c(const StepArgs<float> A) {
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr int BW = (TX + 4) / 2, BH = TY + 4, NB = BW * BH;
    constexpr int TW = TX / 2, NT = TW * TY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2* sHs = reinterpret_cast<V2*>(smem_raw);  // [NQ][BH][BW] h* on tile + 2
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, nx = A.nx;
    for (int k = threadIdx.x; k < NB; k += NTH) {
        const int px = k % BW, ey = k / BW;
        int gy;
        if (!map_axis(y0 - 2 + ey, A.ny, A.bcy, gy)) continue;
        const int xu = x0 - 2 + 2 * px;
        const int gxl = ((xu % nx) + nx) % nx, gxr = ((xu + 1) % nx + nx) % nx;
        const bool contiguous = xu >= 0 && xu + 1 < nx;
        const long long row = (long long)gy * A.pitch;
#pragma unroll
        for (int a = 0; a < NQ; ++a) {
            const float* b = A.xh + a * A.plane + row;
            sHs[a * NB + k] = contiguous ? PairIO<float>::ld(b + xu) : mk(__ldg(b + gxl), __ldg(b + gxr));
        }
    }
    __syncthreads();
    ghost_rows_region<TH, NQ, BH, BW>(sHs, y0 - 2, A);
    __syncthreads();
    S* fout = static_cast<S*>(A.fout);
    S* gout = static_cast<S*>(A.gout);
    for (int k = threadIdx.x; k < NT; k += NTH) {
        const int tx = k % TW, ty = k / TW;
        const int gx = x0 + 2 * tx, gy = y0 + ty;
        if (gx >= nx || gy >= A.ny) continue;
        XPair X;
        load_col(A.coltab, gx, X);
        YPair Y;
        load_row(A.rowtab, gy, Y);
        V2 adv[NQ];
        advect_region_all<TH, NQ, BH, BW, 0>(sHs, tx + 1, ty + 2, X, Y, adv);
        const long long at = (long long)gy * A.pitch + gx;
        const bool both = gx + 1 < nx;
#pragma unroll
        for (int a = 0; a < NQ; ++a) {
            const float* p = A.xfc + a * A.plane + at;
            const V2 fcb = both ? PairIO<float>::ld(p) : mk(__ldg(p), 0.0f);
            const V2 o = fma2(bc(-A.hf), adv[a], fcb);
            S* base = (a < Q ? fout + a * A.plane : gout + (a - Q) * A.plane) + at;
            if (both) PairIO<S>::st(base, o);
            else Store<S>::st(base, o.v.x);
        }
    }
}

template <typename S, bool TH, int TX, int TY, int NTH>
static cudaError_t run_split(const void* vargs, cudaStream_t s) {
    const StepArgs<float>& A = *static_cast<const StepArgs<float>*>(vargs);
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr size_t smem_a = sizeof(V2) * NQ * (((TX + 4) / 2) * (TY + 4) + (TX / 2) * TY);
    constexpr size_t smem_c = sizeof(V2) * NQ * ((TX + 4) / 2) * (TY + 4);
    static_assert(smem_a <= 232448, "shared memory per CTA");
    {
        cudaError_t e = set_max_smem((const void*)k_fv_split_a<S, TH, TX, TY, NTH>, (int)smem_a);
        if (e == cudaSuccess) e = set_max_smem((const void*)k_fv_split_c<S, TH, TX, TY, NTH>, (int)smem_c);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((A.nx + TX - 1) / TX, (A.ny + TY - 1) / TY);
    k_fv_split_a<S, TH, TX, TY, NTH><<<grid, NTH, smem_a, s>>>(A);
    count_launch();
    k_fv_split_c<S, TH, TX, TY, NTH><<<grid, NTH, smem_c, s>>>(A);
    count_launch();
    return cudaGetLastError();
}

template <typename S, bool TH>
static cudaError_t run_split_shape(const void* args, int shape, cudaStream_t s) {
    if (shape == 16) return run_split<S, TH, 16, 16, 128>(args, s);
    return run_split<S, TH, 32, 16, 256>(args, s);
}

cudaError_t launch_fv_split(Prec p, bool th, const void* args, int shape, cudaStream_t s) {
    switch (p) {
        case Prec::F32:
            return th ? run_split_shape<float, true>(args, shape, s) : run_split_shape<float, false>(args, shape, s);
        case Prec::F16:
            return th ? run_split_shape<__half, true>(args, shape, s) : run_split_shape<__half, false>(args, shape, s);
        case Prec::BF16:
            return th ? run_split_shape<__nv_bfloat16, true>(args, shape, s)
                      : run_split_shape<__nv_bfloat16, false>(args, shape, s);
        default: return cudaErrorInvalidValue;
    }
}

// Many grids in one launch (the serving path): CTA b steps tile tiles[b] =
// (request, tile x, tile y) with that request's parameters, picking its
// input buffer from step k of the launch sequence; requests with fewer than
// k + 1 steps left are skipped.  Same tile code whatever else is batched.
template <typename S, bool TH, int TX, int TY, int NTH>
__global__ void __launch_bounds__(NTH)
k_fv_ptile_batched(const BatchReq<float>* reqs, const int4* tiles, const int* ntiles, const int k) {
    if ((int)blockIdx.x >= *ntiles) return;
    const int4 t = tiles[blockIdx.x];
    const BatchReq<float>& B = reqs[t.x];
    if (k >= B.remaining) return;
    StepArgs<float> A = B.args;
    const int p = (B.parity + k) & 1;
    A.fin = B.f[p];
    A.fout = B.f[p ^ 1];
    A.gin = B.g[p];
    A.gout = B.g[p ^ 1];
    ptile_body<S, TH, TX, TY, NTH>(A, t.y * TX, t.z * TY);
}

// Thermal tiles use 512 threads (one CTA per SM by shared memory; the
// corrector splits f and g over two threads per pair-cell), flow tiles 256.
template <typename S, bool TH>
static cudaError_t run_ptile_batched(const void* reqs, const int4* tiles, const int* ntiles, int capacity, int k,
                                     cudaStream_t s) {
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr int NTH = TH ? 512 : 256;
    constexpr size_t smem = sizeof(V2) * NQ * (((32 + 8) / 2) * (16 + 8) + 2 * ((32 + 4) / 2) * (16 + 4)) +
                            sizeof(float) * ptile_tab_floats(32, 16);
    {
        cudaError_t e = set_max_smem((const void*)k_fv_ptile_batched<S, TH, 32, 16, NTH>, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_fv_ptile_batched<S, TH, 32, 16, NTH><<<capacity, NTH, smem, s>>>(static_cast<const BatchReq<float>*>(reqs),
                                                                      tiles, ntiles, k);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fv_ptile_batched(Prec p, bool th, const void* reqs, const int4* tiles, const int* ntiles,
                                    int capacity, int k, cudaStream_t s) {
    switch (p) {
        case Prec::F32:
            return th ? run_ptile_batched<float, true>(reqs, tiles, ntiles, capacity, k, s)
                      : run_ptile_batched<float, false>(reqs, tiles, ntiles, capacity, k, s);
        case Prec::F16:
            return th ? run_ptile_batched<__half, true>(reqs, tiles, ntiles, capacity, k, s)
                      : run_ptile_batched<__half, false>(reqs, tiles, ntiles, capacity, k, s);
        case Prec::BF16:
            return th ? run_ptile_batched<__nv_bfloat16, true>(reqs, tiles, ntiles, capacity, k, s)
                      : run_ptile_batched<__nv_bfloat16, false>(reqs, tiles, ntiles, capacity, k, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename S, bool TH, int TX, int TY, int NTH, int MINB>
static cudaError_t run_ptile(const void* vargs, cudaStream_t s) {
    const StepArgs<float>& A = *static_cast<const StepArgs<float>*>(vargs);
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr size_t smem = sizeof(V2) * NQ * (((TX + 8) / 2) * (TY + 8) + 2 * ((TX + 4) / 2) * (TY + 4)) +
                            sizeof(float) * ptile_tab_floats(TX, TY);
    static_assert(smem <= 232448, "shared memory per CTA");
    {
        cudaError_t e = set_max_smem((const void*)k_fv_ptile<S, TH, TX, TY, NTH, MINB>, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((A.nx + TX - 1) / TX, (A.ny + TY - 1) / TY);
    k_fv_ptile<S, TH, TX, TY, NTH, MINB><<<grid, NTH, smem, s>>>(A);
    count_launch();
    return cudaGetLastError();
}

// shape: 0 = 32 x 16 tiles, 256 threads; 14 = 32 x 14, 256 threads;
// 16 = 16 x 16, 128 threads; 512 = 32 x 16, 512 threads; 526 = 32 x 14,
// 512 threads.  The 14-row tiles let a 512-row grid fill two CTAs on
// nearly every SM (296 tiles for 256 columns) instead of 256 tiles on 152.
template <typename S, bool TH>
static cudaError_t run_ptile_shape(const void* args, int shape, cudaStream_t s) {
    if (shape == 16) return run_ptile<S, TH, 16, 16, 128, 1>(args, s);
    if (shape == 14) return run_ptile<S, TH, 32, 14, 256, 1>(args, s);
    if (shape == 512) return run_ptile<S, TH, 32, 16, 512, TH ? 1 : 2>(args, s);
    if (shape == 526) return run_ptile<S, TH, 32, 14, 512, TH ? 1 : 2>(args, s);
    return run_ptile<S, TH, 32, 16, 256, 1>(args, s);
}

cudaError_t launch_fv_ptile(Prec p, bool th, const void* args, int shape, cudaStream_t s) {
    switch (p) {
        case Prec::F32:
            return th ? run_ptile_shape<float, true>(args, shape, s) : run_ptile_shape<float, false>(args, shape, s);
        case Prec::F16:
            return th ? run_ptile_shape<__half, true>(args, shape, s) : run_ptile_shape<__half, false>(args, shape, s);
        case Prec::BF16:
            return th ? run_ptile_shape<__nv_bfloat16, true>(args, shape, s)
                      : run_ptile_shape<__nv_bfloat16, false>(args, shape, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename S, bool TH, int NT>
static cudaError_t run_pair(const void* vargs, int chunk, cudaStream_t s) {
    const StepArgs<float>& A = *static_cast<const StepArgs<float>*>(vargs);
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr size_t smem = sizeof(V2) * (2 * ring_off(NQ) + 5 * NQ) * NT;
    static_assert(smem <= 232448, "shared memory per CTA");
    {
        cudaError_t e = set_max_smem((const void*)k_fv_pair<S, TH, NT>, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int ch = chunk < 8 ? 8 : chunk;
    constexpr int W = 2 * NT - 8;
    dim3 grid((A.nx + W - 1) / W, (A.ny + ch - 1) / ch);
    k_fv_pair<S, TH, NT><<<grid, NT, smem, s>>>(A, ch);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fv_pair(Prec p, bool th, const void* args, int chunk, cudaStream_t s) {
    switch (p) {
        case Prec::F32: return th ? run_pair<float, true, 56>(args, chunk, s) : run_pair<float, false, 56>(args, chunk, s);
        case Prec::F16: return th ? run_pair<__half, true, 56>(args, chunk, s) : run_pair<__half, false, 56>(args, chunk, s);
        case Prec::BF16:
            return th ? run_pair<__nv_bfloat16, true, 56>(args, chunk, s)
                      : run_pair<__nv_bfloat16, false, 56>(args, chunk, s);
        default: return cudaErrorInvalidValue;
    }
}

// 56 threads per strip: with the rings above, four strips fit one SM (52 KB each)
int pair_width() { return 2 * 56 - 8; }

size_t pair_smem(bool th) { return sizeof(float2) * (2 * ring_off(th ? 18 : 9) + 5 * (th ? 18 : 9)) * 56; }

}  // namespace lbgb
