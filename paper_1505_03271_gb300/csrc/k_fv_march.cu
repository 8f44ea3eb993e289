// k_fv_march.cu -- the FV time step (Sec. II B: Eqs. (semi), (semi-heun),
// QUICK faces of Sec. II B 3, double-reflection walls of Sec. II B 5) as a
// y-marching strip kernel.
//
// A CTA owns NT consecutive columns (one per thread) and marches up a chunk
// of rows.  At row iteration t it runs three stages, each on one row:
//   A(t):   load f~^n of row t (prefetched one iteration ahead), form
//           h^n and f~ + Coll^n                      (all NT columns)
//   B(t-2): f~* = f~ + Coll - dt A[h^n], then h*;   keep f~ + Coll - dt/2 A[h^n]
//                                                     (NT - 4 columns)
//   C(t-4): f~^(n+1) = f~ + Coll - dt/2 (A[h^n] + A[h*])  (NT - 8 columns)
// Rows live in 5-slot rings in shared memory (slot = row mod 5), which is
// exactly what the +-2 QUICK stencil in y needs.  Only x neighbours are read
// across threads, and every cross-thread read is at least two iterations
// after the write, so one barrier per row suffices.  The halo is
// recomputed only in x: (NT)/(NT - 8) for stage A, (NT - 4)/(NT - 8) for B.
// Each thread keeps the QUICK weights of its own two x faces in registers.
#include "lb_internal.cuh"

namespace lbgb {

namespace {

template <typename R>
struct XMetric {  // the thread's column: faces gx (west) and gx + 1 (east)
    R pw[3], pe[3], mw[3], me[3], inv;
};
template <typename R>
struct YMetric {  // one row: faces gy (south) and gy + 1 (north)
    R ps[3], pn[3], ms[3], mn[3], inv;
};

template <typename R>
__device__ __forceinline__ void load_x(const AxisMetric<R>& m, int g, XMetric<R>& X) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        X.pw[r] = m.wp(r, g);
        X.pe[r] = m.wp(r, g + 1);
        X.mw[r] = m.wm(r, g);
        X.me[r] = m.wm(r, g + 1);
    }
    X.inv = m.invd(g);
}

template <typename R>
__device__ __forceinline__ void load_y(const AxisMetric<R>& m, int g, YMetric<R>& Y) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        Y.ps[r] = m.wp(r, g);
        Y.pn[r] = m.wp(r, g + 1);
        Y.ms[r] = m.wm(r, g);
        Y.mn[r] = m.wm(r, g + 1);
    }
    Y.inv = m.invd(g);
}

__device__ __forceinline__ int slot5(int r) {
    const int s = r % 5;
    return s < 0 ? s + 5 : s;
}

// Flux divergence of plane p (population a = p mod 9) at column k of the
// ring's middle row; rows r-2..r+2 are in slots sl[0..4].
template <typename R, int NQ, int NT, int a>
__device__ __forceinline__ R advect_col(const R* ring, const int* sl, int p, int k,
                                        const XMetric<R>& X, const YMetric<R>& Y) {
    R v = 0;
    const R* row = ring + (sl[2] * NQ + p) * NT;
    if constexpr (cx(a) > 0) {
        const R pe = X.pe[0] * row[k - 1] + X.pe[1] * row[k] + X.pe[2] * row[k + 1];
        const R pw = X.pw[0] * row[k - 2] + X.pw[1] * row[k - 1] + X.pw[2] * row[k];
        v += (pe - pw) * X.inv;
    } else if constexpr (cx(a) < 0) {
        const R pe = X.me[0] * row[k] + X.me[1] * row[k + 1] + X.me[2] * row[k + 2];
        const R pw = X.mw[0] * row[k - 1] + X.mw[1] * row[k] + X.mw[2] * row[k + 1];
        v -= (pe - pw) * X.inv;
    }
    if constexpr (cy(a) != 0) {
        R c[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) c[i] = ring[(sl[i] * NQ + p) * NT + k];
        if constexpr (cy(a) > 0) {
            const R pn = Y.pn[0] * c[1] + Y.pn[1] * c[2] + Y.pn[2] * c[3];
            const R ps = Y.ps[0] * c[0] + Y.ps[1] * c[1] + Y.ps[2] * c[2];
            v += (pn - ps) * Y.inv;
        } else {
            const R pn = Y.mn[0] * c[2] + Y.mn[1] * c[3] + Y.mn[2] * c[4];
            const R ps = Y.ms[0] * c[1] + Y.ms[1] * c[2] + Y.ms[2] * c[3];
            v -= (pn - ps) * Y.inv;
        }
    }
    return v;
}

// All populations: the deviations' flux divergence plus the base state's
// own y flux (a per-row constant).
template <typename R, bool TH, int NQ, int NT, int a>
__device__ __forceinline__ void advect_all(const R* ring, const int* sl, int k, const XMetric<R>& X,
                                           const YMetric<R>& Y, const StepArgs<R>& A, int gy, R* out) {
    out[a] = advect_col<R, NQ, NT, a>(ring, sl, a, k, X, Y) + ref_flux<R, a>(A, gy, false);
    if constexpr (TH) out[Q + a] = advect_col<R, NQ, NT, a>(ring, sl, Q + a, k, X, Y) + ref_flux<R, a>(A, gy, true);
    if constexpr (a + 1 < Q) advect_all<R, TH, NQ, NT, a + 1>(ring, sl, k, X, Y, A, gy, out);
}

// Ghost row of a wall on y, own column, on base-state deviations: double
// reflection h'_a = h'_inv(a) for f, anti-reflection h'_a = -h'_inv(a) for g.
template <typename R, bool TH, int NQ, int NT>
__device__ __forceinline__ void ghost_row(R* ring, int dst_slot, int src_slot, int k) {
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        ring[(dst_slot * NQ + a) * NT + k] = ring[(src_slot * NQ + inv(a)) * NT + k];
        if constexpr (TH) ring[(dst_slot * NQ + Q + a) * NT + k] = -ring[(src_slot * NQ + Q + inv(a)) * NT + k];
    }
}

}  // namespace

template <typename R, typename S, bool TH, int NT>
__global__ void __launch_bounds__(NT) k_fv_march(const StepArgs<R> A, const int CH) {
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr int W = NT - 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sH = reinterpret_cast<R*>(smem_raw);  // [5][NQ][NT] h^n
    R* sP = sH + 5 * NQ * NT;                // [5][NQ][NT] f~ + Coll (then - dt/2 A[h^n]), own column
    R* sS = sP + 5 * NQ * NT;                // [5][NQ][NT] h*
    const int k = threadIdx.x;
    const int xu = blockIdx.x * W - 4 + k;  // unwrapped column
    const int ys = blockIdx.y * CH;
    const int ye = min(ys + CH, A.ny);
    int gx = 0;
    const bool colA = map_axis(xu, A.nx, A.bcx, gx);
    const bool colB = colA && k >= 2 && k < NT - 2;
    const bool colC = colA && k >= 4 && k < NT - 4 && xu < A.nx;
    const bool wally = A.bcy == LB_BC_WALLS;
    // x-wall ghost column: its mirror column inside the strip
    int kmir = -1;
    if (!colA && A.bcx == LB_BC_WALLS) {
        if (xu == -1 || xu == -2) kmir = k + (-xu - 1 - xu);
        else if (xu == A.nx || xu == A.nx + 1) kmir = k - (2 * (xu - A.nx) + 1);
        if (kmir < 0 || kmir >= NT) kmir = -1;
    }
    XMetric<R> X;
    if (colB) load_x(A.mx, gx, X);

    const S* fin = static_cast<const S*>(A.fin);
    const S* gin = static_cast<const S*>(A.gin);
    S* fout = static_cast<S*>(A.fout);
    S* gout = static_cast<S*>(A.gout);

    // rows of the march: A on [ys-4, ye+4), B on [ys-2, ye+2), C on [ys, ye)
    auto fluid_row = [&](int r, int& gy) { return map_axis(r, A.ny, A.bcy, gy); };
    R nd[Q], ne[Q];  // prefetched populations of the next A row
    auto prefetch = [&](int r) {
        int gy;
        if (colA && r < ye + 4 && fluid_row(r, gy)) {
            const long long c = (long long)gy * A.pitch + gx;
#pragma unroll
            for (int a = 0; a < Q; ++a) nd[a] = Store<S>::ld(fin + a * A.plane + c);
            if constexpr (TH) {
#pragma unroll
                for (int a = 0; a < Q; ++a) ne[a] = Store<S>::ld(gin + a * A.plane + c);
            }
        }
    };
    prefetch(ys - 4);

    for (int t = ys - 4; t < ye + 4; ++t) {
        // x-wall ghost columns of the rows finished one iteration ago
        if (kmir >= 0) {
            const int rh = t - 1, rs = t - 3;
            int gy;
            if (rh >= ys - 4 && fluid_row(rh, gy)) {
                const int s = slot5(rh);
#pragma unroll
                for (int a = 0; a < Q; ++a) sH[(s * NQ + a) * NT + k] = sH[(s * NQ + inv(a)) * NT + kmir];
            }
            if (rs >= ys - 2 && rs < ye + 2 && fluid_row(rs, gy)) {
                const int s = slot5(rs);
#pragma unroll
                for (int a = 0; a < Q; ++a) sS[(s * NQ + a) * NT + k] = sS[(s * NQ + inv(a)) * NT + kmir];
            }
        }
        // ---- stage A on row t ----
        {
            int gy;
            const int s = slot5(t);
            if (fluid_row(t, gy)) {
                if (colA) {
                    R d[Q], e[Q];
#pragma unroll
                    for (int a = 0; a < Q; ++a) {
                        d[a] = nd[a];
                        if constexpr (TH) e[a] = ne[a];
                    }
                    prefetch(t + 1);
                    Cell<R, TH> m;
                    m.moments(d, e, A, A.roff[gy], A.toff[gy]);
#pragma unroll
                    for (int a = 0; a < Q; ++a) {
                        R feqd, F, geqd = 0;
                        m.eq(a, A, feqd, F, geqd);
                        const R neq = feqd - d[a];
                        sH[(s * NQ + a) * NT + k] = d[a] + A.omh * neq + A.hF * F;
                        sP[(s * NQ + a) * NT + k] = d[a] + A.om * neq + A.cf * F;
                        if constexpr (TH) {
                            const R neqg = geqd - e[a];
                            sH[(s * NQ + Q + a) * NT + k] = e[a] + A.omgh * neqg;
                            sP[(s * NQ + Q + a) * NT + k] = e[a] + A.omg * neqg;
                        }
                    }
                }
            } else {
                prefetch(t + 1);
                // top wall ghosts at their own iteration; bottom ones below
                if (wally && colA && (t == A.ny || t == A.ny + 1))
                    ghost_row<R, TH, NQ, NT>(sH, s, slot5(2 * A.ny - 1 - t), k);
            }
            if (wally && colA && t == 1 && ys == 0) {
                ghost_row<R, TH, NQ, NT>(sH, slot5(-1), slot5(0), k);
                ghost_row<R, TH, NQ, NT>(sH, slot5(-2), slot5(1), k);
            }
        }
        // ---- stage B on row t - 2 ----
        {
            const int r = t - 2;
            int gy;
            if (r >= ys - 2 && r < ye + 2) {
                const int s = slot5(r);
                if (fluid_row(r, gy)) {
                    if (colB) {
                        YMetric<R> Y;
                        load_y(A.my, gy, Y);
                        const int sl[5] = {slot5(r - 2), slot5(r - 1), s, slot5(r + 1), slot5(r + 2)};
                        R adv[NQ];
                        advect_all<R, TH, NQ, NT, 0>(sH, sl, k, X, Y, A, gy, adv);
                        R fs[Q], es[Q];
#pragma unroll
                        for (int a = 0; a < Q; ++a) {
                            const R fc = sP[(s * NQ + a) * NT + k];
                            fs[a] = fc - A.dt * adv[a];
                            sP[(s * NQ + a) * NT + k] = fc - A.hf * adv[a];
                            if constexpr (TH) {
                                const R gc = sP[(s * NQ + Q + a) * NT + k];
                                es[a] = gc - A.dt * adv[Q + a];
                                sP[(s * NQ + Q + a) * NT + k] = gc - A.hf * adv[Q + a];
                            }
                        }
                        Cell<R, TH> m;
                        m.moments(fs, es, A, A.roff[gy], A.toff[gy]);
#pragma unroll
                        for (int a = 0; a < Q; ++a) {
                            R feqd, F, geqd = 0;
                            m.eq(a, A, feqd, F, geqd);
                            sS[(s * NQ + a) * NT + k] = fs[a] + A.omh * (feqd - fs[a]) + A.hF * F;
                            if constexpr (TH) sS[(s * NQ + Q + a) * NT + k] = es[a] + A.omgh * (geqd - es[a]);
                        }
                    }
                } else if (wally && colA && (r == A.ny || r == A.ny + 1)) {
                    ghost_row<R, TH, NQ, NT>(sS, s, slot5(2 * A.ny - 1 - r), k);
                }
                if (wally && colA && r == 1 && ys == 0) {
                    ghost_row<R, TH, NQ, NT>(sS, slot5(-1), slot5(0), k);
                    ghost_row<R, TH, NQ, NT>(sS, slot5(-2), slot5(1), k);
                }
            }
        }
        // ---- stage C on row t - 4 ----
        {
            const int r = t - 4;
            if (r >= ys && r < ye && colC) {
                const int s = slot5(r);
                YMetric<R> Y;
                load_y(A.my, r, Y);
                const int sl[5] = {slot5(r - 2), slot5(r - 1), s, slot5(r + 1), slot5(r + 2)};
                R adv[NQ];
                advect_all<R, TH, NQ, NT, 0>(sS, sl, k, X, Y, A, r, adv);
                const long long c = (long long)r * A.pitch + gx;
#pragma unroll
                for (int a = 0; a < Q; ++a)
                    Store<S>::st(fout + a * A.plane + c, sP[(s * NQ + a) * NT + k] - A.hf * adv[a]);
                if constexpr (TH) {
#pragma unroll
                    for (int a = 0; a < Q; ++a)
                        Store<S>::st(gout + a * A.plane + c, sP[(s * NQ + Q + a) * NT + k] - A.hf * adv[Q + a]);
                }
            }
        }
        __syncthreads();
    }
}

template <typename R, typename S, bool TH, int NT>
static cudaError_t run_march(const void* vargs, int chunk, cudaStream_t s) {
    const StepArgs<R>& A = *static_cast<const StepArgs<R>*>(vargs);
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr size_t smem = sizeof(R) * 15 * NQ * NT;
    static_assert(smem <= 232448, "shared memory per CTA");
    {
        cudaError_t e = set_max_smem((const void*)k_fv_march<R, S, TH, NT>, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int ch = chunk < 8 ? 8 : chunk;
    dim3 grid((A.nx + (NT - 8) - 1) / (NT - 8), (A.ny + ch - 1) / ch);
    k_fv_march<R, S, TH, NT><<<grid, NT, smem, s>>>(A, ch);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fv_march(Prec p, bool th, const void* args, int chunk, cudaStream_t s) {
    switch (p) {
        case Prec::F64:
            return th ? run_march<double, double, true, 64>(args, chunk, s)
                      : run_march<double, double, false, 128>(args, chunk, s);
        case Prec::F32:
            return th ? run_march<float, float, true, 128>(args, chunk, s)
                      : run_march<float, float, false, 128>(args, chunk, s);
        case Prec::F16:
            return th ? run_march<float, __half, true, 128>(args, chunk, s)
                      : run_march<float, __half, false, 128>(args, chunk, s);
        case Prec::BF16:
            return th ? run_march<float, __nv_bfloat16, true, 128>(args, chunk, s)
                      : run_march<float, __nv_bfloat16, false, 128>(args, chunk, s);
    }
    return cudaErrorInvalidValue;
}

int march_width(Prec p, bool th) { return (p == Prec::F64 && th) ? 56 : 120; }

size_t march_smem(Prec p, bool th) {
    const size_t r = p == Prec::F64 ? 8 : 4;
    const size_t nt = (p == Prec::F64 && th) ? 64 : 128;
    return r * 15 * (th ? 18 : 9) * nt;
}

}  // namespace lbgb
