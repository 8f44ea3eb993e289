// k3.cu -- the D3Q19 (three-dimensional) time steps of Sec. II and the
// observables' kernels.
//
// ST, Eq. (ST): one fused collide-and-push kernel, one thread per cell;
// half-way bounce-back at walls, anti-bounce-back of g at the z plates.
//
// FV, Eqs. (semi) and (semi-heun): three passes over the grid, each a plain
// per-cell kernel, with the intermediate fields in HBM:
//   k3_pre   f~ -> h^n and f~ + Coll^n                       (local)
//   k3_mid   A[h^n] (QUICK on the cross stencil, ghosts formed on the fly)
//            -> f~* = f~ + Coll - dt A, h*, and f~ + Coll - dt/2 A
//   k3_post  A[h*] -> f~^(n+1) = f~ + Coll - dt/2 (A[h^n] + A[h*])
// A fused 3-D tile would recompute a 4-cell halo on all six faces, or hold
// 19 (38) populations of several halo planes in shared memory; three passes
// recompute nothing and move 5x the compulsory bytes, which keeps the step
// on the HBM roof.  Faces are taken dimension by dimension from the nodes of
// their own grid line (Sec. II B 3), so only face ghosts are ever read.
#include "lb3.cuh"

namespace lbgb {

namespace {

__host__ __device__ inline long long cell3(const int* n, int i, int j, int k) {
    return ((long long)k * n[1] + j) * n[0] + i;
}

// Moments and equilibria of one cell from deviations d = f - w, e = g - w T0:
// rho = 1 + sum d, T = T0 + sum e, a_z += beta g (T - T0),
// u = sum c d / rho + hf a (hf = dt/2 for tilded populations).
template <typename R, bool TH>
struct Cell3 {
    R rp, rho, ux, uy, uz, Td, T, az;
    __device__ __forceinline__ void moments(const R* d, const R* e, const Args3<R>& A) {
        R r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int a = 0; a < Q3; ++a) {
            r += d[a];
            jx += R(c3x(a)) * d[a];
            jy += R(c3y(a)) * d[a];
            jz += R(c3z(a)) * d[a];
        }
        Td = 0;
        if constexpr (TH) {
#pragma unroll
            for (int a = 0; a < Q3; ++a) Td += e[a];
        }
        rp = r;
        rho = R(1) + r;
        T = A.T0 + Td;
        az = A.az + (TH ? A.bg * Td : R(0));
        const R ir = R(1) / rho;
        ux = jx * ir + A.hf * A.ax;
        uy = jy * ir + A.hf * A.ay;
        uz = jz * ir + A.hf * az;
    }
    // the same from the sums sum d, sum c d (3) and sum e
    __device__ __forceinline__ void from_sums(R r, R jx, R jy, R jz, R td, const Args3<R>& A) {
        Td = TH ? td : R(0);
        rp = r;
        rho = R(1) + r;
        T = A.T0 + Td;
        az = A.az + (TH ? A.bg * Td : R(0));
        const R ir = R(1) / rho;
        ux = jx * ir + A.hf * A.ax;
        uy = jy * ir + A.hf * A.ay;
        uz = jz * ir + A.hf * az;
    }
    // f_eq - w, Guo force F (Eq. (F2)) and g_eq - w T0
    __device__ __forceinline__ void eq(int a, const Args3<R>& A, R& feqd, R& F, R& geqd) const {
        const R w = w3<R>(a);
        const R cxa = R(c3comp(a, 0)), cya = R(c3comp(a, 1)), cza = R(c3comp(a, 2));
        const R cu = cxa * ux + cya * uy + cza * uz;
        const R uu = ux * ux + uy * uy + uz * uz;
        const R poly = R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu;
        feqd = w * (rp + rho * poly);
        const R ca = cxa * A.ax + cya * A.ay + cza * az;
        const R ua = ux * A.ax + uy * A.ay + uz * az;
        F = w * rho * (R(3) * (ca - ua) + R(9) * cu * ca);
        geqd = TH ? w * (Td + T * poly) : R(0);
    }
};

template <typename S, typename R>
__device__ __forceinline__ void load19(const void* src, long long N, long long c, R* d) {
    const S* p = static_cast<const S*>(src);
#pragma unroll
    for (int a = 0; a < Q3; ++a) d[a] = (R)Store<S>::ld(p + a * N + c);
}

// Advected-field value of population a at (i, j, k), where at most one
// index lies outside the grid: periodic axes wrap, walls mirror the node and
// reflect the population, h_a(ghost) = h_inv(a)(node) (Sec. II B 5); the
// thermal field is anti-reflected at the z plates,
// hg'_a(ghost) = 2 w_a (T_wall - T0) - hg'_inv(a)(node).
template <typename R, bool G>
__device__ __forceinline__ R hval(const R* P, int a, int i, int j, int k, const Args3<R>& A) {
    int idx[3] = {i, j, k};
    int b = a;
    bool flip = false;
    R wallv = 0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const int n = A.n[ax];
        if (idx[ax] >= 0 && idx[ax] < n) continue;
        if (A.bc[ax] == LB_BC_PERIODIC) {
            idx[ax] = ((idx[ax] % n) + n) % n;  // axes of 1 or 2 cells wrap more than once
        } else {
            const bool lo = idx[ax] < 0;
            idx[ax] = lo ? -idx[ax] - 1 : 2 * n - 1 - idx[ax];
            b = inv3(a);
            if (G) {
                flip = true;
                wallv = R(2) * w3<R>(a) * (lo ? A.dTb : A.dTt);
            }
        }
    }
    const R v = __ldg(P + (long long)b * A.N + cell3(A.n, idx[0], idx[1], idx[2]));
    return flip ? wallv - v : v;
}

// Flux divergence of population a at (i, j, k), Eq. (fv): for each axis
// with c != 0, c (Phi_+ - Phi_-) / width with QUICK faces.
template <typename R, bool G, int a>
__device__ __forceinline__ R advect3(const R* P, int i, int j, int k, const Args3<R>& A) {
    R v = 0;
    const int cc[3] = {c3x(a), c3y(a), c3z(a)};
    const int pos[3] = {i, j, k};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (cc[ax] == 0) continue;
        const int m = pos[ax];
        R h[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int id[3] = {i, j, k};
            id[ax] = m + s + (cc[ax] > 0 ? -2 : -1);
            h[s] = hval<R, G>(P, a, id[0], id[1], id[2], A);
        }
        const AxisMetric<R>& M = A.m[ax];
        if (cc[ax] > 0) {
            const R pw = M.wp(0, m) * h[0] + M.wp(1, m) * h[1] + M.wp(2, m) * h[2];
            const R pe = M.wp(0, m + 1) * h[1] + M.wp(1, m + 1) * h[2] + M.wp(2, m + 1) * h[3];
            v += (pe - pw) * M.invd(m);
        } else {
            const R pw = M.wm(0, m) * h[0] + M.wm(1, m) * h[1] + M.wm(2, m) * h[2];
            const R pe = M.wm(0, m + 1) * h[1] + M.wm(1, m + 1) * h[2] + M.wm(2, m + 1) * h[3];
            v -= (pe - pw) * M.invd(m);
        }
    }
    return v;
}

template <typename R, bool G, int a>
__device__ __forceinline__ void advect_all(const R* P, int i, int j, int k, const Args3<R>& A, R* out) {
    out[a] = advect3<R, G, a>(P, i, j, k, A);
    if constexpr (a + 1 < Q3) advect_all<R, G, a + 1>(P, i, j, k, A, out);
}


// Offsets (in cells) of the stencil nodes s = -2..2 along each axis,
// wrapped once on periodic axes.  `inside` is false when a node falls past
// a wall, i.e. when the ghost rules are needed.
struct Nbr3 {
    int off[3][5];
    bool inside;
};

__device__ __forceinline__ Nbr3 neighbours3(const int* n, const int* bc, int i, int j, int k) {
    Nbr3 nb;
    nb.inside = true;
    const int pos[3] = {i, j, k};
    const int stride[3] = {1, n[0], n[0] * n[1]};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
#pragma unroll
        for (int s = -2; s <= 2; ++s) {
            int p = pos[ax] + s;
            if (p < 0 || p >= n[ax]) {
                if (bc[ax] == LB_BC_PERIODIC) {
                    p = ((p % n[ax]) + n[ax]) % n[ax];
                } else {
                    nb.inside = false;
                    p = pos[ax];
                }
            }
            nb.off[ax][s + 2] = (p - pos[ax]) * stride[ax];
        }
    }
    return nb;
}

// Flux divergence of population a from in-grid nodes only (Eq. (fv)).
template <typename R, int a>
__device__ __forceinline__ R advect3_in(const R* P, long long c, const Nbr3& nb, const int* pos,
                                        const Args3<R>& A) {
    const R* base = P + (long long)a * A.N + c;
    const int cc[3] = {c3x(a), c3y(a), c3z(a)};
    R v = 0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (cc[ax] == 0) continue;
        const int m = pos[ax], sh = cc[ax] > 0 ? 0 : 1;
        R h[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) h[s] = __ldg(base + nb.off[ax][s + sh]);
        const AxisMetric<R>& M = A.m[ax];
        if (cc[ax] > 0) {
            const R pw = M.wp(0, m) * h[0] + M.wp(1, m) * h[1] + M.wp(2, m) * h[2];
            const R pe = M.wp(0, m + 1) * h[1] + M.wp(1, m + 1) * h[2] + M.wp(2, m + 1) * h[3];
            v += (pe - pw) * M.invd(m);
        } else {
            const R pw = M.wm(0, m) * h[0] + M.wm(1, m) * h[1] + M.wm(2, m) * h[2];
            const R pe = M.wm(0, m + 1) * h[1] + M.wm(1, m + 1) * h[2] + M.wm(2, m + 1) * h[3];
            v -= (pe - pw) * M.invd(m);
        }
    }
    return v;
}

template <typename R, int a>
__device__ __forceinline__ void advect_all_in(const R* P, long long c, const Nbr3& nb, const int* pos,
                                              const Args3<R>& A, R* out) {
    out[a] = advect3_in<R, a>(P, c, nb, pos, A);
    if constexpr (a + 1 < Q3) advect_all_in<R, a + 1>(P, c, nb, pos, A, out);
}

// All 19 flux divergences of one cell: direct offsets when the whole
// stencil is in the grid, the ghost rules otherwise.  A warp shares its z
// plane, so with plates on z only the two planes next to each plate take
// the general path and the rest never fetch its instructions.
template <typename R, bool G>
__device__ __forceinline__ void advect_cell(const R* P, int i, int j, int k, long long c, const Nbr3& nb,
                                            const Args3<R>& A, R* out) {
    if (nb.inside) {
        const int pos[3] = {i, j, k};
        advect_all_in<R, 0>(P, c, nb, pos, A, out);
    } else {
        advect_all<R, G, 0>(P, i, j, k, A, out);
    }
}

__device__ __forceinline__ bool cell_index(const int* n, int& i, int& j, int& k) {
    i = blockIdx.x * blockDim.x + threadIdx.x;
    j = blockIdx.y * blockDim.y + threadIdx.y;
    k = blockIdx.z;
    return i < n[0] && j < n[1];
}

// ---- FV pass 1: h^n and f~ + Coll^n (Eq. (semi)) ----
template <typename R, typename S, bool TH>
__global__ void __launch_bounds__(256) k3_pre(const Args3<R> A) {
    int i, j, k;
    if (!cell_index(A.n, i, j, k)) return;
    const long long c = cell3(A.n, i, j, k), N = A.N;
    R d[Q3], e[Q3];
    load19<S>(A.fin, N, c, d);
    if constexpr (TH) load19<S>(A.gin, N, c, e);
    Cell3<R, TH> m;
    m.moments(d, e, A);
#pragma unroll
    for (int a = 0; a < Q3; ++a) {
        R feqd, F, geqd;
        m.eq(a, A, feqd, F, geqd);
        const R neq = feqd - d[a];
        A.H[a * N + c] = d[a] + A.omh * neq + A.hf * F;
        A.FC[a * N + c] = d[a] + A.om * neq + A.cf * F;
        if constexpr (TH) {
            const R neqg = geqd - e[a];
            A.HG[a * N + c] = e[a] + A.omgh * neqg;
            A.GC[a * N + c] = e[a] + A.omg * neqg;
        }
    }
}

// Flux divergence of population a (a runtime index: the passes below loop
// over the populations so that neither their code nor their registers grow
// with 19 or 38 populations).
template <typename R, bool G>
__device__ __forceinline__ R advect_pop(const R* P, int a, int i, int j, int k, long long c, const Nbr3& nb,
                                        const Args3<R>& A) {
    const int pos[3] = {i, j, k};
    const R* base = P + (long long)a * A.N + c;
    R v = 0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const int cv = c3comp(a, ax);
        if (cv == 0) continue;
        const int m = pos[ax];
        const bool up = cv > 0;  // upwind nodes (m-2, m-1, m, m+1) or (m-1, m, m+1, m+2)
        R h[4];
        if (nb.inside) {
#pragma unroll
            for (int s = 0; s < 4; ++s) h[s] = __ldg(base + (up ? nb.off[ax][s] : nb.off[ax][s + 1]));
        } else {
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                int id[3] = {i, j, k};
                id[ax] = m + s + (up ? -2 : -1);
                h[s] = hval<R, G>(P, a, id[0], id[1], id[2], A);
            }
        }
        // weights of faces m and m + 1 from the face-major table
        const R* fw = A.ft[ax] + kFaceRow * m + (up ? 0 : 3);
        const R* fe = fw + kFaceRow;
        const R pw = __ldg(fw) * h[0] + __ldg(fw + 1) * h[1] + __ldg(fw + 2) * h[2];
        const R pe = __ldg(fe) * h[1] + __ldg(fe + 1) * h[2] + __ldg(fe + 2) * h[3];
        const R invd = __ldg(A.ft[ax] + kFaceRow * m + 6);
        v += R(cv) * (pe - pw) * invd;
    }
    return v;
}

// ---- FV pass 2: predictor f~* = f~ + Coll - dt A[h^n], then h* ----
// f~* is parked in the h* buffer while its moments accumulate, then
// overwritten there by h* (same thread, same addresses).
template <typename R, bool TH>
__global__ void __launch_bounds__(256) k3_mid(const Args3<R> A) {
    int i, j, k;
    if (!cell_index(A.n, i, j, k)) return;
    const long long c = cell3(A.n, i, j, k), N = A.N;
    const Nbr3 nb = neighbours3(A.n, A.bc, i, j, k);
    R r = 0, jx = 0, jy = 0, jz = 0, td = 0;
#pragma unroll 1
    for (int a = 0; a < Q3; ++a) {
        const R adv = advect_pop<R, false>(A.H, a, i, j, k, c, nb, A);
        const R fc = A.FC[a * N + c];
        const R fs = fc - A.dt * adv;
        A.FC[a * N + c] = fc - A.hf * adv;
        A.HS[a * N + c] = fs;
        r += fs;
        jx += R(c3comp(a, 0)) * fs;
        jy += R(c3comp(a, 1)) * fs;
        jz += R(c3comp(a, 2)) * fs;
    }
    if constexpr (TH) {
#pragma unroll 1
        for (int a = 0; a < Q3; ++a) {
            const R adv = advect_pop<R, true>(A.HG, a, i, j, k, c, nb, A);
            const R gc = A.GC[a * N + c];
            const R es = gc - A.dt * adv;
            A.GC[a * N + c] = gc - A.hf * adv;
            A.HGS[a * N + c] = es;
            td += es;
        }
    }
    Cell3<R, TH> m;
    m.from_sums(r, jx, jy, jz, td, A);
#pragma unroll 1
    for (int a = 0; a < Q3; ++a) {
        R feqd, F, geqd;
        m.eq(a, A, feqd, F, geqd);
        const R fs = A.HS[a * N + c];
        A.HS[a * N + c] = fs + A.omh * (feqd - fs) + A.hf * F;
        if constexpr (TH) {
            const R es = A.HGS[a * N + c];
            A.HGS[a * N + c] = es + A.omgh * (geqd - es);
        }
    }
}

// ---- FV pass 3: corrector, Eq. (semi-heun) ----
template <typename R, typename S, bool TH>
__global__ void __launch_bounds__(256) k3_post(const Args3<R> A) {
    int i, j, k;
    if (!cell_index(A.n, i, j, k)) return;
    const long long c = cell3(A.n, i, j, k), N = A.N;
    const Nbr3 nb = neighbours3(A.n, A.bc, i, j, k);
    S* out = static_cast<S*>(A.fout);
#pragma unroll 1
    for (int a = 0; a < Q3; ++a)
        Store<S>::st(out + a * N + c, A.FC[a * N + c] - A.hf * advect_pop<R, false>(A.HS, a, i, j, k, c, nb, A));
    if constexpr (TH) {
        S* gout = static_cast<S*>(A.gout);
#pragma unroll 1
        for (int a = 0; a < Q3; ++a)
            Store<S>::st(gout + a * N + c,
                         A.GC[a * N + c] - A.hf * advect_pop<R, true>(A.HGS, a, i, j, k, c, nb, A));
    }
}

// ---- ST: collide and push, Eq. (ST) at dt = dx = 1 ----
template <typename R, typename S, bool TH>
__global__ void __launch_bounds__(256) k3_st(const Args3<R> A) {
    int i, j, k;
    if (!cell_index(A.n, i, j, k)) return;
    const long long c = cell3(A.n, i, j, k), N = A.N;
    R d[Q3], e[Q3];
    load19<S>(A.fin, N, c, d);
    if constexpr (TH) load19<S>(A.gin, N, c, e);
    Cell3<R, TH> m;
    m.moments(d, e, A);
    S* fo = static_cast<S*>(A.fout);
    S* go = static_cast<S*>(A.gout);
#pragma unroll
    for (int a = 0; a < Q3; ++a) {
        R feqd, F, geqd;
        m.eq(a, A, feqd, F, geqd);
        const R post = d[a] + A.om * (feqd - d[a]) + A.cf * F;
        const R gpost = TH ? e[a] + A.omg * (geqd - e[a]) : R(0);
        int t[3] = {i + c3x(a), j + c3y(a), k + c3z(a)};
        bool out = false;
        R tw = 0;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            if (t[ax] >= 0 && t[ax] < A.n[ax]) continue;
            if (A.bc[ax] == LB_BC_PERIODIC) {
                t[ax] = t[ax] < 0 ? t[ax] + A.n[ax] : t[ax] - A.n[ax];
            } else {
                out = true;
                if (ax == 2) tw = t[2] < 0 ? A.dTb : A.dTt;
            }
        }
        if (out) {  // half-way bounce-back; g anti-bounce-back at the plates
            Store<S>::st(fo + inv3(a) * N + c, post);
            if constexpr (TH) Store<S>::st(go + inv3(a) * N + c, -gpost + R(2) * w3<R>(a) * tw);
        } else {
            const long long tc = cell3(A.n, t[0], t[1], t[2]);
            Store<S>::st(fo + a * N + tc, post);
            if constexpr (TH) Store<S>::st(go + a * N + tc, gpost);
        }
    }
}

// ---- observables ----
template <typename S, bool TH>
__global__ void k3_init(const Aux3 X, const double* fields, S* f, S* g) {
    int i, j, k;
    if (!cell_index(X.n, i, j, k)) return;
    const long long c = cell3(X.n, i, j, k), N = X.N;
    const double rho = fields[c], ux = fields[N + c], uy = fields[2 * N + c], uz = fields[3 * N + c];
    const double T = fields[4 * N + c];
    const double az = X.az + (TH ? X.bg * (T - X.T0) : 0.0);
    const double uu = ux * ux + uy * uy + uz * uz;
    for (int a = 0; a < Q3; ++a) {
        const double w = w3<double>(a);
        const double cu = c3x(a) * ux + c3y(a) * uy + c3z(a) * uz;
        const double poly = 3.0 * cu + 4.5 * cu * cu - 1.5 * uu;
        const double ca = c3x(a) * X.ax + c3y(a) * X.ay + c3z(a) * az;
        const double ua = ux * X.ax + uy * X.ay + uz * az;
        const double F = w * rho * (3.0 * (ca - ua) + 9.0 * cu * ca);
        Store<S>::st(f + a * N + c, (S)(w * ((rho - 1.0) + rho * poly) - 0.5 * X.dt * F));
        if (TH) Store<S>::st(g + a * N + c, (S)(w * ((T - X.T0) + T * poly)));
    }
}

template <typename S, bool TH>
__global__ void k3_moments(const Aux3 X, double* out) {
    int i, j, k;
    if (!cell_index(X.n, i, j, k)) return;
    const long long c = cell3(X.n, i, j, k), N = X.N;
    const S* f = static_cast<const S*>(X.f);
    const S* g = static_cast<const S*>(X.g);
    double r = 0, jx = 0, jy = 0, jz = 0, td = 0;
    for (int a = 0; a < Q3; ++a) {
        const double v = (double)Store<S>::ld(f + a * N + c);
        r += v;
        jx += c3x(a) * v;
        jy += c3y(a) * v;
        jz += c3z(a) * v;
        if (TH) td += (double)Store<S>::ld(g + a * N + c);
    }
    const double rho = 1.0 + r, T = X.T0 + td, az = X.az + (TH ? X.bg * td : 0.0);
    out[c] = rho;
    out[N + c] = jx / rho + 0.5 * X.dt * X.ax;
    out[2 * N + c] = jy / rho + 0.5 * X.dt * X.ay;
    out[3 * N + c] = jz / rho + 0.5 * X.dt * az;
    out[4 * N + c] = T;
}

template <typename S>
__global__ void k3_pack(const double* src, S* dst, long long N, double off) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= Q3 * N) return;
    Store<S>::st(dst + t, (S)(src[t] - w3<double>((int)(t / N)) * off));
}

template <typename S>
__global__ void k3_unpack(const S* src, double* dst, long long N, double off) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= Q3 * N) return;
    dst[t] = (double)Store<S>::ld(src + t) + w3<double>((int)(t / N)) * off;
}

// One block per z plane, fixed-order tree over a 256-thread block.
__global__ void __launch_bounds__(256) k3_plane_sums(const double* F, const double* dx, const double* dy,
                                                     const double* dz, int nx, int ny, int nz, double T0,
                                                     double* out) {
    constexpr int K = 8;
    __shared__ double sh[K][256];
    const int k = blockIdx.x;
    const long long N = (long long)nx * ny * nz;
    double acc[K] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < nx * ny; t += blockDim.x) {
        const int i = t % nx, j = t / nx;
        const long long c = ((long long)k * ny + j) * nx + i;
        const double A = dx[i] * dy[j], V = A * dz[k];
        const double rho = F[c], T = F[4 * N + c];
        acc[0] += V * rho;
        acc[1] += V * rho * F[N + c];
        acc[2] += V * rho * F[2 * N + c];
        acc[3] += V * rho * F[3 * N + c];
        acc[4] += V * T;
        acc[5] += V * F[3 * N + c] * (T - T0);
        acc[6] += A * T;
        acc[7] += V;
    }
#pragma unroll
    for (int q = 0; q < K; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int q = 0; q < K; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < K) out[k * K + threadIdx.x] = sh[threadIdx.x][0];
}

dim3 grid3(const int* n) { return dim3((n[0] + 31) / 32, (n[1] + 7) / 8, n[2]); }

template <typename R, typename S, bool TH>
cudaError_t run_fv3(const Args3<R>& A, cudaStream_t s) {
    const dim3 b(32, 8), g = grid3(A.n);
    k3_pre<R, S, TH><<<g, b, 0, s>>>(A);
    count_launch();
    k3_mid<R, TH><<<g, b, 0, s>>>(A);
    count_launch();
    k3_post<R, S, TH><<<g, b, 0, s>>>(A);
    count_launch();
    return cudaGetLastError();
}

template <typename R, typename S, bool TH>
cudaError_t run_st3(const Args3<R>& A, cudaStream_t s) {
    k3_st<R, S, TH><<<grid3(A.n), dim3(32, 8), 0, s>>>(A);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch3_fv(Prec p, bool th, const void* args, cudaStream_t s) {
    if (p == Prec::F64) {
        const auto& A = *static_cast<const Args3<double>*>(args);
        return th ? run_fv3<double, double, true>(A, s) : run_fv3<double, double, false>(A, s);
    }
    if (p == Prec::F32) {
        const auto& A = *static_cast<const Args3<float>*>(args);
        return th ? run_fv3<float, float, true>(A, s) : run_fv3<float, float, false>(A, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch3_st(Prec p, bool th, const void* args, cudaStream_t s) {
    if (p == Prec::F64) {
        const auto& A = *static_cast<const Args3<double>*>(args);
        return th ? run_st3<double, double, true>(A, s) : run_st3<double, double, false>(A, s);
    }
    if (p == Prec::F32) {
        const auto& A = *static_cast<const Args3<float>*>(args);
        return th ? run_st3<float, float, true>(A, s) : run_st3<float, float, false>(A, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch3_init(Prec p, bool th, const Aux3& a, const double* fields, void* f, void* g, cudaStream_t s) {
    const dim3 b(32, 8), gr = grid3(a.n);
    if (p == Prec::F64) {
        if (th) k3_init<double, true><<<gr, b, 0, s>>>(a, fields, (double*)f, (double*)g);
        else k3_init<double, false><<<gr, b, 0, s>>>(a, fields, (double*)f, (double*)g);
    } else if (p == Prec::F32) {
        if (th) k3_init<float, true><<<gr, b, 0, s>>>(a, fields, (float*)f, (float*)g);
        else k3_init<float, false><<<gr, b, 0, s>>>(a, fields, (float*)f, (float*)g);
    } else {
        return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch3_moments(Prec p, bool th, const Aux3& a, double* fields, cudaStream_t s) {
    const dim3 b(32, 8), gr = grid3(a.n);
    if (p == Prec::F64) {
        if (th) k3_moments<double, true><<<gr, b, 0, s>>>(a, fields);
        else k3_moments<double, false><<<gr, b, 0, s>>>(a, fields);
    } else if (p == Prec::F32) {
        if (th) k3_moments<float, true><<<gr, b, 0, s>>>(a, fields);
        else k3_moments<float, false><<<gr, b, 0, s>>>(a, fields);
    } else {
        return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch3_pack(Prec p, const double* src, void* dst, long long N, double off, cudaStream_t s) {
    const long long n = Q3 * N;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (p == Prec::F64) k3_pack<double><<<blocks, 256, 0, s>>>(src, (double*)dst, N, off);
    else if (p == Prec::F32) k3_pack<float><<<blocks, 256, 0, s>>>(src, (float*)dst, N, off);
    else return cudaErrorInvalidValue;
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch3_unpack(Prec p, const void* src, double* dst, long long N, double off, cudaStream_t s) {
    const long long n = Q3 * N;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (p == Prec::F64) k3_unpack<double><<<blocks, 256, 0, s>>>((const double*)src, dst, N, off);
    else if (p == Prec::F32) k3_unpack<float><<<blocks, 256, 0, s>>>((const float*)src, dst, N, off);
    else return cudaErrorInvalidValue;
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch3_plane_sums(const double* fields, const double* dx, const double* dy, const double* dz,
                               int nx, int ny, int nz, double T0, double* out, cudaStream_t s) {
    k3_plane_sums<<<nz, 256, 0, s>>>(fields, dx, dy, dz, nx, ny, nz, T0, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lbgb
