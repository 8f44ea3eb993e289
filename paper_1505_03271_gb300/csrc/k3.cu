// k3.cu -- the D3Q19 (three-dimensional) time steps of Sec. II and the
// observables' kernels.
//
// ST, Eq. (ST): one fused collide-and-push kernel, one thread per cell;
// half-way bounce-back at walls, anti-bounce-back of g at the z plates.
//
// FV, Eqs. (semi) and (semi-heun): four passes over the grid with the
// intermediate fields in HBM:
//   k3_pre          f~ -> h^n (and its z ghost planes) and f~ + Coll^n  (local)
//   k3_adv (pred.)  A[h^n] per population (QUICK on its own stencil)
//                   -> f~* (parked), f~ + Coll - dt/2 A
//   k3_star         moments of f~* -> h* (and its z ghost planes)       (local)
//   k3_adv (corr.)  A[h*] -> f~^(n+1) = f~ + Coll - dt/2 (A[h^n] + A[h*])
// The flux passes are k3_adv below or, where the grid allows it, the staged
// passes of k3_staged.cu.
// A fused 3-D tile would recompute a 4-cell halo on all six faces, or hold
// 19 (38) populations of several halo planes in shared memory; these passes
// recompute nothing and stream about 6x the compulsory bytes.  Faces are
// taken dimension by dimension from the nodes of their own grid line
// (Sec. II B 3), so only face ghosts are ever read.
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

// Padded layout of the advected fields h, h* (and hg, hg*): two ghost
// planes below and above the grid in z, [pop][nz + 4][ny][nx], so that the
// z stencil never leaves the array.  zghost fills the ghost planes:
// periodic copies, or the wall rules of Sec. II B 5 (double reflection,
// h_a(ghost) = h_inv(a)(mirror); the thermal field anti-reflected,
// hg'_a(ghost) = 2 w_a (T_wall - T0) - hg'_inv(a)(mirror)).
__device__ __forceinline__ long long padded3(const int* n, int i, int j, int k) {
    return ((long long)(k + 2) * n[1] + j) * n[0] + i;
}

// Advected-field value at (i, j, padded plane k + 2) when i or j lies
// outside the grid (never both: the stencil is a cross): periodic wrap or
// wall mirror with the reflected population.  Thermal grids are periodic in
// x and y, so only the flow field meets these walls.
template <typename R>
__device__ __forceinline__ R hval_xy(const R* P, int a, int i, int j, int k, const Args3<R>& A) {
    int idx[2] = {i, j};
    int b = a;
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        const int n = A.n[ax];
        if (idx[ax] >= 0 && idx[ax] < n) continue;
        if (A.bc[ax] == LB_BC_PERIODIC) {
            idx[ax] = ((idx[ax] % n) + n) % n;
        } else {
            idx[ax] = idx[ax] < 0 ? -idx[ax] - 1 : 2 * n - 1 - idx[ax];
            b = inv3(a);
        }
    }
    return __ldg(P + (long long)b * A.NP + padded3(A.n, idx[0], idx[1], k));
}

__device__ __forceinline__ bool cell_index(const int* n, int& i, int& j, int& k) {
    i = blockIdx.x * blockDim.x + threadIdx.x;
    j = blockIdx.y * blockDim.y + threadIdx.y;
    k = blockIdx.z;
    return i < n[0] && j < n[1];
}

// z ghost planes of the padded advected field (Sec. II B 5), written by the
// cells they copy, so that no separate pass fills them.  Periodic z: ghost
// plane gk in {-2, -1, nz, nz + 1} holds plane gk mod nz.  z walls: the
// ghost -1 - k (k = 0, 1) and 2 nz - 1 - k (k = nz - 2, nz - 1) of the
// reflected population inv(a) hold h_a of plane k (double reflection); the
// thermal field is anti-reflected about the plate: 2 w (T_wall - T0) - h.
template <typename R>
__device__ __forceinline__ void zghost(R* P, int a, R v, int i, int j, int k, bool th, const Args3<R>& A) {
    const int nz = A.n[2];
    if (A.bc[2] == LB_BC_PERIODIC) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int gk = g < 2 ? g - 2 : nz + g - 2;
            const int src = ((gk % nz) + nz) % nz;
            if (src == k) P[(long long)a * A.NP + padded3(A.n, i, j, gk)] = v;
        }
    } else {
        const int b = inv3(a);
        if (k <= 1) P[(long long)b * A.NP + padded3(A.n, i, j, -1 - k)] = th ? R(2) * w3<R>(b) * A.dTb - v : v;
        if (k >= nz - 2)
            P[(long long)b * A.NP + padded3(A.n, i, j, 2 * nz - 1 - k)] = th ? R(2) * w3<R>(b) * A.dTt - v : v;
    }
}

// The ghost images of cell (i, j, k) of h (and hg), from the values this
// thread has just stored; k is uniform over the CTA, so interior planes
// skip it at no cost.
template <typename R, bool TH>
__device__ __forceinline__ void zghosts(R* P, R* PG, int i, int j, int k, const Args3<R>& A) {
    if (k >= 2 && k < A.n[2] - 2) return;
    const long long cp = padded3(A.n, i, j, k);
    for (int a = 0; a < Q3; ++a) {
        zghost(P, a, P[a * A.NP + cp], i, j, k, false, A);
        if constexpr (TH) zghost(PG, a, PG[a * A.NP + cp], i, j, k, true, A);
    }
}

// ---- FV pass 1: h^n and f~ + Coll^n (Eq. (semi)) ----
template <typename R, typename S, bool TH>
__global__ void __launch_bounds__(256) k3_pre(const Args3<R> A) {
    int i, j, k;
    if (!cell_index(A.n, i, j, k)) return;
    const long long c = cell3(A.n, i, j, k), N = A.N, cp = padded3(A.n, i, j, k), NP = A.NP;
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
        A.H[a * NP + cp] = d[a] + A.omh * neq + A.hF * F;
        A.FC[a * N + c] = d[a] + A.om * neq + A.cf * F;
        if constexpr (TH) {
            const R neqg = geqd - e[a];
            A.HG[a * NP + cp] = e[a] + A.omgh * neqg;
            A.GC[a * N + c] = e[a] + A.omg * neqg;
        }
    }
    zghosts<R, TH>(A.H, A.HG, i, j, k, A);
}

// ---- FV flux passes, one population per CTA ----
// The flux of population a reads only population a's own advected field,
// so the predictor's and the corrector's flux passes run one population per
// CTA: a 32 x 8 block of columns marches up a chunk of z planes, keeping
// the four z-stencil nodes of its column in registers (one new value per
// plane; the padded ghost planes make every z node a plain load).  The x
// and y node offsets and weights of a column are set once.
//   predictor (CORR = false): f~* = f~ + Coll - dt A[h^n] into the h* buffer
//                             (parked until k3_star), f~ + Coll -= dt/2 A
//   corrector (CORR = true):  f~^(n+1) = (f~ + Coll - dt/2 A[h^n]) - dt/2 A[h*]
// blockIdx.z = chunk * np + p; p < 19 flow, p >= 19 thermal population p - 19.

// x or y stencil offsets of a column: nodes s = -2..2 (wrapped once on
// periodic axes); `in` is false when a node lies past a wall.
struct Line5 {
    int off[5];
    bool in;
};

__device__ __forceinline__ Line5 line5(int pos, int n, int bc, int stride) {
    Line5 L;
    L.in = true;
#pragma unroll
    for (int s = -2; s <= 2; ++s) {
        int p = pos + s;
        if (p < 0 || p >= n) {
            if (bc == LB_BC_PERIODIC) p = ((p % n) + n) % n;
            else { L.in = false; p = pos; }
        }
        L.off[s + 2] = (p - pos) * stride;
    }
    return L;
}

// QUICK weights of one axis at cell m for the sign of c: west-face and
// east-face triples and 1/width (row-major metric).
template <typename R>
struct AxisW {
    R w[3], e[3], inv;
    __device__ __forceinline__ void load(const AxisMetric<R>& M, int m, int cv) {
        const int r0 = cv > 0 ? 0 : 3;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            w[r] = M.row(r0 + r, m);
            e[r] = M.row(r0 + r, m + 1);
        }
        inv = M.invd(m);
    }
    __device__ __forceinline__ R div(int cv, const R* h) const {
        const R pw = w[0] * h[0] + w[1] * h[1] + w[2] * h[2];
        const R pe = e[0] * h[1] + e[1] * h[2] + e[2] * h[3];
        return R(cv) * (pe - pw) * inv;
    }
};

template <typename R, typename S, bool CORR, bool G, bool FAST>
__device__ __forceinline__ void adv_pop_column(const Args3<R>& A, int a, int i, int j, int k0, int k1,
                                               const Line5& lx, const Line5& ly) {
    const long long N = A.N, NP = A.NP;
    const int nx = A.n[0], ny = A.n[1];
    const long long plane = (long long)nx * ny;
    const R* P = G ? (CORR ? A.HGS : A.HG) : (CORR ? A.HS : A.H);
    R* FCp = G ? A.GC : A.FC;
    R* park = G ? A.HGS : A.HS;
    const int cx = c3comp(a, 0), cy = c3comp(a, 1), cz = c3comp(a, 2);
    const R* col = P + (long long)a * NP + (long long)j * nx + i;  // padded plane 0 of this column
    AxisW<R> WX, WY;
    int ox[4] = {0, 0, 0, 0}, oy[4] = {0, 0, 0, 0};
    if (cx != 0) {
        WX.load(A.m[0], i, cx);
#pragma unroll
        for (int s = 0; s < 4; ++s) ox[s] = cx > 0 ? lx.off[s] : lx.off[s + 1];
    }
    if (cy != 0) {
        WY.load(A.m[1], j, cy);
#pragma unroll
        for (int s = 0; s < 4; ++s) oy[s] = cy > 0 ? ly.off[s] : ly.off[s + 1];
    }
    const int zs = cz > 0 ? -2 : -1;  // z nodes (k-2..k+1) or (k-1..k+2)
    R zr[4] = {0, 0, 0, 0};
    if (cz != 0) {
#pragma unroll
        for (int s = 0; s < 3; ++s) zr[s] = __ldg(col + (long long)(k0 + zs + s + 2) * plane);
    }
    for (int k = k0; k < k1; ++k) {
        const R* cp = col + (long long)(k + 2) * plane;
        R v = 0;
        if (cx != 0) {
            R h[4];
#pragma unroll
            for (int s = 0; s < 4; ++s)
                h[s] = FAST ? __ldg(cp + ox[s]) : hval_xy<R>(P, a, i + s + (cx > 0 ? -2 : -1), j, k, A);
            v += WX.div(cx, h);
        }
        if (cy != 0) {
            R h[4];
#pragma unroll
            for (int s = 0; s < 4; ++s)
                h[s] = FAST ? __ldg(cp + oy[s]) : hval_xy<R>(P, a, i, j + s + (cy > 0 ? -2 : -1), k, A);
            v += WY.div(cy, h);
        }
        if (cz != 0) {
            zr[3] = __ldg(cp + (long long)(zs + 3) * plane);
            const R* fz = A.ft[2] + kFaceRow * k + (cz > 0 ? 0 : 3);  // uniform over the block
            const R pw = __ldg(fz) * zr[0] + __ldg(fz + 1) * zr[1] + __ldg(fz + 2) * zr[2];
            const R pe = __ldg(fz + kFaceRow) * zr[1] + __ldg(fz + kFaceRow + 1) * zr[2] +
                         __ldg(fz + kFaceRow + 2) * zr[3];
            v += R(cz) * (pe - pw) * __ldg(A.ft[2] + kFaceRow * k + 6);
            zr[0] = zr[1];
            zr[1] = zr[2];
            zr[2] = zr[3];
        }
        const long long q = (long long)a * N + (long long)k * plane + (long long)j * nx + i;
        const R fc = FCp[q];
        if constexpr (CORR) {
            S* out = static_cast<S*>(G ? A.gout : A.fout);
            Store<S>::st(out + q, fc - A.hf * v);
        } else {
            FCp[q] = fc - A.hf * v;
            park[(long long)a * NP + (long long)(k + 2) * plane + (long long)j * nx + i] = fc - A.dt * v;
        }
    }
}

template <typename R, typename S, bool CORR>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 2 : 4) k3_adv(const Args3<R> A, int np, int kc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= A.n[0] || j >= A.n[1]) return;
    const int p = blockIdx.z % np, chunk = blockIdx.z / np;
    const int k0 = chunk * kc, k1 = min(k0 + kc, A.n[2]);
    const Line5 lx = line5(i, A.n[0], A.bc[0], 1), ly = line5(j, A.n[1], A.bc[1], A.n[0]);
    const bool fast = lx.in && ly.in;
    if (p < Q3) {
        if (fast) adv_pop_column<R, S, CORR, false, true>(A, p, i, j, k0, k1, lx, ly);
        else adv_pop_column<R, S, CORR, false, false>(A, p, i, j, k0, k1, lx, ly);
    } else {
        // thermal grids are periodic in x and y: always the plain path
        adv_pop_column<R, S, CORR, true, true>(A, p - Q3, i, j, k0, k1, lx, ly);
    }
}

// ---- FV: moments of f~* (parked in the h* buffers) and h* ----
// Two CTAs per SM for FP32 (at most 128 registers): the compiler keeps the
// 38 loaded values live between the moment sums and the h* stores.
template <typename R, bool TH>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 1 : 2) k3_star(const Args3<R> A) {
    int i, j, k;
    if (!cell_index(A.n, i, j, k)) return;
    const long long cp = padded3(A.n, i, j, k), NP = A.NP;
    // moments of f~* (and g~*) summed as they are read; the h* pass then
    // reads each value again
    R r = 0, jx = 0, jy = 0, jz = 0, td = 0;
#pragma unroll
    for (int a = 0; a < Q3; ++a) {
        const R fs = A.HS[a * NP + cp];
        r += fs;
        jx += R(c3x(a)) * fs;
        jy += R(c3y(a)) * fs;
        jz += R(c3z(a)) * fs;
        if constexpr (TH) td += A.HGS[a * NP + cp];
    }
    Cell3<R, TH> m;
    m.from_sums(r, jx, jy, jz, td, A);
#pragma unroll
    for (int a = 0; a < Q3; ++a) {
        R feqd, F, geqd;
        m.eq(a, A, feqd, F, geqd);
        const R fs = A.HS[a * NP + cp];
        A.HS[a * NP + cp] = fs + A.omh * (feqd - fs) + A.hF * F;
        if constexpr (TH) {
            const R es = A.HGS[a * NP + cp];
            A.HGS[a * NP + cp] = es + A.omgh * (geqd - es);
        }
    }
    zghosts<R, TH>(A.HS, A.HGS, i, j, k, A);
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

// z planes per CTA of the flux passes
constexpr int kZChunk = 16;

// staged: the flux passes of k3_staged.cu instead of k3_adv
template <typename R, typename S, bool TH>
cudaError_t run_fv3(const Args3<R>& A, bool staged, cudaStream_t s) {
    const dim3 b(32, 8), g = grid3(A.n);
    const int np = TH ? 2 * Q3 : Q3;
    const int chunks = (A.n[2] + kZChunk - 1) / kZChunk;
    const dim3 gx((A.n[0] + 31) / 32, (A.n[1] + 7) / 8, 1);
    const dim3 ga(gx.x, gx.y, chunks * np);
    const Prec p = sizeof(R) == 8 ? Prec::F64 : Prec::F32;
    cudaError_t e;
    k3_pre<R, S, TH><<<g, b, 0, s>>>(A);
    if (staged) {
        if ((e = launch3_adv_staged(p, false, np, &A, s)) != cudaSuccess) return e;
    } else {
        k3_adv<R, S, false><<<ga, b, 0, s>>>(A, np, kZChunk);
        count_launch();
    }
    k3_star<R, TH><<<g, b, 0, s>>>(A);
    if (staged) {
        if ((e = launch3_adv_staged(p, true, np, &A, s)) != cudaSuccess) return e;
    } else {
        k3_adv<R, S, true><<<ga, b, 0, s>>>(A, np, kZChunk);
        count_launch();
    }
    for (int q = 0; q < 2; ++q) count_launch();
    return cudaGetLastError();
}

template <typename R, typename S, bool TH>
cudaError_t run_st3(const Args3<R>& A, cudaStream_t s) {
    k3_st<R, S, TH><<<grid3(A.n), dim3(32, 8), 0, s>>>(A);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch3_fv(Prec p, bool th, bool staged, const void* args, cudaStream_t s) {
    if (p == Prec::F64) {
        const auto& A = *static_cast<const Args3<double>*>(args);
        return th ? run_fv3<double, double, true>(A, staged, s) : run_fv3<double, double, false>(A, staged, s);
    }
    if (p == Prec::F32) {
        const auto& A = *static_cast<const Args3<float>*>(args);
        return th ? run_fv3<float, float, true>(A, staged, s) : run_fv3<float, float, false>(A, staged, s);
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
        if (st3_pair_ok(p, A.n)) return launch3_st_pair(th, args, s);
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
