// k3_st_pair.cu -- the D3Q19 ST step (Eq. (ST), Sec. II A, dt = dx = 1)
// with FP32 storage, two adjacent x cells per thread and packed FP32 pair
// arithmetic (Blackwell f32x2), for grids with an even nx.
//
// Every population of the thread's two cells is one 8-byte load.  A warp
// holds 64 consecutive cells of one (y, z) row, so its rows and planes are
// the same for all lanes.  When the row's destinations need no wall rule
// (x periodic, and y and z periodic or interior), every post-collision
// value is stored as part of an aligned pair: the populations that move in
// x are realigned across lanes with one shuffle, and only the lanes at the
// warp's or the row's ends add single stores, wrapping periodically.  Rows
// next to a wall (half-way bounce-back for f, anti-bounce-back through the
// plate temperature for g) store value by value.
#include "lb3_pair.cuh"

namespace lbgb {

namespace {

using namespace pairmath;

// The ST relaxation of population a of the pair: post-collision f (and g).
template <bool TH, int a>
__device__ __forceinline__ void post(const Cell3P<TH>& m, const V2 d, const V2 e, const Args3<float>& A, V2& pf,
                                     V2& pg) {
    V2 feqd, F, geqd;
    m.template eq<a>(A, feqd, F, geqd);
    pf = fma2(bc(A.om), feqd - d, fma2(bc(A.cf), F, d));
    pg = TH ? fma2(bc(A.omg), geqd - e, e) : bc(0.0f);
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

template <bool TH, int a>
__device__ __forceinline__ void store_fast(float* fo, float* go, long long base, int i, int nx, int lane, bool on,
                                           bool right_on, V2 pf, V2 pg) {
    const unsigned full = 0xffffffffu;
    if constexpr (c3x(a) == 0) {
        if (on) {
            PairIO<float>::st(fo + base + i, pf);
            if constexpr (TH) PairIO<float>::st(go + base + i, pg);
        }
    } else if constexpr (c3x(a) > 0) {
        // cells i, i+1 move to i+1, i+2: the pair at i is (i-1's, i's)
        const float lf = __shfl_up_sync(full, pf.v.y, 1);
        const float lg = TH ? __shfl_up_sync(full, pg.v.y, 1) : 0.0f;
        if (on) {
            if (lane > 0) {
                PairIO<float>::st(fo + base + i, mk(lf, pf.v.x));
                if constexpr (TH) PairIO<float>::st(go + base + i, mk(lg, pg.v.x));
            } else {
                fo[base + i + 1] = pf.v.x;
                if constexpr (TH) go[base + i + 1] = pg.v.x;
            }
            if (lane == 31 || !right_on) {
                const int t = i + 2 == nx ? 0 : i + 2;
                fo[base + t] = pf.v.y;
                if constexpr (TH) go[base + t] = pg.v.y;
            }
        }
    } else {
        // cells i, i+1 move to i-1, i: the pair at i is (i+1's, i+2's)
        const float rf = __shfl_down_sync(full, pf.v.x, 1);
        const float rg = TH ? __shfl_down_sync(full, pg.v.x, 1) : 0.0f;
        if (on) {
            if (lane < 31 && right_on) {
                PairIO<float>::st(fo + base + i, mk(pf.v.y, rf));
                if constexpr (TH) PairIO<float>::st(go + base + i, mk(pg.v.y, rg));
            } else {
                fo[base + i] = pf.v.y;
                if constexpr (TH) go[base + i] = pg.v.y;
            }
            if (lane == 0) {
                const int t = i == 0 ? nx - 1 : i - 1;
                fo[base + t] = pf.v.x;
                if constexpr (TH) go[base + t] = pg.v.x;
            }
        }
    }
}

template <bool TH, int a>
__device__ __forceinline__ void store_general(float* fo, float* go, const Args3<float>& A, int i, int j, int k,
                                              V2 pf, V2 pg) {
    const long long N = A.N;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float vf = h ? pf.v.y : pf.v.x, vg = h ? pg.v.y : pg.v.x;
        int t[3] = {i + h + c3x(a), j + c3y(a), k + c3z(a)};
        bool out = false;
        float tw = 0.0f;
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
        const long long c = ((long long)k * A.n[1] + j) * A.n[0] + i + h;
        if (out) {
            fo[inv3(a) * N + c] = vf;
            if constexpr (TH) go[inv3(a) * N + c] = -vg + 2.0f * w3<float>(a) * tw;
        } else {
            const long long tc = ((long long)t[2] * A.n[1] + t[1]) * A.n[0] + t[0];
            fo[a * N + tc] = vf;
            if constexpr (TH) go[a * N + tc] = vg;
        }
    }
}

template <bool TH, int a>
__device__ __forceinline__ void do_pop(const Cell3P<TH>& m, const V2* d, const V2* e, const Args3<float>& A,
                                       float* fo, float* go, bool fast, int i, int j, int k, int lane, bool on,
                                       bool right_on) {
    V2 pf, pg;
    post<TH, a>(m, d[a], TH ? e[a] : bc(0.0f), A, pf, pg);
    if (fast) {
        const int jj = wrapi(j + c3y(a), A.n[1]), kk = wrapi(k + c3z(a), A.n[2]);
        const long long base = a * A.N + ((long long)kk * A.n[1] + jj) * A.n[0];
        store_fast<TH, a>(fo, go, base, i, A.n[0], lane, on, right_on, pf, pg);
    } else if (on) {
        store_general<TH, a>(fo, go, A, i, j, k, pf, pg);
    }
    if constexpr (a + 1 < Q3) do_pop<TH, a + 1>(m, d, e, A, fo, go, fast, i, j, k, lane, on, right_on);
}

}  // namespace

// blockDim = (32, 8): a warp is 32 pairs (64 cells) of one row.
template <bool TH>
__global__ void __launch_bounds__(256, 2) k3_st_pair(const Args3<float> A) {
    const int lane = threadIdx.x;
    const int i = 2 * (blockIdx.x * 32 + lane);
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const int nx = A.n[0], ny = A.n[1], nz = A.n[2];
    if (j >= ny) return;  // whole warps: j is the same on every lane
    const bool on = i < nx;
    const long long N = A.N, c = ((long long)k * ny + j) * nx + i;
    V2 d[Q3], e[Q3];
#pragma unroll
    for (int a = 0; a < Q3; ++a) {
        d[a] = on ? PairIO<float>::ld(static_cast<const float*>(A.fin) + a * N + c) : bc(0.0f);
        if constexpr (TH) e[a] = on ? PairIO<float>::ld(static_cast<const float*>(A.gin) + a * N + c) : bc(0.0f);
    }
    Cell3P<TH> m;
    m.moments(d, e, A);
    const bool right_on = i + 2 < nx;  // the next lane's pair exists
    const bool fast = A.bc[0] == LB_BC_PERIODIC && (A.bc[1] == LB_BC_PERIODIC || (j >= 1 && j + 1 < ny)) &&
                      (A.bc[2] == LB_BC_PERIODIC || (k >= 1 && k + 1 < nz));
    do_pop<TH, 0>(m, d, e, A, static_cast<float*>(A.fout), static_cast<float*>(A.gout), fast, i, j, k, lane, on,
                  right_on);
}

bool st3_pair_ok(Prec p, const int* n) { return p == Prec::F32 && n[0] % 2 == 0; }

cudaError_t launch3_st_pair(bool th, const void* args, cudaStream_t s) {
    const Args3<float>& A = *static_cast<const Args3<float>*>(args);
    const dim3 b(32, 8), g((A.n[0] / 2 + 31) / 32, (A.n[1] + 7) / 8, A.n[2]);
    if (th) k3_st_pair<true><<<g, b, 0, s>>>(A);
    else k3_st_pair<false><<<g, b, 0, s>>>(A);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lbgb
