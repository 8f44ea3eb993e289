// k3_staged.cu -- the flux passes of the 3-D FV step (Eqs. (semi) and
// (semi-heun); QUICK faces of Sec. II B 3 taken dimension by dimension)
// with their operands staged in shared memory by bulk asynchronous copies.
//
// The plain passes of k3.cu read every stencil node through L1/L2 and keep
// about three cache lines in flight per warp, which holds them near 1.5-1.8
// TB/s.  Here a CTA owns one population, a tile of ty whole x rows and a
// chunk of z planes.  Eight warps compute; one thread of a ninth warp keeps
// `ahead` planes (3 by default) of copies in flight beyond the planes the
// arithmetic uses:
//   - the rows of h (h* in the corrector) of the next plane, with two halo
//     rows on each side in y when c_y != 0.  The x rows are whole, so the
//     periodic x wrap is an index wrap in shared memory;
//   - the rows of f~ + Coll of the plane that the same step completes.
// Consecutive rows are contiguous in memory, so each run of them is one
// cp.async.bulk (two or three per plane) completing on the plane's
// mbarrier; a second mbarrier per ring slot tells the copy thread when the
// computing warps are done with it.  Every x, y and z stencil node is then a
// shared-memory load, and HBM sees each operand once per pass.  FP32 runs
// two adjacent x cells per thread in f32x2 arithmetic.
//
// Grids served (adv3_staged_ok): x and y periodic, and nx a power of two
// <= 256 whose rows are a multiple of 16 bytes (the bulk-copy granule).  z
// may be periodic or walls: the collision and star passes of k3.cu write
// the padded z ghost planes of h and h*.
//
// Every wait on a copy is bounded (Args3::wait_ns).  A CTA whose wait runs
// out sets *Args3::werr, waits (bounded again) for the copies it has issued,
// and returns; the host reports LB_ERR_TIMEOUT.
#include <type_traits>

#include "lb3.cuh"
#include "lb_async.cuh"
#include "lb_pair.cuh"

namespace lbgb {

namespace {

constexpr int kThreads = 256;        // computing threads; one more warp issues the copies
constexpr int kCells = 4;              // cells per thread and plane, at most
constexpr int kMaxSlots = 16;          // h ring slots (4 + ahead), one full and one empty barrier each
constexpr int kMaxSmem = 200 * 1024;   // dynamic shared memory of the largest shape

// Tile shape and shared-memory layout of one launch.  The h ring holds the
// four z nodes of the plane in work plus `ahead` planes in flight (4 + ahead
// slots, one mbarrier each); the f~ + Coll ring ahead + 1 planes.
struct Shape {
    int ty;                      // rows per tile (nx * ty <= kCells * kThreads)
    int kc;                      // z planes per CTA
    int ahead;                   // planes of copies in flight beyond those in use
    int zc_off, h_off, fc_off;   // byte offsets: z weights, h ring, f~ + Coll ring
    int bytes;
};

// Defaults, and the checks of a requested shape (0 = default).
int max_rows(int nx, size_t rs) { return (int)((rs == 4 ? kCells * kThreads : kCells * kThreads / 2) / nx); }

Shape staged_shape(int nx, int nz, size_t rs, int ty, int kc, int ahead) {
    Shape s;
    const int tmax = max_rows(nx, rs);
    s.ty = ty > 0 ? ty : (tmax < 1 ? 1 : (tmax > 16 ? 16 : tmax));
    s.kc = kc > 0 ? kc : 16;
    s.kc = s.kc < nz ? s.kc : nz;
    s.ahead = ahead > 0 ? ahead : 3;
    s.zc_off = 2 * kMaxSlots * 8;  // full and empty mbarriers
    s.h_off = s.zc_off + (int)((s.kc * 4 * rs + 15) / 16 * 16);
    s.fc_off = s.h_off + (int)((4 + s.ahead) * (s.ty + 4) * nx * rs);
    s.bytes = s.fc_off + (int)((s.ahead + 1) * s.ty * nx * rs);
    return s;
}

// Folded QUICK divergence weights of one cell on one axis: with the faces'
// weights w (west face) and e (east face) of the nodes (m-2..m+1) for c > 0
// or (m-1..m+2) for c < 0, c (Phi_e - Phi_w) / dx_m = sum_s K_s h(node s).
template <typename R>
__device__ __forceinline__ void fold4(const R* w, const R* e, R s, R* K) {
    K[0] = -w[0] * s;
    K[1] = (e[0] - w[1]) * s;
    K[2] = (e[1] - w[2]) * s;
    K[3] = e[2] * s;
}

template <typename R>
__device__ __forceinline__ void axis_fold(const AxisMetric<R>& M, int m, int cv, R* K) {
    const int q0 = cv > 0 ? 0 : 3;
    R w[3], e[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        w[r] = M.row(q0 + r, m);
        e[r] = M.row(q0 + r, m + 1);
    }
    fold4(w, e, R(cv) * M.invd(m), K);
}

// blockIdx = (y tile, z chunk, population p); p < 19 flow, p >= 19 thermal.
//   predictor (CORR = false): reads h^n and f~ + Coll; writes f~* (parked in
//                             the h* buffer) and f~ + Coll - dt/2 A[h^n]
//   corrector (CORR = true):  reads h* and f~ + Coll - dt/2 A[h^n]; writes
//                             f~^(n+1) = that - dt/2 A[h*]
// Warps 0..7 compute; one thread of warp 8 issues the copies.  Load step L
// brings h plane k0 - zlo + L (and, from step Z on, f~ + Coll of plane
// k0 + L - Z) into ring slot L % RS; full[slot] completes when its bytes
// have landed, empty[slot] when the eight computing warps are done with it.
template <typename R, typename S, bool CORR>
__global__ void __launch_bounds__(kThreads + 32, sizeof(R) == 8 ? 2 : 3)
    k3_adv_staged(const Args3<R> A, const Shape sh) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kMaxSlots;
    R* zc = reinterpret_cast<R*>(smem + sh.zc_off);     // [kc][4] folded z weights of the chunk
    R* hring = reinterpret_cast<R*>(smem + sh.h_off);   // [4 + ahead][ty + 4][nx]
    R* fring = reinterpret_cast<R*>(smem + sh.fc_off);  // [ahead + 1][ty][nx]

    const int tid = threadIdx.x, lane = tid & 31;
    const int nx = A.n[0], ny = A.n[1], nz = A.n[2], ty = sh.ty, rows = ty + 4;
    const int j0 = blockIdx.x * ty;
    const int k0 = blockIdx.y * sh.kc, nit = min(k0 + sh.kc, nz) - k0;
    const bool G = (int)blockIdx.z >= Q3;
    const int a = G ? (int)blockIdx.z - Q3 : (int)blockIdx.z;
    const int cx = c3comp(a, 0), cy = c3comp(a, 1), cz = c3comp(a, 2);
    const bool moving = (cx | cy | cz) != 0;
    // iteration it (plane k0 + it) reads load steps it .. it + Z (its z
    // nodes; the plane itself is step it + zlo) and releases step it
    const int zlo = cz > 0 ? 2 : (cz < 0 ? 1 : 0), Z = cz != 0 ? 3 : 0;
    const int RS = Z + 1 + sh.ahead, FS = sh.ahead + 1, nload = nit + Z;
    const long long N = A.N, NP = A.NP, plane = (long long)nx * ny;
    const unsigned rowb = (unsigned)(nx * sizeof(R));

    if (tid == 0) {
        for (int s = 0; s < RS; ++s) {
            async::bar_init(&full[s], 1);
            async::bar_init(&empty[s], kThreads / 32);
        }
        async::bar_init_fence();
    }
    if (cz != 0) {
        for (int t = tid; t < nit; t += kThreads + 32) {
            const R* f0 = A.ft[2] + kFaceRow * (k0 + t) + (cz > 0 ? 0 : 3);
            R w[3], e[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                w[r] = __ldg(f0 + r);
                e[r] = __ldg(f0 + kFaceRow + r);
            }
            fold4(w, e, R(cz) * __ldg(A.ft[2] + kFaceRow * (k0 + t) + 6), zc + 4 * t);
        }
    }
    __syncthreads();  // barriers initialised, z weights written

    if (tid >= kThreads) {  // the copy warp
        if (lane != 0) return;
        const R* P = G ? (CORR ? A.HGS : A.HG) : (CORR ? A.HS : A.H);
        const R* FCp = G ? A.GC : A.FC;
        const int hrows = moving ? (cy != 0 ? rows : ty) : 0, hr0 = cy != 0 ? 0 : 2;
        int L = 0, slot = 0, round = 0, fslot = 0;  // slot = L % RS, round = L / RS, fslot = (L - Z) % FS
        for (; L < nload; ++L) {
            const int itf = L - Z;
            if (round > 0 && !async::bar_wait(&empty[slot], (round - 1) & 1, A.wait_ns)) break;
            const int frows = itf >= 0 ? min(ty, ny - j0) : 0;
            async::fence_async_shared();
            async::bar_arrive_expect(&full[slot], (unsigned)(hrows + frows) * rowb);
            if (!(A.drop_copy && L == 0)) {  // test hook: the copies of step 0 never start
                // the h rows j0 - 2 + rr, wrapped in y: one copy per run of consecutive rows
                const long long hp = (long long)a * NP + (long long)(k0 - zlo + L + 2) * plane;
                for (int rr = hr0, rend = hr0 + hrows; rr < rend;) {
                    int j = (j0 - 2 + rr) % ny;
                    j = j < 0 ? j + ny : j;
                    const int len = min(rend - rr, ny - j);
                    async::bulk_load(hring + ((size_t)slot * rows + rr) * nx, P + hp + (long long)j * nx,
                                     (unsigned)len * rowb, &full[slot]);
                    rr += len;
                }
                if (frows > 0)
                    async::bulk_load(fring + (size_t)fslot * ty * nx,
                                     FCp + (long long)a * N + (long long)(k0 + itf) * plane + (long long)j0 * nx,
                                     (unsigned)frows * rowb, &full[slot]);
            }
            if (++slot == RS) {
                slot = 0;
                ++round;
            }
            if (itf >= 0 && ++fslot == FS) fslot = 0;
        }
        if (L < nload) {
            // a wait ran out: report, then let the copies of the last RS
            // steps land before the CTA's shared memory is released
            atomicOr(A.werr, 1);
            for (int q = max(0, L - RS); q < L; ++q) async::bar_wait(&full[q % RS], (q / RS) & 1, A.wait_ns);
        }
        return;
    }

    // The computing warps' loop over the chunk's planes.  Ring positions are
    // kept incrementally: s0 = it % RS (the step the iteration releases),
    // sw = (it + Z) % RS and its phase (the step it waits for), sf = it % FS
    // (its f~ + Coll).  body(hz, hc, fcp, kz, qb, pb) updates the thread's
    // cells of plane k0 + it: hz[s] are the planes of the z nodes,
    // hc the plane itself, fcp its f~ + Coll, kz its folded z weights, qb
    // and pb the offsets of plane k0 + it of population a in the unpadded
    // and padded fields.
    auto planes = [&](auto&& body) {
        bool ok = true;
        for (int L = 0; L < Z && ok; ++L) ok = async::bar_wait(&full[L], 0, A.wait_ns);  // Z < RS: first round
        int s0 = 0, sw = Z, sf = 0;
        unsigned ph = 0;
        for (int it = 0; it < nit && ok; ++it) {
            if (!(ok = async::bar_wait(&full[sw], ph, A.wait_ns))) break;
            const int k = k0 + it;
            const R* hz[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) hz[s] = hring + (size_t)(s0 + s < RS ? s0 + s : s0 + s - RS) * rows * nx;
            const R* hc = zlo == 2 ? hz[2] : (zlo == 1 ? hz[1] : hz[0]);
            R kz[4] = {0, 0, 0, 0};
            if (cz != 0) {
#pragma unroll
                for (int s = 0; s < 4; ++s) kz[s] = zc[4 * it + s];
            }
            body(hz, hc, fring + (size_t)sf * ty * nx, kz, (long long)a * N + (long long)k * plane,
                 (long long)a * NP + (long long)(k + 2) * plane);
            __syncwarp();
            if (lane == 0) async::bar_arrive(&empty[s0]);
            s0 = s0 + 1 == RS ? 0 : s0 + 1;
            sf = sf + 1 == FS ? 0 : sf + 1;
            if (++sw == RS) {
                sw = 0;
                ph ^= 1;
            }
        }
        return ok;
    };

    bool ok;
    if constexpr (sizeof(R) == 4) {
        // FP32: two adjacent x cells per thread (nx is even), packed f32x2
        // arithmetic on 8-byte shared loads and 8-byte stores
        static_assert(std::is_same<S, float>::value, "the FP32 staged pass stores FP32 populations");
        using namespace pairmath;
        const int np2 = nx >> 1, i = 2 * (tid % np2), rstep = kThreads / np2, r0 = tid / np2;
        int xp[3] = {0, 0, 0};  // pairs (i-2, i-1), (i, i+1), (i+2, i+3), wrapped in x
        float kl[4] = {0, 0, 0, 0}, kr[4] = {0, 0, 0, 0};
        if (cx != 0) {
            xp[0] = (i - 2 + nx) % nx;
            xp[1] = i;
            xp[2] = (i + 2) % nx;
            axis_fold(A.m[0], i, cx, kl);
            axis_fold(A.m[0], i + 1, cx, kr);
        }
        constexpr int kPairs = kCells / 2;
        float ky[kPairs][4];
#pragma unroll
        for (int m = 0; m < kPairs; ++m) {
            const int j = j0 + r0 + m * rstep;
#pragma unroll
            for (int s = 0; s < 4; ++s) ky[m][s] = 0;
            if (cy != 0 && r0 + m * rstep < ty && j < ny) axis_fold(A.m[1], j, cy, ky[m]);
        }
        ok = planes([&](const R* const* hz, const R* hc, const R* fcp, const R* kz, long long qb, long long pb) {
#pragma unroll
            for (int m = 0; m < kPairs; ++m) {
                const int r = r0 + m * rstep, j = j0 + r;
                if (r >= ty || j >= ny) continue;
                V2 v = bc(0.0f);
                if (cx != 0) {
                    const float* row = hc + (r + 2) * nx;
                    const float2 p0 = *reinterpret_cast<const float2*>(row + xp[0]);
                    const float2 p1 = *reinterpret_cast<const float2*>(row + xp[1]);
                    const float2 p2 = *reinterpret_cast<const float2*>(row + xp[2]);
                    // nodes of the left cell, then of the right one: (i-2..i+1 | i-1..i+2) for
                    // c > 0, (i-1..i+2 | i..i+3) for c < 0
                    const bool pos = cx > 0;
                    const float n0 = pos ? p0.x : p0.y, n1 = pos ? p0.y : p1.x, n2 = pos ? p1.x : p1.y,
                                n3 = pos ? p1.y : p2.x, n4 = pos ? p2.x : p2.y;
                    v = fma2(mk(kl[0], kr[0]), mk(n0, n1), v);
                    v = fma2(mk(kl[1], kr[1]), mk(n1, n2), v);
                    v = fma2(mk(kl[2], kr[2]), mk(n2, n3), v);
                    v = fma2(mk(kl[3], kr[3]), mk(n3, n4), v);
                }
                if (cy != 0) {
                    const float* col = hc + (r + (cy > 0 ? 0 : 1)) * nx + i;
#pragma unroll
                    for (int s = 0; s < 4; ++s)
                        v = fma2(bc(ky[m][s]), V2{*reinterpret_cast<const float2*>(col + s * nx)}, v);
                }
                if (cz != 0) {
                    const int o = (r + 2) * nx + i;
#pragma unroll
                    for (int s = 0; s < 4; ++s) v = fma2(bc(kz[s]), V2{*reinterpret_cast<const float2*>(hz[s] + o)}, v);
                }
                const V2 f{*reinterpret_cast<const float2*>(fcp + r * nx + i)};
                const int jo = j * nx + i;
                if constexpr (CORR) {
                    *reinterpret_cast<float2*>(static_cast<float*>(G ? A.gout : A.fout) + qb + jo) =
                        fma2(bc(-A.hf), v, f).v;
                } else {
                    *reinterpret_cast<float2*>((G ? A.GC : A.FC) + qb + jo) = fma2(bc(-A.hf), v, f).v;
                    *reinterpret_cast<float2*>((G ? A.HGS : A.HS) + pb + jo) = fma2(bc(-A.dt), v, f).v;
                }
            }
        });
    } else {
        // FP64: one cell per thread-slot, column i, rows r0 + m rstep of the tile
        const int i = tid % nx, rstep = kThreads / nx, r0 = tid / nx;
        int xo[4] = {0, 0, 0, 0};
        R kx[4] = {0, 0, 0, 0};
        if (cx != 0) {
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                int c = (i + s + (cx > 0 ? -2 : -1)) % nx;
                xo[s] = c < 0 ? c + nx : c;
            }
            axis_fold(A.m[0], i, cx, kx);
        }
        R ky[kCells][4];
#pragma unroll
        for (int m = 0; m < kCells; ++m) {
            const int j = j0 + r0 + m * rstep;
#pragma unroll
            for (int s = 0; s < 4; ++s) ky[m][s] = 0;
            if (cy != 0 && r0 + m * rstep < ty && j < ny) axis_fold(A.m[1], j, cy, ky[m]);
        }
        ok = planes([&](const R* const* hz, const R* hc, const R* fcp, const R* kz, long long qb, long long pb) {
#pragma unroll
            for (int m = 0; m < kCells; ++m) {
                const int r = r0 + m * rstep, j = j0 + r;
                if (r >= ty || j >= ny) continue;
                R v = 0;
                if (cx != 0) {
                    const R* row = hc + (r + 2) * nx;
                    v = kx[0] * row[xo[0]] + kx[1] * row[xo[1]] + kx[2] * row[xo[2]] + kx[3] * row[xo[3]];
                }
                if (cy != 0) {
                    const R* col = hc + (r + (cy > 0 ? 0 : 1)) * nx + i;
                    v += ky[m][0] * col[0] + ky[m][1] * col[nx] + ky[m][2] * col[2 * nx] + ky[m][3] * col[3 * nx];
                }
                if (cz != 0) {
                    const int o = (r + 2) * nx + i;
                    v += kz[0] * hz[0][o] + kz[1] * hz[1][o] + kz[2] * hz[2][o] + kz[3] * hz[3][o];
                }
                const R f = fcp[r * nx + i];
                const int jo = j * nx + i;
                if constexpr (CORR) {
                    Store<S>::st(static_cast<S*>(G ? A.gout : A.fout) + qb + jo, f - A.hf * v);
                } else {
                    (G ? A.GC : A.FC)[qb + jo] = f - A.hf * v;
                    (G ? A.HGS : A.HS)[pb + jo] = f - A.dt * v;
                }
            }
        });
    }
    if (!ok && lane == 0) atomicOr(A.werr, 1);
}

template <typename R, typename S, bool CORR>
cudaError_t run_staged(const Args3<R>& A, int np, cudaStream_t s) {
    const Shape sh = staged_shape(A.n[0], A.n[2], sizeof(R), A.sshape[0], A.sshape[1], A.sshape[2]);
    if (sh.bytes > kMaxSmem) return cudaErrorInvalidValue;
    {
        cudaError_t e = set_max_smem((const void*)k3_adv_staged<R, S, CORR>, kMaxSmem);
        if (e != cudaSuccess) return e;
    }
    const dim3 g((A.n[1] + sh.ty - 1) / sh.ty, (A.n[2] + sh.kc - 1) / sh.kc, np);
    k3_adv_staged<R, S, CORR><<<g, kThreads + 32, sh.bytes, s>>>(A, sh);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

bool adv3_staged_shape_ok(const int* n, Prec p, int ty, int kc, int ahead) {
    const size_t rs = p == Prec::F64 ? 8 : 4;
    if (ty < 0 || kc < 0 || ahead < 0 || ahead > 12 || kc > 256) return false;
    if (ty > max_rows(n[0], rs)) return false;
    return staged_shape(n[0], n[2], rs, ty, kc, ahead).bytes <= kMaxSmem;
}

void adv3_staged_resolve(const int* n, Prec p, int* ty, int* kc, int* ahead) {
    const Shape sh = staged_shape(n[0], n[2], p == Prec::F64 ? 8 : 4, *ty, *kc, *ahead);
    *ty = sh.ty;
    *kc = sh.kc;
    *ahead = sh.ahead;
}

bool adv3_staged_ok(const int* n, const int* bc, Prec p) {
    const int nx = n[0];
    const size_t rs = p == Prec::F64 ? 8 : 4;
    if (p != Prec::F64 && p != Prec::F32) return false;
    if (bc[0] != LB_BC_PERIODIC || bc[1] != LB_BC_PERIODIC) return false;
    if (nx < 1 || nx > kThreads || kThreads % nx != 0) return false;
    return (nx * rs) % 16 == 0;
}

cudaError_t launch3_adv_staged(Prec p, bool corr, int np, const void* args, cudaStream_t s) {
    if (p == Prec::F64) {
        const auto& A = *static_cast<const Args3<double>*>(args);
        return corr ? run_staged<double, double, true>(A, np, s) : run_staged<double, double, false>(A, np, s);
    }
    const auto& A = *static_cast<const Args3<float>*>(args);
    return corr ? run_staged<float, float, true>(A, np, s) : run_staged<float, float, false>(A, np, s);
}

}  // namespace lbgb
