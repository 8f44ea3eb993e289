// k_st.cu -- fused collide-and-stream (ST) step, Eq. (ST) of Sec. II A with
// dt = dx = 1, push form: each thread loads the populations of its cell
// (coalesced along x in the [q][y][x] layout), relaxes them with the BGK
// collision plus Guo forcing, and writes each post-collision value to the
// neighbour it streams to.  Walls: half-way bounce-back for f and
// anti-bounce-back through the plate temperature for g,
// g_inv(a)(x) = -g*_a(x) + 2 w_a T_wall.
#include "lb_pair.cuh"

namespace lbgb {

template <typename R, typename S, bool TH>
__global__ void __launch_bounds__(256) k_st(const StepArgs<R> A) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= A.nx) return;
    const S* fin = static_cast<const S*>(A.fin);
    S* fout = static_cast<S*>(A.fout);
    const S* gin = static_cast<const S*>(A.gin);
    S* gout = static_cast<S*>(A.gout);
    const long long c = (long long)y * A.pitch + x;

    R d[Q], e[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) d[a] = Store<S>::ld(fin + a * A.plane + c);
    if (TH) {
#pragma unroll
        for (int a = 0; a < Q; ++a) e[a] = Store<S>::ld(gin + a * A.plane + c);
    }
    const R ro = A.roff[y], to = TH ? A.toff[y] : R(0);
    Cell<R, TH> m;
    m.moments(d, e, A, ro, to);

#pragma unroll
    for (int a = 0; a < Q; ++a) {
        R feqd, F, geqd = 0;
        m.eq(a, A, feqd, F, geqd);
        // right-hand side of Eq. (ST), dt = 1: om = 1/tau~, cf = 1 - 1/(2 tau~)
        const R post = d[a] + A.om * (feqd - d[a]) + A.cf * F;
        R gpost = 0;
        if (TH) gpost = e[a] + A.omg * (geqd - e[a]);
        int tx = x + cx(a), ty = y + cy(a);
        bool out = false;
        R dTw = 0;
        if (tx < 0 || tx >= A.nx) {
            if (A.bcx == LB_BC_PERIODIC) tx = tx < 0 ? tx + A.nx : tx - A.nx;
            else out = true;
        }
        if (ty < 0 || ty >= A.ny) {
            if (A.bcy == LB_BC_PERIODIC) {
                ty = ty < 0 ? ty + A.ny : ty - A.ny;
            } else {
                out = true;
                dTw = ty < 0 ? A.dTb : A.dTt;
            }
        }
        // post and gpost are deviations from the base state of row y; a
        // population streamed to row ty is stored against ty's base state
        if (out) {
            const long long o = inv(a) * A.plane + c;
            Store<S>::st(fout + o, post);
            if (TH) Store<S>::st(gout + o, -gpost + R(2) * wgt<R>(a) * (dTw - to));
        } else {
            const long long o = a * A.plane + (long long)ty * A.pitch + tx;
            Store<S>::st(fout + o, post + wgt<R>(a) * (ro - A.roff[ty]));
            if (TH) Store<S>::st(gout + o, gpost + wgt<R>(a) * (to - A.toff[ty]));
        }
    }
}

// The same step for two adjacent cells per thread with packed FP32 pair
// arithmetic: populations are loaded as pairs (8-byte FP32, 4-byte half2 /
// bfloat162), the collision runs on f32x2 pairs, populations with c_x = 0
// are stored as pairs and the others per cell (their neighbour is shifted by
// one column).
template <typename S, bool TH>
__global__ void __launch_bounds__(256, TH ? 2 : 4) k_st_pair(const StepArgs<float> A) {
    using namespace pairmath;
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y;
    if (x >= A.nx) return;
    const bool two = x + 1 < A.nx;
    const S* fin = static_cast<const S*>(A.fin);
    S* fout = static_cast<S*>(A.fout);
    const S* gin = static_cast<const S*>(A.gin);
    S* gout = static_cast<S*>(A.gout);
    const long long c = (long long)y * A.pitch + x;
    auto ld = [&](const S* p) { return two ? PairIO<S>::ld(p) : bc(Store<S>::ld(p)); };
    V2 d[Q], e[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) d[a] = ld(fin + a * A.plane + c);
    if (TH) {
#pragma unroll
        for (int a = 0; a < Q; ++a) e[a] = ld(gin + a * A.plane + c);
    }
    const float ro = A.roff[y], to = TH ? A.toff[y] : 0.0f;
    PairCell<TH> m;
    m.build(d, e, A, ro, to);
    // Interior pairs (both cells and all their neighbours inside the grid)
    // stream to fixed offsets with no wrap or wall test.
    if (x >= 1 && x + 2 < A.nx && y >= 1 && y + 1 < A.ny) {
        const float rdn = A.roff[y - 1], rup = A.roff[y + 1];
        const float tdn = TH ? A.toff[y - 1] : 0.0f, tup = TH ? A.toff[y + 1] : 0.0f;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const float w = wgt<float>(a);
            const float rt = cy(a) > 0 ? rup : (cy(a) < 0 ? rdn : ro);
            const float tt = cy(a) > 0 ? tup : (cy(a) < 0 ? tdn : to);
            const V2 post = fma2(bc(A.om), m.feqd[a] - d[a], fma2(bc(A.cf), m.F[a], d[a])) + bc(w * (ro - rt));
            V2 gpost = bc(0.0f);
            if (TH) gpost = fma2(bc(A.omg), m.geqd[a] - e[a], e[a]) + bc(w * (to - tt));
            const long long o = a * A.plane + c + (long long)cy(a) * A.pitch + cx(a);
            if (cx(a) == 0) {
                PairIO<S>::st(fout + o, post);
                if (TH) PairIO<S>::st(gout + o, gpost);
            } else {
                Store<S>::st(fout + o, post.v.x);
                Store<S>::st(fout + o + 1, post.v.y);
                if (TH) {
                    Store<S>::st(gout + o, gpost.v.x);
                    Store<S>::st(gout + o + 1, gpost.v.y);
                }
            }
        }
        return;
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const V2 post = fma2(bc(A.om), m.feqd[a] - d[a], fma2(bc(A.cf), m.F[a], d[a]));
        V2 gpost = bc(0.0f);
        if (TH) gpost = fma2(bc(A.omg), m.geqd[a] - e[a], e[a]);
        const float w = wgt<float>(a);
        int ty = y + cy(a);
        bool outy = false;
        float dTw = 0.0f;
        if (ty < 0 || ty >= A.ny) {
            if (A.bcy == LB_BC_PERIODIC) {
                ty = ty < 0 ? ty + A.ny : ty - A.ny;
            } else {
                outy = true;
                dTw = ty < 0 ? A.dTb : A.dTt;
            }
        }
        if (cx(a) == 0) {
            // both cells stream to the same row: one pair store
            long long o;
            V2 fv, gv;
            if (outy) {
                o = inv(a) * A.plane + c;
                fv = post;
                gv = bc(2.0f * w * (dTw - to)) - gpost;
            } else {
                o = a * A.plane + (long long)ty * A.pitch + x;
                fv = post + bc(w * (ro - A.roff[ty]));
                if (TH) gv = gpost + bc(w * (to - A.toff[ty]));
            }
            if (two) {
                PairIO<S>::st(fout + o, fv);
                if (TH) PairIO<S>::st(gout + o, gv);
            } else {
                Store<S>::st(fout + o, fv.v.x);
                if (TH) Store<S>::st(gout + o, gv.v.x);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                if (i == 1 && !two) break;
                const float pv = i ? post.v.y : post.v.x;
                const float gp = i ? gpost.v.y : gpost.v.x;
                int tx = x + i + cx(a);
                bool out = outy;
                if (tx < 0 || tx >= A.nx) {
                    if (A.bcx == LB_BC_PERIODIC) tx = tx < 0 ? tx + A.nx : tx - A.nx;
                    else out = true;
                }
                if (out) {
                    const long long o = inv(a) * A.plane + c + i;
                    Store<S>::st(fout + o, pv);
                    if (TH) Store<S>::st(gout + o, -gp + 2.0f * w * (dTw - to));
                } else {
                    const long long o = a * A.plane + (long long)ty * A.pitch + tx;
                    Store<S>::st(fout + o, pv + w * (ro - A.roff[ty]));
                    if (TH) Store<S>::st(gout + o, gp + w * (to - A.toff[ty]));
                }
            }
        }
    }
}

// 16-bit flow grids: the kernel waits on memory latency (about half of its
// DRAM peak at 32 warps per SM), so each thread takes two rows and issues the
// second row's loads (kept as packed 16-bit pairs, one register each) before
// the first row's arithmetic.  The per-row arithmetic and stores are those of
// k_st_pair without the thermal populations.
template <typename S>
__device__ __forceinline__ pairmath::V2 cvt_pair(unsigned u, bool two);
template <>
__device__ __forceinline__ pairmath::V2 cvt_pair<__half>(unsigned u, bool two) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&u));
    const pairmath::V2 v{make_float2(f.x * (1.0f / kF16Scale), f.y * (1.0f / kF16Scale))};
    return two ? v : pairmath::bc(v.v.x);
}
template <>
__device__ __forceinline__ pairmath::V2 cvt_pair<__nv_bfloat16>(unsigned u, bool two) {
    const pairmath::V2 v{__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u))};
    return two ? v : pairmath::bc(v.v.x);
}

template <typename S>
__device__ __forceinline__ void st_pair_row_flow(const StepArgs<float>& A, const int x, const int y, const bool two,
                                                 const pairmath::V2* d) {
    using namespace pairmath;
    S* fout = static_cast<S*>(A.fout);
    const long long c = (long long)y * A.pitch + x;
    const float ro = A.roff[y];
    PairCell<false> m;
    m.build(d, d, A, ro, 0.0f);
    if (x >= 1 && x + 2 < A.nx && y >= 1 && y + 1 < A.ny) {
        const float rdn = A.roff[y - 1], rup = A.roff[y + 1];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const float w = wgt<float>(a);
            const float rt = cy(a) > 0 ? rup : (cy(a) < 0 ? rdn : ro);
            const V2 post = fma2(bc(A.om), m.feqd[a] - d[a], fma2(bc(A.cf), m.F[a], d[a])) + bc(w * (ro - rt));
            const long long o = a * A.plane + c + (long long)cy(a) * A.pitch + cx(a);
            if (cx(a) == 0) {
                PairIO<S>::st(fout + o, post);
            } else {
                Store<S>::st(fout + o, post.v.x);
                Store<S>::st(fout + o + 1, post.v.y);
            }
        }
        return;
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const V2 post = fma2(bc(A.om), m.feqd[a] - d[a], fma2(bc(A.cf), m.F[a], d[a]));
        const float w = wgt<float>(a);
        int ty = y + cy(a);
        bool outy = false;
        if (ty < 0 || ty >= A.ny) {
            if (A.bcy == LB_BC_PERIODIC) ty = ty < 0 ? ty + A.ny : ty - A.ny;
            else outy = true;
        }
        if (cx(a) == 0) {
            long long o;
            V2 fv;
            if (outy) {
                o = inv(a) * A.plane + c;
                fv = post;
            } else {
                o = a * A.plane + (long long)ty * A.pitch + x;
                fv = post + bc(w * (ro - A.roff[ty]));
            }
            if (two) PairIO<S>::st(fout + o, fv);
            else Store<S>::st(fout + o, fv.v.x);
        } else {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                if (i == 1 && !two) break;
                const float pv = i ? post.v.y : post.v.x;
                int tx = x + i + cx(a);
                bool out = outy;
                if (tx < 0 || tx >= A.nx) {
                    if (A.bcx == LB_BC_PERIODIC) tx = tx < 0 ? tx + A.nx : tx - A.nx;
                    else out = true;
                }
                if (out) Store<S>::st(fout + inv(a) * A.plane + c + i, pv);
                else Store<S>::st(fout + a * A.plane + (long long)ty * A.pitch + tx, pv + w * (ro - A.roff[ty]));
            }
        }
    }
}

// Three CTAs per SM (80 registers): measured faster than four with the
// 64-register cap, which spills.
template <typename S>
__global__ void __launch_bounds__(256, 3) k_st_pair_rows(const StepArgs<float> A) {
    using namespace pairmath;
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = 2 * blockIdx.y;
    if (x >= A.nx) return;
    const bool two = x + 1 < A.nx, second = y + 1 < A.ny;
    // a pair load at an odd last column reads one element of the row's
    // padding (the pitch is a multiple of 32), which cvt_pair then drops
    const unsigned* p = reinterpret_cast<const unsigned*>(static_cast<const S*>(A.fin) + (long long)y * A.pitch + x);
    const long long pl = A.plane / 2, pr = A.pitch / 2;  // in 32-bit words
    unsigned r0[Q], r1[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) r0[a] = __ldg(p + a * pl);
    if (second) {
#pragma unroll
        for (int a = 0; a < Q; ++a) r1[a] = __ldg(p + a * pl + pr);
    }
    V2 d[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) d[a] = cvt_pair<S>(r0[a], two);
    st_pair_row_flow<S>(A, x, y, two, d);
    if (second) {
#pragma unroll
        for (int a = 0; a < Q; ++a) d[a] = cvt_pair<S>(r1[a], two);
        st_pair_row_flow<S>(A, x, y + 1, two, d);
    }
}

template <typename R, typename S, bool TH>
static cudaError_t run_st(const void* vargs, cudaStream_t s) {
    const StepArgs<R>& A = *static_cast<const StepArgs<R>*>(vargs);
    if constexpr (sizeof(R) == 4 && sizeof(S) == 2 && !TH) {
        // 16-bit flow grids: one thread per two cells of two rows
        const int half = (A.nx + 1) / 2;
        int bx = half >= 256 ? 256 : ((half + 31) / 32) * 32;
        dim3 grid((half + bx - 1) / bx, (A.ny + 1) / 2);
        k_st_pair_rows<S><<<grid, bx, 0, s>>>(A);
    } else if constexpr (sizeof(R) == 4) {
        // packed pairs: one thread per two cells
        const int half = (A.nx + 1) / 2;
        int bx = half >= 256 ? 256 : ((half + 31) / 32) * 32;
        dim3 grid((half + bx - 1) / bx, A.ny);
        k_st_pair<S, TH><<<grid, bx, 0, s>>>(A);
    } else {
        int bx = A.nx >= 256 ? 256 : ((A.nx + 31) / 32) * 32;
        dim3 grid((A.nx + bx - 1) / bx, A.ny);
        k_st<R, S, TH><<<grid, bx, 0, s>>>(A);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_st(Prec p, bool th, const void* args, cudaStream_t s) {
    switch (p) {
        case Prec::F64: return th ? run_st<double, double, true>(args, s) : run_st<double, double, false>(args, s);
        case Prec::F32: return th ? run_st<float, float, true>(args, s) : run_st<float, float, false>(args, s);
        case Prec::F16: return th ? run_st<float, __half, true>(args, s) : run_st<float, __half, false>(args, s);
        case Prec::BF16:
            return th ? run_st<float, __nv_bfloat16, true>(args, s) : run_st<float, __nv_bfloat16, false>(args, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbgb
