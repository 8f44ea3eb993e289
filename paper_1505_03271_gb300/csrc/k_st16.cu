// k_st16.cu -- the ST step (Eq. (ST), Sec. II A, dt = dx = 1) for 16-bit
// deviation storage on flow grids that are periodic in x with nx a multiple
// of 4: four adjacent cells of two rows per thread, every population moved
// in 64-bit words.
//
// Why: with 16-bit storage a pair of cells is only 4 bytes, so the pair
// kernel's loads fetch 128 bytes per warp instruction and the shifted
// populations are written as single 16-bit values; the kernel is then
// bound by the number of memory requests in flight, not by DRAM.  Here
//   - each population of four cells is one 8-byte load (256 bytes per warp
//     instruction), both rows' loads issued before any arithmetic;
//   - the collision runs on packed FP32 pairs in storage units, with the
//     even and odd parts of each pair of opposite populations shared;
//   - every output is an aligned 8-byte store of four cells: the populations
//     that move in x are realigned across lanes with one warp shuffle (the
//     value that crosses a four-cell boundary), so only the lanes at a
//     warp's or a row's ends add 2- or 4-byte stores for the cells whose
//     word another warp writes.
// Rows at a wall on y (half-way bounce-back) store value by value; interior
// and periodic rows take the word path.  On flow grids the base state is
// rho_r = 1 on every row, so no row offsets enter the push.
#include "lb_pair.cuh"

namespace lbgb {

namespace {

using namespace pairmath;

template <typename S> struct Half;
template <> struct Half<__half> {
    static constexpr int kScale = int(kF16Scale);  // storage units per deviation unit
    // two stored values as floats in storage units (no rescaling)
    __device__ static V2 raw(unsigned u) { return {__half22float2(*reinterpret_cast<const __half2*>(&u))}; }
    __device__ static unsigned raw_pack(V2 v) {
        const __half2 h = __floats2half2_rn(v.v.x, v.v.y);
        return *reinterpret_cast<const unsigned*>(&h);
    }
    // two values -> one 32-bit word (low half = first), FP16 holds x * 2^12
    __device__ static unsigned pack(V2 v) {
        const __half2 h = __floats2half2_rn(v.v.x * kF16Scale, v.v.y * kF16Scale);
        return *reinterpret_cast<const unsigned*>(&h);
    }
    __device__ static V2 unpack(unsigned u) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&u));
        return mk(f.x * (1.0f / kF16Scale), f.y * (1.0f / kF16Scale));
    }
};
template <> struct Half<__nv_bfloat16> {
    static constexpr int kScale = 1;
    __device__ static V2 raw(unsigned u) { return {__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u))}; }
    __device__ static unsigned raw_pack(V2 v) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.v.x, v.v.y);
        return *reinterpret_cast<const unsigned*>(&h);
    }
    __device__ static unsigned pack(V2 v) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.v.x, v.v.y);
        return *reinterpret_cast<const unsigned*>(&h);
    }
    __device__ static V2 unpack(unsigned u) {
        return {__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u))};
    }
};

__device__ __forceinline__ void st16(void* base, long long i, unsigned short v) {
    reinterpret_cast<unsigned short*>(base)[i] = v;
}
__device__ __forceinline__ void st32(void* base, long long i, unsigned v) {
    *reinterpret_cast<unsigned*>(reinterpret_cast<unsigned short*>(base) + i) = v;
}
__device__ __forceinline__ void st64(void* base, long long i, unsigned lo, unsigned hi) {
    *reinterpret_cast<uint2*>(reinterpret_cast<unsigned short*>(base) + i) = make_uint2(lo, hi);
}

// One row of four cells x .. x+3 (interior or periodic in y): collide and
// push.  u[a] holds population a of the four cells as two words (cells
// x, x+1 and x+2, x+3).  All 32 lanes of the warp call this together (the
// shuffles need them); `on` marks lanes whose cells exist.
template <typename S>
__device__ __forceinline__ void row_words(const StepArgs<float>& A, int x, int y, bool on, const uint2* u) {
    void* fout = A.fout;
    const int yd = y == 0 ? A.ny - 1 : y - 1, yu = y + 1 == A.ny ? 0 : y + 1;
    unsigned lo[Q], hi[Q];  // post-collision words of cells (x, x+1) and (x+2, x+3)
    {
        V2 d[Q], p[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) d[a] = Half<S>::raw(u[a].x);
        collide_units<Half<S>::kScale>(d, A, p);
#pragma unroll
        for (int a = 0; a < Q; ++a) lo[a] = Half<S>::raw_pack(p[a]);
    }
    {
        V2 d[Q], p[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) d[a] = Half<S>::raw(u[a].y);
        collide_units<Half<S>::kScale>(d, A, p);
#pragma unroll
        for (int a = 0; a < Q; ++a) hi[a] = Half<S>::raw_pack(p[a]);
    }
    const int lane = threadIdx.x & 31;
    // this lane's right neighbour in the row holds cells x+4..x+7
    const bool right_on = __shfl_down_sync(0xffffffffu, on ? 1 : 0, 1) != 0;
    const bool left_end = lane == 0, right_end = lane == 31 || !right_on;
    const int xl = x == 0 ? A.nx - 1 : x - 1;      // periodic x
    const int xr = x + 4 == A.nx ? 0 : x + 4;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int ty = cy(a) > 0 ? yu : (cy(a) < 0 ? yd : y);
        const long long row = a * A.plane + (long long)ty * A.pitch;
        // cx(a) is the same on every lane, so the shuffles below run on all 32
        if (cx(a) == 0) {
            if (on) st64(fout, row + x, lo[a], hi[a]);
        } else if (cx(a) > 0) {
            // cells x..x+3 move to x+1..x+4; word at x = (x-1's last, x, x+1, x+2)
            const unsigned prev = __shfl_up_sync(0xffffffffu, hi[a], 1);
            const unsigned w0 = __byte_perm(prev, lo[a], 0x5432);
            const unsigned w1 = __byte_perm(lo[a], hi[a], 0x5432);
            if (on) {
                if (!left_end) {
                    st64(fout, row + x, w0, w1);
                } else {
                    st16(fout, row + x + 1, (unsigned short)(lo[a] & 0xffffu));
                    st32(fout, row + x + 2, w1);
                }
                if (right_end) st16(fout, row + xr, (unsigned short)(hi[a] >> 16));
            }
        } else {
            // cells x..x+3 move to x-1..x+2; word at x = (x+1, x+2, x+3, x+4's first)
            const unsigned next = __shfl_down_sync(0xffffffffu, lo[a], 1);
            const unsigned w0 = __byte_perm(lo[a], hi[a], 0x5432);
            const unsigned w1 = __byte_perm(hi[a], next, 0x5432);
            if (on) {
                if (!right_end) {
                    st64(fout, row + x, w0, w1);
                } else {
                    st32(fout, row + x, w0);
                    st16(fout, row + x + 2, (unsigned short)(hi[a] >> 16));
                }
                if (left_end) st16(fout, row + xl, (unsigned short)(lo[a] & 0xffffu));
            }
        }
    }
}

// A row at a wall on y (y = 0 or ny - 1): the same collision, every value
// stored on its own; populations leaving through the wall return to their
// cell reversed (half-way bounce-back, Sec. II A).  Only two rows of a grid
// take this path.
template <typename S>
__device__ void row_wall(const StepArgs<float>& A, int x, int y, const uint2* u) {
    unsigned short* fout = static_cast<unsigned short*>(A.fout);
    const float ro = A.roff[y];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        V2 d[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) d[a] = Half<S>::unpack(h ? u[a].y : u[a].x);
        PairCell<false> m;
        m.build(d, d, A, ro, 0.0f);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const V2 post = fma2(bc(A.om), m.feqd[a] - d[a], fma2(bc(A.cf), m.F[a], d[a]));
            const int ty = y + cy(a);
            const bool out = ty < 0 || ty >= A.ny;
            const float shift = out ? 0.0f : wgt<float>(a) * (ro - A.roff[out ? y : ty]);
            const unsigned word = Half<S>::pack(post + bc(shift));
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int xc = x + 2 * h + i;  // source cell
                const unsigned short v = (unsigned short)(i ? word >> 16 : word & 0xffffu);
                if (out) {
                    fout[inv(a) * A.plane + (long long)y * A.pitch + xc] = v;
                } else {
                    int tx = xc + cx(a);
                    tx = tx < 0 ? tx + A.nx : (tx >= A.nx ? tx - A.nx : tx);
                    fout[a * A.plane + (long long)ty * A.pitch + tx] = v;
                }
            }
        }
    }
}

}  // namespace

// R rows per thread (y = R blockIdx.y ...), four cells each; all rows'
// loads are issued before the first row's arithmetic.
template <typename S, int R, int MINB>
__global__ void __launch_bounds__(256, MINB) k_st16_quad(const StepArgs<float> A) {
    const int x = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y0 = R * blockIdx.y;
    const bool on = x < A.nx;
    const S* fin = static_cast<const S*>(A.fin);
    uint2 u[R][Q];
    if (on) {
        const uint2* p = reinterpret_cast<const uint2*>(fin + (long long)y0 * A.pitch + x);
        const long long pl = A.plane / 4, pr = A.pitch / 4;  // in 8-byte words
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r == 0 || y0 + r < A.ny) {
#pragma unroll
                for (int a = 0; a < Q; ++a) u[r][a] = __ldg(p + a * pl + r * pr);
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int a = 0; a < Q; ++a) u[r][a] = make_uint2(0u, 0u);
    }
    const bool walls = A.bcy == LB_BC_WALLS;
    // a block's threads share their rows, so these branches are uniform
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = y0 + r;
        if (r > 0 && y >= A.ny) break;
        if (walls && (y == 0 || y == A.ny - 1)) {
            if (on) row_wall<S>(A, x, y, u[r]);
        } else {
            row_words<S>(A, x, y, on, u[r]);
        }
    }
}

template <typename S, int R, int MINB>
static cudaError_t run_st16_r(const StepArgs<float>& A, cudaStream_t s) {
    const int quads = A.nx / 4;
    const int bx = quads >= 256 ? 256 : ((quads + 31) / 32) * 32;
    dim3 grid((quads + bx - 1) / bx, (A.ny + R - 1) / R);
    k_st16_quad<S, R, MINB><<<grid, bx, 0, s>>>(A);
    count_launch();
    return cudaGetLastError();
}

// Two rows per thread at three CTAs of 256 threads per SM (80 registers, a
// 48-byte spill).  At 8192^2 this beats two CTAs at 128 registers by 16 %
// (FP16) and 14 % (BF16): the latency of the loads and of the f32x2
// dependency chains is hidden by 24 warps per SM instead of 16.  One row per
// thread, three or four rows, and four CTAs per SM were slower.
template <typename S>
static cudaError_t run_st16(const void* vargs, cudaStream_t s) {
    return run_st16_r<S, 2, 3>(*static_cast<const StepArgs<float>*>(vargs), s);
}

bool st16_applies(Prec p, bool thermal, int nx, int bcx) {
    return (p == Prec::F16 || p == Prec::BF16) && !thermal && bcx == LB_BC_PERIODIC && nx % 4 == 0;
}

cudaError_t launch_st16(Prec p, const void* args, cudaStream_t s) {
    if (p == Prec::F16) return run_st16<__half>(args, s);
    if (p == Prec::BF16) return run_st16<__nv_bfloat16>(args, s);
    return cudaErrorInvalidValue;
}

}  // namespace lbgb
