// k_st_quad.cu -- the ST step (Eq. (ST), Sec. II A, dt = dx = 1) for FP32
// storage on flow grids that are periodic in x with nx a multiple of 4:
// four adjacent cells per thread, every population moved in 16-byte words.
//
//   - each population of the four cells is one 16-byte load;
//   - the collision runs on two packed FP32 pairs (collide_units, K = 1);
//   - every output is an aligned 16-byte store of four cells: a population
//     that moves in x takes the value that crosses the four-cell boundary
//     from the neighbouring lane by one warp shuffle, so only the lanes at
//     a warp's or a row's ends add 4- and 8-byte stores for the cells whose
//     word another warp writes (x wraps periodically).
// Rows at a wall on y (half-way bounce-back) store value by value.  On flow
// grids the base state is rho_r = 1 on every row, so no row offsets enter
// the push.
#include "lb_pair.cuh"

namespace lbgb {

namespace {

using namespace pairmath;

__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st2(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }

// One row of four cells x .. x+3 (interior or periodic in y): collide and
// push.  All 32 lanes of the warp call this together (the shuffles need
// them); `on` marks lanes whose cells exist.
__device__ __forceinline__ void row_quad(const StepArgs<float>& A, int x, int y, bool on, const float4* u) {
    float* fout = static_cast<float*>(A.fout);
    const int yd = y == 0 ? A.ny - 1 : y - 1, yu = y + 1 == A.ny ? 0 : y + 1;
    V2 lo[Q], hi[Q];  // post-collision values of cells (x, x+1) and (x+2, x+3)
    {
        V2 d[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) d[a] = mk(u[a].x, u[a].y);
        collide_units<1>(d, A, lo);
    }
    {
        V2 d[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) d[a] = mk(u[a].z, u[a].w);
        collide_units<1>(d, A, hi);
    }
    const int lane = threadIdx.x & 31;
    // this lane's right neighbour in the row holds cells x+4..x+7
    const bool right_on = __shfl_down_sync(0xffffffffu, on ? 1 : 0, 1) != 0;
    const bool left_end = lane == 0, right_end = lane == 31 || !right_on;
    const int xl = x == 0 ? A.nx - 1 : x - 1;  // periodic x
    const int xr = x + 4 == A.nx ? 0 : x + 4;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int ty = cy(a) > 0 ? yu : (cy(a) < 0 ? yd : y);
        float* row = fout + a * A.plane + (long long)ty * A.pitch;
        // cx(a) is the same on every lane, so the shuffles below run on all 32
        if (cx(a) == 0) {
            if (on) st4(row + x, lo[a].v.x, lo[a].v.y, hi[a].v.x, hi[a].v.y);
        } else if (cx(a) > 0) {
            // cells x..x+3 move to x+1..x+4: the word at x is (x-1's, x, x+1, x+2)
            const float prev = __shfl_up_sync(0xffffffffu, hi[a].v.y, 1);
            if (on) {
                if (!left_end) {
                    st4(row + x, prev, lo[a].v.x, lo[a].v.y, hi[a].v.x);
                } else {
                    row[x + 1] = lo[a].v.x;
                    st2(row + x + 2, lo[a].v.y, hi[a].v.x);
                }
                if (right_end) row[xr] = hi[a].v.y;
            }
        } else {
            // cells x..x+3 move to x-1..x+2: the word at x is (x+1, x+2, x+3, x+4's)
            const float next = __shfl_down_sync(0xffffffffu, lo[a].v.x, 1);
            if (on) {
                if (!right_end) {
                    st4(row + x, lo[a].v.y, hi[a].v.x, hi[a].v.y, next);
                } else {
                    st2(row + x, lo[a].v.y, hi[a].v.x);
                    row[x + 2] = hi[a].v.y;
                }
                if (left_end) row[xl] = lo[a].v.x;
            }
        }
    }
}

// A row at a wall on y (y = 0 or ny - 1): the same collision, every value
// stored on its own; populations leaving through the wall return to their
// cell reversed (half-way bounce-back, Sec. II A).  Only two rows of a grid
// take this path.
__device__ void row_wall(const StepArgs<float>& A, int x, int y, const float4* u) {
    float* fout = static_cast<float*>(A.fout);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        V2 d[Q], p[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) d[a] = h ? mk(u[a].z, u[a].w) : mk(u[a].x, u[a].y);
        collide_units<1>(d, A, p);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int ty = y + cy(a);
            const bool out = ty < 0 || ty >= A.ny;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int xc = x + 2 * h + i;  // source cell
                const float v = i ? p[a].v.y : p[a].v.x;
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
template <int R, int MINB>
__global__ void __launch_bounds__(256, MINB) k_st_quad(const StepArgs<float> A) {
    const int x = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y0 = R * blockIdx.y;
    const bool on = x < A.nx;
    float4 u[R][Q];
    if (on) {
        const float4* p = reinterpret_cast<const float4*>(static_cast<const float*>(A.fin) +
                                                          (long long)y0 * A.pitch + x);
        const long long pl = A.plane / 4, pr = A.pitch / 4;  // in 16-byte words
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
            for (int a = 0; a < Q; ++a) u[r][a] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    const bool walls = A.bcy == LB_BC_WALLS;
    // a block's threads share their rows, so these branches are uniform
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = y0 + r;
        if (r > 0 && y >= A.ny) break;
        if (walls && (y == 0 || y == A.ny - 1)) {
            if (on) row_wall(A, x, y, u[r]);
        } else {
            row_quad(A, x, y, on, u[r]);
        }
    }
}

template <int R, int MINB>
static cudaError_t run_st_quad_r(const StepArgs<float>& A, cudaStream_t s) {
    const int quads = A.nx / 4;
    const int bx = quads >= 256 ? 256 : ((quads + 31) / 32) * 32;
    dim3 grid((quads + bx - 1) / bx, (A.ny + R - 1) / R);
    k_st_quad<R, MINB><<<grid, bx, 0, s>>>(A);
    count_launch();
    return cudaGetLastError();
}

bool st_quad_applies(Prec p, bool thermal, int nx, int bcx) {
    return p == Prec::F32 && !thermal && bcx == LB_BC_PERIODIC && nx % 4 == 0;
}

// One row per thread at three CTAs of 256 threads per SM (80 registers, no
// spill).  At 8192^2 this beat two CTAs (one row, 98 registers; two rows,
// 126 registers) and four CTAs (64 registers, a spill) by 0.4-1.5 %.
cudaError_t launch_st_quad(const void* args, cudaStream_t s) {
    return run_st_quad_r<1, 3>(*static_cast<const StepArgs<float>*>(args), s);
}

}  // namespace lbgb
