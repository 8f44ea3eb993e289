// lb_internal.cuh -- types and device helpers shared by the library's CUDA
// translation units (not part of the public ABI; see include/lb.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/lb.h"

namespace lbgb {

constexpr int Q = 9;

// D2Q9 lattice in the order of include/lb.h (Sec. II, D3Q19 reduced to 2-D).
__host__ __device__ constexpr int cx(int a) {
    return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy(int a) {
    return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0);
}
__host__ __device__ constexpr int inv(int a) {
    return a == 0 ? 0 : (a <= 4 ? ((a + 1) & 3) + 1 : ((a - 3) & 3) + 5);
}
template <typename R>
__host__ __device__ constexpr R wgt(int a) {
    return a == 0 ? R(4) / R(9) : (a <= 4 ? R(1) / R(9) : R(1) / R(36));
}
static_assert(inv(1) == 3 && inv(3) == 1 && inv(2) == 4 && inv(4) == 2, "inv");
static_assert(inv(5) == 7 && inv(7) == 5 && inv(6) == 8 && inv(8) == 6 && inv(0) == 0, "inv");

// ---- storage and arithmetic frame ----
// The state holds f - w rho_r(y) and g - w T_r(y): deviations from a per-row
// base state, which on a grid with plates is the hydrostatic, conductive RB
// state (barometric rho_r, linear T_r) and elsewhere rho_r = 1, T_r = T0.
// Kernels compute in the same frame: moments add the row's rho_r and T_r,
// and the y flux divergence of the base state itself enters as a per-row
// constant (QUICK is linear, so A[h' + w ref] = A[h'] + w A[ref]).  Near the
// plates every quantity the kernels round is then small, so the wall
// temperature gradient (the Nusselt number) keeps its digits in FP32
// arithmetic and in 16-bit storage.  Ghost rows extend the base state by the
// wall's own symmetry (rho_r even, T_r odd about T_wall), which turns the
// wall rules into h'_a(x_-k) = h'_inv(a)(x_k) for f and -h'_inv(a)(x_k) for g.
template <typename S> struct Store;
template <> struct Store<double> {
    __device__ static double ld(const double* p) { return __ldg(p); }
    __device__ static void st(double* p, double v) { *p = v; }
};
template <> struct Store<float> {
    __device__ static float ld(const float* p) { return __ldg(p); }
    __device__ static void st(float* p, float v) { *p = v; }
};
// FP16 holds the deviation times 2^12: the deviations are O(1e-1) at most,
// so the scale keeps the small ones (buoyancy and wall increments of 1e-8)
// out of FP16's subnormal range, where the spacing is 6e-8.  The largest
// storable deviation is 65504 / 4096 = 16.  Powers of two scale exactly.
constexpr float kF16Scale = 4096.0f;
template <> struct Store<__half> {
    __device__ static float ld(const __half* p) { return __half2float(__ldg(p)) * (1.0f / kF16Scale); }
    __device__ static void st(__half* p, float v) { *p = __float2half_rn(v * kF16Scale); }
};
template <> struct Store<__nv_bfloat16> {
    __device__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    __device__ static void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// Per-axis metric in compute precision: for faces k = 0..n the QUICK
// weights wp[0..2][k] (nodes k-2, k-1, k; used when c > 0) and wm[0..2][k]
// (nodes k-1, k, k+1; c < 0); then 1/dx for cells 0..n-1.
// Layout: [6][n + 1] followed by [n].
template <typename R>
struct AxisMetric {
    const R* m;
    int n1;  // n + 1
    __device__ R wp(int r, int k) const { return __ldg(m + r * n1 + k); }
    __device__ R wm(int r, int k) const { return __ldg(m + (3 + r) * n1 + k); }
    __device__ R invd(int i) const { return __ldg(m + 6 * n1 + i); }
    __device__ R row(int r, int k) const { return __ldg(m + r * n1 + k); }  // r = 0..2 wp, 3..5 wm
};

// Parameters of one step, in compute precision R.
template <typename R>
struct StepArgs {
    const void* fin;
    void* fout;
    const void* gin;
    void* gout;
    int nx, ny, pitch;
    long long plane;  // pitch * ny
    int bcx, bcy;
    AxisMetric<R> mx, my;
    int stages;             // 2: Heun corrector (Eq. (semi-heun)); 1: the predictor is the new state
    R dt, om, omh, cf, hf;  // dt/tau~, dt/(2 tau~), dt (1 - dt/(2 tau~)), dt/2 (Euler: dt/tau, 0, dt, 0)
    R hF;                   // force part of the advected field: dt/2 (1 - dt/(2 tau~)) (Euler: 0)
    R omg, omgh;            // dt/tau~_g, dt/(2 tau~_g)
    R ax, ay, bg;           // external acceleration, beta * grav
    R dTb, dTt;             // T_bot - T0, T_top - T0
    R T0;                   // reference temperature
    R rhobd[4];             // imposed face density - 1 of LB_BC_DENSITY axes: x0, x1, y0, y1
    const R* toff;          // per row: T_r - T0 (thermal grids)
    const R* roff;          // per row: rho_r - 1
    const R* dref;          // [4][ny]: y flux divergence of rho_r (c_y > 0, < 0), of T_r (> 0, < 0)
    const float* rowtab;    // [ny][20] per-row y data of the paired kernels (FP32 grids)
    const float* coltab;    // [nx][20] per-column-pair x data of the paired tile kernel
    float* xh;              // split schedule: h* of the step, [NQ][ny][pitch] (FP32)
    float* xfc;             // split schedule: f~ + Coll - dt/2 A[h^n], same layout
};

// Wrap or reject a global index on one axis: periodic axes wrap, wall axes
// reject indices outside the domain.
__device__ __forceinline__ bool map_axis(int g, int n, int bc, int& out) {
    if (g >= 0 && g < n) {
        out = g;
        return true;
    }
    if (bc == LB_BC_PERIODIC) {
        int r = g % n;
        out = r < 0 ? r + n : r;
        return true;
    }
    return false;
}

// Macroscopic moments of one cell from base-state deviations d (and e) of a
// row with references rho_r = 1 + ro, T_r = T0 + to:
// rho = rho_r + sum d, T = T_r + sum e, a = (ax, ay + beta grav (T - T0)),
// u = sum c d / rho + dt/2 a (Sec. II B 4).
template <typename R, bool TH>
struct Cell {
    R rp, rho, ux, uy, Td, T, ay;  // rp = rho - rho_r, Td = T - T_r: kept unrounded
    __device__ __forceinline__ void moments(const R* d, const R* e, const StepArgs<R>& A, R ro, R to) {
        R r = 0, jx = 0, jy = 0;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            r += d[a];
            jx += R(cx(a)) * d[a];
            jy += R(cy(a)) * d[a];
        }
        Td = 0;
        if (TH) {
#pragma unroll
            for (int a = 0; a < Q; ++a) Td += e[a];
        }
        rp = r;
        rho = (R(1) + ro) + r;
        const R dT0 = to + Td;  // T - T0
        T = A.T0 + dT0;
        ay = A.ay + (TH ? A.bg * dT0 : R(0));
        R ir = R(1) / rho;
        ux = jx * ir + A.hf * A.ax;
        uy = jy * ir + A.hf * ay;
    }
    // f_eq - w rho_r, Guo force F (Eq. (F2)) and, if thermal, g_eq - w T_r.
    __device__ __forceinline__ void eq(int a, const StepArgs<R>& A, R& feqd, R& F, R& geqd) const {
        const R w = wgt<R>(a);
        const R cu = R(cx(a)) * ux + R(cy(a)) * uy;
        const R uu = ux * ux + uy * uy;
        const R poly = R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu;
        feqd = w * (rp + rho * poly);
        const R ca = R(cx(a)) * A.ax + R(cy(a)) * ay;
        const R ua = ux * A.ax + uy * ay;
        F = w * rho * (R(3) * (ca - ua) + R(9) * cu * ca);
        if (TH) geqd = w * (Td + T * poly);
    }
};

// y flux divergence of the base state for population a at row gy (zero for
// c_y = 0): c_y w_a (Phi_n - Phi_s)[ref] / dy.
template <typename R, int a>
__device__ __forceinline__ R ref_flux(const StepArgs<R>& A, int gy, bool thermal) {
    if constexpr (cy(a) == 0) {
        return R(0);
    } else {
        const int k = (thermal ? 2 : 0) + (cy(a) > 0 ? 0 : 1);
        return R(cy(a)) * wgt<R>(a) * __ldg(A.dref + k * A.ny + gy);
    }
}

}  // namespace lbgb

// ---- launchers (implemented in the kernel translation units) ----
namespace lbgb {
enum class Prec { F64, F32, F16, BF16 };

cudaError_t launch_st(Prec p, bool thermal, const void* args, cudaStream_t s);
cudaError_t launch_fv(Prec p, bool thermal, const void* args, int shape, cudaStream_t s);
// One request of a batched FV launch: its step parameters, both buffers
// of each population set, the parity of its current state at step 0 of the
// launch sequence and how many steps it still has to take.
template <typename R>
struct BatchReq {
    StepArgs<R> args;
    void* f[2];
    void* g[2];
    int parity;
    int remaining;
};
// tiles[b] = (request, tile x, tile y, 0); CTAs beyond *ntiles exit
cudaError_t launch_fv_batched(Prec p, bool thermal, const void* reqs, const int4* tiles, const int* ntiles,
                              int capacity, int k, cudaStream_t s);
void tile_shape(Prec p, bool thermal, int* tx, int* ty);
// y-marching FV kernel: strips of march_width() output columns, `chunk` rows per CTA
cudaError_t launch_fv_march(Prec p, bool thermal, const void* args, int chunk, cudaStream_t s);
int march_width(Prec p, bool thermal);
size_t march_smem(Prec p, bool thermal);
// paired-column marching FV kernel (FP32 arithmetic, x-periodic grids only)
cudaError_t launch_fv_pair(Prec p, bool thermal, const void* args, int chunk, cudaStream_t s);
int pair_width();
size_t pair_smem(bool thermal);
// paired tile kernel: shape 0 = 32 x 16, 16 = 16 x 16 (x-periodic, FP32 arithmetic)
cudaError_t launch_fv_ptile(Prec p, bool thermal, const void* args, int shape, cudaStream_t s);
// split paired schedule: two launches per step (collision + predictor, corrector),
// h* and f~ + Coll - dt/2 A[h^n] through the xh / xfc buffers
cudaError_t launch_fv_split(Prec p, bool thermal, const void* args, int shape, cudaStream_t s);
// batched paired tile (32 x 16) over a request table, as launch_fv_batched
cudaError_t launch_fv_ptile_batched(Prec p, bool thermal, const void* reqs, const int4* tiles, const int* ntiles,
                                    int capacity, int k, cudaStream_t s);

struct AuxArgs {
    const void* f;  // state buffers (deviation storage)
    const void* g;
    int nx, ny, pitch;
    long long plane;
    double dt, ax, ay, bg, T0;
    const double* toff; // per-row storage offset of g (thermal grids)
    const double* roff; // per-row storage offset of f
    const double* dxv;  // cell widths x (nx), FP64
    const double* dyv;  // cell widths y (ny)
    const double* xc;   // centres x
    const double* yc;   // centres y
};

// Moments of every cell into out[4][ny][nx] (rho, ux, uy, T), FP64.
cudaError_t launch_moments(Prec p, bool thermal, const AuxArgs& a, double* out, cudaStream_t s);
// Block partial sums of the reduction quantities (kRed values) then a final
// fixed-order sum into out[kRed].
constexpr int kRed = 10;
cudaError_t launch_reduce(Prec p, bool thermal, const AuxArgs& a, double* partial, int nblocks,
                          double* out, cudaStream_t s);
int reduce_blocks(int nx, int ny);

// Populations FP64 host layout [9][ny][nx] (device copy) -> storage, and back.
// Stored value = value - w (off + rowoff[y]); rowoff may be NULL.
cudaError_t launch_pack(Prec p, const double* src, void* dst, int nx, int ny, int pitch,
                        long long plane, double off, const double* rowoff, cudaStream_t s);
// Window [9][h][w] starting at (x0, y0), indices wrapping modulo nx, ny.
cudaError_t launch_unpack(Prec p, const void* src, double* dst, int nx, int ny, int pitch,
                          long long plane, double off, const double* rowoff, int x0, int y0, int w,
                          int h, cudaStream_t s);

struct InitArgs {
    void* f;
    void* g;
    int nx, ny, pitch;
    long long plane;
    int kind, mode;
    double u0, amp;
    unsigned long long seed;
    double lx, ly;
    double dt, ax, ay, bg, T0, Tb, Tt;
    double rho_norm;
    const double* toff;
    const double* roff;
    const double* xc;
    const double* yc;
    const double* fields;  // LB_INIT_FIELDS: [4][ny][nx] rho, ux, uy, T on device
};
cudaError_t launch_init(Prec p, bool thermal, const InitArgs& a, cudaStream_t s);
// n doubles at p set to v; and the smallest index i with !(rho[i] > 0) into
// *first (all ones when there is none)
cudaError_t launch_fill(double* p, long long n, double v, cudaStream_t s);
cudaError_t launch_first_nonpositive(const double* rho, long long n, unsigned long long* first, cudaStream_t s);

void count_launch();

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device.  The attribute belongs to the function in each device's context, so
// it is set once per (device, function) under a lock; safe from any thread.
cudaError_t set_max_smem(const void* fn, int bytes);
}  // namespace lbgb
