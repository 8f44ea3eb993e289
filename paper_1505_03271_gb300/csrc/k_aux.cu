// k_aux.cu -- initialisation, population copy-in/out, moments and the FP64
// reductions (conservation sums, Nusselt numbers, divergence check).
#include "lb_internal.cuh"

namespace lbgb {

// ------------------------------------------------------------------ init --

// SplitMix64 (Steele, Lea & Flood 2014), one step from state seed ^ counter,
// top 53 bits mapped to [0, 1): the seeded perturbation of the RB preset.
__device__ __forceinline__ double splitmix_u01(unsigned long long seed, unsigned long long ctr) {
    unsigned long long z = (seed ^ ctr) + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
}

// Initial state at equilibrium in tilded variables (Appendix A):
// f~ = f_eq(rho, u) - dt/2 F(rho, u, a), g~ = (T / rho) f_eq; stored as
// deviations f~ - w and g~ - w T0.
template <typename S, bool TH>
__global__ void k_init(const InitArgs A) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= A.nx) return;
    const double X = A.xc[x], Y = A.yc[y];
    const size_t cell = (size_t)y * A.nx + x;
    double rho = 1.0, ux = 0.0, uy = 0.0, T = A.T0;
    const double twopi = 6.283185307179586476925286766559;
    const double dT = A.Tb - A.Tt;
    switch (A.kind) {
        case LB_INIT_TGV: {
            const double kx = twopi / A.lx, ky = twopi / A.ly, r = kx / ky;
            ux = -A.u0 * cos(kx * X) * sin(ky * Y);
            uy = A.u0 * r * sin(kx * X) * cos(ky * Y);
            rho = 1.0 - 0.75 * A.u0 * A.u0 * (cos(2.0 * kx * X) + r * r * cos(2.0 * ky * Y));
            if (A.amp != 0.0) ux += A.amp * sin(twopi * A.mode * Y / A.ly);
            break;
        }
        case LB_INIT_SHEAR: ux = A.amp * sin(twopi * A.mode * Y / A.ly); break;
        case LB_INIT_POISEUILLE: ux = 4.0 * A.u0 * Y * (A.ly - Y) / (A.ly * A.ly); break;
        case LB_INIT_RB: {
            const double U = splitmix_u01(A.seed, (unsigned long long)cell);
            T = A.T0 + dT * (0.5 - Y / A.ly) + A.amp * dT * (2.0 * U - 1.0);
            rho = A.rho_norm * exp(3.0 * A.bg * dT * (0.5 * Y - 0.5 * Y * Y / A.ly));
            break;
        }
        default: {  // LB_INIT_FIELDS
            const size_t n = (size_t)A.nx * A.ny;
            rho = A.fields[cell];
            ux = A.fields[n + cell];
            uy = A.fields[2 * n + cell];
            T = A.fields[3 * n + cell];
        }
    }
    const double ax = A.ax, ay = A.ay + (TH ? A.bg * (T - A.T0) : 0.0);
    S* f = static_cast<S*>(A.f);
    S* g = static_cast<S*>(A.g);
    const long long c = (long long)y * A.pitch + x;
    const double uu = ux * ux + uy * uy;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const double w = wgt<double>(a);
        const double cu = cx(a) * ux + cy(a) * uy;
        const double feq = w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        const double ca = cx(a) * ax + cy(a) * ay;
        const double F = w * rho * (3.0 * (ca - (ux * ax + uy * ay)) + 9.0 * cu * ca);
        Store<S>::st(f + a * A.plane + c, (feq - w * (1.0 + A.roff[y])) - 0.5 * A.dt * F);
        if (TH) Store<S>::st(g + a * A.plane + c, (T / rho) * feq - w * (A.T0 + A.toff[y]));
    }
}

template <typename S>
static cudaError_t run_init(bool th, const InitArgs& a, cudaStream_t s) {
    int bx = a.nx >= 256 ? 256 : ((a.nx + 31) / 32) * 32;
    dim3 grid((a.nx + bx - 1) / bx, a.ny);
    if (th) k_init<S, true><<<grid, bx, 0, s>>>(a);
    else k_init<S, false><<<grid, bx, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_init(Prec p, bool th, const InitArgs& a, cudaStream_t s) {
    switch (p) {
        case Prec::F64: return run_init<double>(th, a, s);
        case Prec::F32: return run_init<float>(th, a, s);
        case Prec::F16: return run_init<__half>(th, a, s);
        case Prec::BF16: return run_init<__nv_bfloat16>(th, a, s);
    }
    return cudaErrorInvalidValue;
}

// Host fields of LB_INIT_FIELDS go to the device as they are; an absent
// field is filled here, and the density is checked here rather than on the
// host, so lb_init reads each host array once, by DMA.
__global__ void k_fill(double* p, long long n, double v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// Smallest index whose density is not > 0 (NaN included) into *first,
// which the caller sets to all ones beforehand.
__global__ void k_first_nonpositive(const double* rho, long long n, unsigned long long* first) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(rho[i] > 0.0)) atomicMin(first, (unsigned long long)i);
}

static int aux_blocks(long long n) {
    const long long b = (n + 255) / 256;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

cudaError_t launch_fill(double* p, long long n, double v, cudaStream_t s) {
    k_fill<<<aux_blocks(n), 256, 0, s>>>(p, n, v);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_first_nonpositive(const double* rho, long long n, unsigned long long* first, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(first, 0xff, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_first_nonpositive<<<aux_blocks(n), 256, 0, s>>>(rho, n, first);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------ pack / unpack --

template <typename S>
__global__ void k_pack(const double* src, S* dst, int nx, int ny, int pitch, long long plane,
                       double off, const double* rowoff) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const double o = off + (rowoff ? rowoff[y] : 0.0);
#pragma unroll
    for (int a = 0; a < Q; ++a)
        Store<S>::st(dst + a * plane + (long long)y * pitch + x,
                     src[((size_t)a * ny + y) * nx + x] - wgt<double>(a) * o);
}

template <typename S>
__global__ void k_unpack(const S* src, double* dst, int nx, int ny, int pitch, long long plane,
                         double off, const double* rowoff, int x0, int y0, int w, int h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= w) return;
    const int x = (x0 + i) % nx, y = (y0 + j) % ny;
    const double o = off + (rowoff ? rowoff[y] : 0.0);
#pragma unroll
    for (int a = 0; a < Q; ++a)
        dst[((size_t)a * h + j) * w + i] =
            (double)Store<S>::ld(src + a * plane + (long long)y * pitch + x) + wgt<double>(a) * o;
}

template <typename S>
static cudaError_t run_pack(const double* src, void* dst, int nx, int ny, int pitch, long long plane,
                            double off, const double* ro, cudaStream_t s) {
    int bx = nx >= 256 ? 256 : ((nx + 31) / 32) * 32;
    dim3 grid((nx + bx - 1) / bx, ny);
    k_pack<S><<<grid, bx, 0, s>>>(src, static_cast<S*>(dst), nx, ny, pitch, plane, off, ro);
    count_launch();
    return cudaGetLastError();
}

template <typename S>
static cudaError_t run_unpack(const void* src, double* dst, int nx, int ny, int pitch, long long plane,
                              double off, const double* ro, int x0, int y0, int w, int h, cudaStream_t s) {
    int bx = w >= 256 ? 256 : ((w + 31) / 32) * 32;
    dim3 grid((w + bx - 1) / bx, h);
    k_unpack<S><<<grid, bx, 0, s>>>(static_cast<const S*>(src), dst, nx, ny, pitch, plane, off, ro, x0,
                                   y0, w, h);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pack(Prec p, const double* src, void* dst, int nx, int ny, int pitch, long long plane,
                        double off, const double* ro, cudaStream_t s) {
    switch (p) {
        case Prec::F64: return run_pack<double>(src, dst, nx, ny, pitch, plane, off, ro, s);
        case Prec::F32: return run_pack<float>(src, dst, nx, ny, pitch, plane, off, ro, s);
        case Prec::F16: return run_pack<__half>(src, dst, nx, ny, pitch, plane, off, ro, s);
        case Prec::BF16: return run_pack<__nv_bfloat16>(src, dst, nx, ny, pitch, plane, off, ro, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_unpack(Prec p, const void* src, double* dst, int nx, int ny, int pitch,
                          long long plane, double off, const double* ro, int x0, int y0, int w, int h,
                          cudaStream_t s) {
    switch (p) {
        case Prec::F64: return run_unpack<double>(src, dst, nx, ny, pitch, plane, off, ro, x0, y0, w, h, s);
        case Prec::F32: return run_unpack<float>(src, dst, nx, ny, pitch, plane, off, ro, x0, y0, w, h, s);
        case Prec::F16: return run_unpack<__half>(src, dst, nx, ny, pitch, plane, off, ro, x0, y0, w, h, s);
        case Prec::BF16:
            return run_unpack<__nv_bfloat16>(src, dst, nx, ny, pitch, plane, off, ro, x0, y0, w, h, s);
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------- moments, reductions --

// FP64 moments of one cell: rho = 1 + sum d, T = T0 + sum e,
// u = sum c d / rho + dt/2 a (Sec. II B 4).
template <typename S, bool TH>
__device__ __forceinline__ void cell_moments(const AuxArgs& A, int x, int y, double& rho, double& ux,
                                             double& uy, double& T) {
    const S* f = static_cast<const S*>(A.f);
    const S* g = static_cast<const S*>(A.g);
    const long long c = (long long)y * A.pitch + x;
    double r = 0, jx = 0, jy = 0, t = 0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const double d = (double)Store<S>::ld(f + a * A.plane + c) + wgt<double>(a) * A.roff[y];
        r += d;
        jx += cx(a) * d;
        jy += cy(a) * d;
    }
    if (TH) {
#pragma unroll
        for (int a = 0; a < Q; ++a) t += (double)Store<S>::ld(g + a * A.plane + c);
        t += A.toff[y];  // sum_a w_a toff = toff
    }
    rho = 1.0 + r;
    T = A.T0 + t;
    const double ay = A.ay + (TH ? A.bg * t : 0.0);
    ux = jx / rho + 0.5 * A.dt * A.ax;
    uy = jy / rho + 0.5 * A.dt * ay;
}

template <typename S, bool TH>
__global__ void k_moments(const AuxArgs A, double* out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= A.nx) return;
    double rho, ux, uy, T;
    cell_moments<S, TH>(A, x, y, rho, ux, uy, T);
    const size_t n = (size_t)A.nx * A.ny, c = (size_t)y * A.nx + x;
    out[c] = rho;
    out[n + c] = ux;
    out[2 * n + c] = uy;
    out[3 * n + c] = T;
}

constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum kRed values over the block in a fixed order; thread 0 gets the totals.
__device__ void block_sum(double (&v)[kRed], double (*sm)[kRedThreads / 32]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kRed; ++q) {
        const double s = warp_sum(v[q]);
        if (lane == 0) sm[q][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kRed; ++q) {
            double s = 0;
            for (int w = 0; w < kRedThreads / 32; ++w) s += sm[q][w];
            v[q] = s;
        }
    }
}

// Per cell: V rho, V rho ux, V rho uy, V T, V uy (T - T0), V, and dx T on the
// rows 0, 1, ny-2, ny-1 (for the plate gradients).  Grid-stride loop with a
// fixed cell-to-thread assignment, so the result is run-to-run identical.
template <typename S, bool TH>
__global__ void __launch_bounds__(kRedThreads) k_reduce(const AuxArgs A, double* partial) {
    __shared__ double sm[kRed][kRedThreads / 32];
    double v[kRed];
#pragma unroll
    for (int q = 0; q < kRed; ++q) v[q] = 0.0;
    const long long n = (long long)A.nx * A.ny;
    for (long long c = (long long)blockIdx.x * kRedThreads + threadIdx.x; c < n;
         c += (long long)gridDim.x * kRedThreads) {
        const int x = (int)(c % A.nx), y = (int)(c / A.nx);
        double rho, ux, uy, T;
        cell_moments<S, TH>(A, x, y, rho, ux, uy, T);
        const double V = A.dxv[x] * A.dyv[y];
        v[0] += V * rho;
        v[1] += V * rho * ux;
        v[2] += V * rho * uy;
        v[3] += V * T;
        v[4] += V * uy * (T - A.T0);
        v[5] += V;
        const double dxT = A.dxv[x] * T;
        if (y == 0) v[6] += dxT;
        if (y == 1) v[7] += dxT;
        if (y == A.ny - 2) v[8] += dxT;
        if (y == A.ny - 1) v[9] += dxT;
    }
    block_sum(v, sm);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kRed; ++q) partial[q * gridDim.x + blockIdx.x] = v[q];
    }
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_final(const double* partial, int nb, double* out) {
    __shared__ double sm[kRed][kRedThreads / 32];
    double v[kRed];
#pragma unroll
    for (int q = 0; q < kRed; ++q) {
        double s = 0;
        for (int b = threadIdx.x; b < nb; b += kRedThreads) s += partial[q * nb + b];
        v[q] = s;
    }
    block_sum(v, sm);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kRed; ++q) out[q] = v[q];
    }
}

int reduce_blocks(int nx, int ny) {
    long long n = (long long)nx * ny;
    long long b = (n + kRedThreads - 1) / kRedThreads;
    return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

template <typename S>
static cudaError_t run_moments(bool th, const AuxArgs& a, double* out, cudaStream_t s) {
    int bx = a.nx >= 256 ? 256 : ((a.nx + 31) / 32) * 32;
    dim3 grid((a.nx + bx - 1) / bx, a.ny);
    if (th) k_moments<S, true><<<grid, bx, 0, s>>>(a, out);
    else k_moments<S, false><<<grid, bx, 0, s>>>(a, out);
    count_launch();
    return cudaGetLastError();
}

template <typename S>
static cudaError_t run_reduce(bool th, const AuxArgs& a, double* partial, int nb, double* out,
                              cudaStream_t s) {
    if (th) k_reduce<S, true><<<nb, kRedThreads, 0, s>>>(a, partial);
    else k_reduce<S, false><<<nb, kRedThreads, 0, s>>>(a, partial);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, kRedThreads, 0, s>>>(partial, nb, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_moments(Prec p, bool th, const AuxArgs& a, double* out, cudaStream_t s) {
    switch (p) {
        case Prec::F64: return run_moments<double>(th, a, out, s);
        case Prec::F32: return run_moments<float>(th, a, out, s);
        case Prec::F16: return run_moments<__half>(th, a, out, s);
        case Prec::BF16: return run_moments<__nv_bfloat16>(th, a, out, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_reduce(Prec p, bool th, const AuxArgs& a, double* partial, int nb, double* out,
                          cudaStream_t s) {
    switch (p) {
        case Prec::F64: return run_reduce<double>(th, a, partial, nb, out, s);
        case Prec::F32: return run_reduce<float>(th, a, partial, nb, out, s);
        case Prec::F16: return run_reduce<__half>(th, a, partial, nb, out, s);
        case Prec::BF16: return run_reduce<__nv_bfloat16>(th, a, partial, nb, out, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbgb
