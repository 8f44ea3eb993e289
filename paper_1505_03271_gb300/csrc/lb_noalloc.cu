// lb_noalloc.cu -- lb_conservation_noalloc: the volume sums of
// lb_conservation computed on population buffers that the caller owns,
// without allocating anything.
//
// Who needs it: a host program that hands all device memory to its own pool
// or arena (a serving process that reserves HBM up front, a framework with a
// caching allocator) and forbids side allocations, or code on a latency path
// where cudaMalloc/cudaFree would synchronise the device.  Such a caller
// cannot create an lb_grid (that allocates) but can still ask for mass,
// momentum and heat of a state it keeps in its own buffers.
//
// The reduction needs scratch for one partial sum per block and a counter
// that lets the last block finish the sum.  That scratch is the file-scope
// array below, so it exists once per GPU that loads the library and stays
// allocated until the process exits.  Consequences for callers:
//   - Sizes are capped: one partial per block of kCellsPerBlock cells and at
//     most kMaxBlocks blocks, i.e. kMaxCells = 8,388,608 cells per call.
//     Larger grids are rejected with LB_ERR_ARG.
//   - Every call uses the same array.  Calls whose work overlaps on the GPU
//     (different streams, or different host threads on the same device)
//     race on it and give wrong sums; serialise them.
//   - Every call looks up the array's device address (cudaGetSymbolAddress)
//     in the context current on the calling thread, so a device that was
//     reset, or a non-primary context, gets the address of its own copy.
//     The first call in a context loads the library's module there; make
//     that first call before any stream capture begins.

#include "lb_internal.cuh"

namespace lbgb {
lb_status set_last_error(lb_status s, const char* msg);
}

namespace {

using lbgb::Q;

constexpr int kThreads = 256;
constexpr int kCellsPerBlock = 2048;  // 8 cells per thread
constexpr int kMaxBlocks = 4096;
constexpr long long kMaxCells = (long long)kMaxBlocks * kCellsPerBlock;
constexpr int kSums = 4;  // mass, momentum x, momentum y, heat
constexpr int kCounter = kSums * kMaxBlocks;  // slot of the completion counter

// Partial sums [kSums][kMaxBlocks] followed by the completion counter
// (4 * 4096 * 8 B + 256 B = 128.25 KiB per device).
static __device__ __align__(256) double g_scratch[kSums * kMaxBlocks + 32];

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum kSums values over the block in a fixed order; thread 0 gets the totals.
__device__ void block_sum(double (&v)[kSums], double (*sm)[kThreads / 32]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kSums; ++q) {
        const double s = warp_sum(v[q]);
        if (lane == 0) sm[q][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kSums; ++q) {
            double s = 0;
            for (int w = 0; w < kThreads / 32; ++w) s += sm[q][w];
            v[q] = s;
        }
    }
    __syncthreads();
}

// Block b sums cells [b * kCellsPerBlock, (b + 1) * kCellsPerBlock) into its
// scratch slot; the last block to finish adds the slots in block order and
// writes the totals to out, then resets the counter.
__global__ void __launch_bounds__(kThreads)
k_conservation_noalloc(const float* f, const float* g, int nx, int ny, int pitch, const double* dxv,
                       const double* dyv, double dt, double ax, double ay, double bg, double T0,
                       double* scratch, double* out) {
    __shared__ double sm[kSums][kThreads / 32];
    __shared__ bool last;
    const long long n = (long long)nx * ny;
    const long long c0 = (long long)blockIdx.x * kCellsPerBlock;
    const long long c1 = c0 + kCellsPerBlock < n ? c0 + kCellsPerBlock : n;
    const long long plane = (long long)pitch * ny;
    double v[kSums] = {0.0, 0.0, 0.0, 0.0};
    for (long long c = c0 + threadIdx.x; c < c1; c += kThreads) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        const long long o = (long long)y * pitch + x;
        double r = 0, jx = 0, jy = 0, t = 0;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const double d = (double)f[a * plane + o];
            r += d;
            jx += lbgb::cx(a) * d;
            jy += lbgb::cy(a) * d;
        }
        if (g) {
#pragma unroll
            for (int a = 0; a < Q; ++a) t += (double)g[a * plane + o];
        }
        const double rho = 1.0 + r, T = T0 + t;
        const double ux = jx / rho + 0.5 * dt * ax;
        const double uy = jy / rho + 0.5 * dt * (ay + (g ? bg * t : 0.0));
        const double V = dxv[x] * dyv[y];
        v[0] += V * rho;
        v[1] += V * rho * ux;
        v[2] += V * rho * uy;
        v[3] += V * T;
    }
    block_sum(v, sm);
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kCounter);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kSums; ++q) scratch[q * kMaxBlocks + blockIdx.x] = v[q];
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s[kSums];
#pragma unroll
    for (int q = 0; q < kSums; ++q) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads)
            acc += *((volatile double*)&scratch[q * kMaxBlocks + b]);
        s[q] = acc;
    }
    block_sum(s, sm);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kSums; ++q) out[q] = s[q];
        *counter = 0u;
    }
}

// Device address of g_scratch in the current context.  The lookup is a
// symbol-table query once the module is loaded, so it is repeated on every
// call rather than cached: a cached address would be stale after
// cudaDeviceReset or under another context of the same device.
lb_status scratch_address(double** ptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
        return lbgb::set_last_error(LB_ERR_CUDA, "cudaGetSymbolAddress of the no-alloc scratch failed");
    *ptr = static_cast<double*>(p);
    return LB_OK;
}

}  // namespace

extern "C" lb_status lb_conservation_noalloc(const float* f, const float* g, int nx, int ny, int pitch,
                                             const double* dx, const double* dy, double dt, double ax,
                                             double ay, double beta_grav, double T0, double* out,
                                             void* cuda_stream) {
    if (!f || !dx || !dy || !out) return lbgb::set_last_error(LB_ERR_ARG, "NULL pointer argument");
    if (nx < 1 || ny < 1 || pitch < nx)
        return lbgb::set_last_error(LB_ERR_ARG, "need nx, ny >= 1 and pitch >= nx");
    if ((long long)nx * ny > kMaxCells)
        return lbgb::set_last_error(
            LB_ERR_ARG, "lb_conservation_noalloc: grid larger than its fixed scratch allows "
                        "(at most 8388608 cells per call); use lb_conservation on an lb_grid");
    double* scratch = nullptr;
    lb_status st = scratch_address(&scratch);
    if (st != LB_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the completion counter must start at zero
    cudaError_t e = cudaMemsetAsync(scratch + kCounter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return lbgb::set_last_error(LB_ERR_CUDA, cudaGetErrorString(e));
    const long long n = (long long)nx * ny;
    const int blocks = (int)((n + kCellsPerBlock - 1) / kCellsPerBlock);
    k_conservation_noalloc<<<blocks, kThreads, 0, s>>>(f, g, nx, ny, pitch, dx, dy, dt, ax, ay, beta_grav,
                                                       T0, scratch, out);
    lbgb::count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return lbgb::set_last_error(LB_ERR_CUDA, cudaGetErrorString(e));
    return LB_OK;
}
