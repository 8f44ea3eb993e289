// lb_abi.cu -- host side of the C ABI declared in include/lb.h: grid and
// metric construction, parameter checks, kernel dispatch and observables.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "lb_grid.cuh"

using namespace lbgb;

namespace {

thread_local std::string g_err;
std::atomic<unsigned long long> g_launches{0};
// While this thread captures a step graph, launches are tallied here: they
// run (and count) only when the graph is replayed.
thread_local unsigned long long* t_captured = nullptr;

lb_status fail(lb_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CK(call)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                      \
    } while (0)

}  // namespace

namespace lbgb {
void count_launch() {
    if (t_captured) ++*t_captured;
    else g_launches.fetch_add(1, std::memory_order_relaxed);
}
cudaError_t set_max_smem(const void* fn, int bytes) {
    static std::mutex mu;
    static std::set<std::tuple<int, const void*, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({dev, fn, bytes})) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.insert({dev, fn, bytes});
    return e;
}
// 16-bit ST on flow grids periodic in x with nx % 4 == 0 (k_st16.cu).
bool st16_applies(Prec p, bool thermal, int nx, int bcx);
cudaError_t launch_st16(Prec p, const void* args, cudaStream_t s);
// FP32 ST on flow grids periodic in x with nx % 4 == 0 (k_st_quad.cu).
bool st_quad_applies(Prec p, bool thermal, int nx, int bcx);
cudaError_t launch_st_quad(const void* args, cudaStream_t s);
// Record a failure message for lb_last_error() from another translation unit.
lb_status set_last_error(lb_status s, const char* msg) { return fail(s, "%s", msg); }
}  // namespace lbgb

namespace {

void release(lb_grid* G) {
    void* ptrs[] = {G->f[0], G->f[1], G->g[0], G->g[1], G->mx, G->my, G->dxv, G->dyv, G->xc,
                    G->yc, G->toff, G->toff_r, G->roff, G->roff_r, G->dref_r, G->rowtab, G->coltab, G->fields,
                    G->partial, G->red, G->xh, G->xfc};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (G->cap) cudaStreamDestroy(G->cap);
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

AuxArgs aux_args(const lb_grid* G) {
    AuxArgs a{};
    a.f = G->f[G->cur];
    a.g = G->g[G->cur];
    a.nx = G->nx;
    a.ny = G->ny;
    a.pitch = G->pitch;
    a.plane = G->plane;
    a.dt = G->fv_scheme == LB_FV_EULER ? 0.0 : G->p.dt;  // dt/2 a shift of the tilded moments
    a.ax = G->p.ax;
    a.ay = G->p.ay;
    a.bg = G->p.beta * G->p.grav;
    a.T0 = G->p.T0;
    a.toff = G->toff;
    a.roff = G->roff;
    a.dxv = G->dxv;
    a.dyv = G->dyv;
    a.xc = G->xc;
    a.yc = G->yc;
    return a;
}

lb_status check_ready(lb_grid* G) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    if (!G->has_params) return fail(LB_ERR_STATE, "grid has no parameters: call lb_init first");
    if (G->poisoned) return fail(LB_ERR_STATE, "grid diverged (LB_ERR_UNSTABLE); call lb_init again");
    return LB_OK;
}

bool pair_ok(const lb_grid* G) {
    return G->prec != Prec::F64 && G->d.bcx == LB_BC_PERIODIC && G->d.bcy != LB_BC_DENSITY;
}

bool has_density_axis(const lb_grid* G) { return G->d.bcx == LB_BC_DENSITY || G->d.bcy == LB_BC_DENSITY; }

// Schedule actually used: AUTO takes a marching kernel (the paired one when
// it applies) once the grid is wide and tall enough to fill the GPU with
// strips, else the tile kernel.
int resolved_kernel(const lb_grid* G) {
    if (G->fv_kernel != LB_FV_AUTO) return G->fv_kernel;
    if (G->nx >= 480 && G->ny >= 256 && !G->d.thermal) return pair_ok(G) ? LB_FV_PAIR : LB_FV_MARCH;
    return pair_ok(G) ? LB_FV_PTILE : LB_FV_TILE;
}

// Rows per CTA of the marching kernels: one wave of resident CTAs.
int resolved_chunk(const lb_grid* G) {
    if (G->fv_chunk > 0) return G->fv_chunk;
    const bool th = G->d.thermal != 0;
    const bool pr = resolved_kernel(G) == LB_FV_PAIR;
    const int width = pr ? pair_width() : march_width(G->prec, th);
    const int strips = (G->nx + width - 1) / width;
    const size_t smem = pr ? pair_smem(th) : march_smem(G->prec, th);
    int per_sm = (int)(227 * 1024 / smem);
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 4) per_sm = 4;
    // about four waves of resident CTAs: short marches balance better than
    // one wave with a ragged tail, at 12 halo rows per chunk
    const long long slots = (long long)G->sms * per_sm;
    long long chunks = (4 * slots + strips - 1) / strips;
    if (chunks < 1) chunks = 1;
    int ch = (int)((G->ny + chunks - 1) / chunks);
    return ch < 32 ? 32 : ch;
}

// The split schedule's two FP32 buffers (NQ planes each), allocated on
// first use.
cudaError_t ensure_split_buffers(lb_grid* G) {
    if (G->xh) return cudaSuccess;
    const size_t bytes = sizeof(float) * (G->d.thermal ? 18 : 9) * (size_t)G->plane;
    cudaError_t e = cudaMalloc(&G->xh, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&G->xfc, bytes);
    if (e != cudaSuccess) {
        if (G->xh) cudaFree(G->xh);
        G->xh = G->xfc = nullptr;
    }
    return e;
}

template <typename R>
cudaError_t launch_fv_step(lb_grid* G) {
    StepArgs<R> A = step_args<R>(G, G->p.dt);
    const bool th = G->d.thermal != 0;
    if (A.stages == 1 || has_density_axis(G))  // single-stage schemes, density boundaries: scalar tile kernel
        return launch_fv(G->prec, th, &A, G->fv_kernel == LB_FV_TILE ? G->fv_chunk : 0, G->stream);
    const int k = resolved_kernel(G);
    if (k == LB_FV_SPLIT) {
        cudaError_t e = ensure_split_buffers(G);
        if (e != cudaSuccess) return e;
        A.xh = G->xh;
        A.xfc = G->xfc;
        return launch_fv_split(G->prec, th, &A, G->fv_chunk, G->stream);
    }
    if (k == LB_FV_PAIR) return launch_fv_pair(G->prec, th, &A, resolved_chunk(G), G->stream);
    if (k == LB_FV_PTILE) return launch_fv_ptile(G->prec, th, &A, G->fv_kernel == LB_FV_PTILE ? G->fv_chunk : 0,
                                                 G->stream);
    if (k == LB_FV_MARCH) return launch_fv_march(G->prec, th, &A, resolved_chunk(G), G->stream);
    return launch_fv(G->prec, th, &A, G->fv_kernel == LB_FV_TILE ? G->fv_chunk : 0, G->stream);
}

lb_status upload(void** dst, const std::vector<double>& v, bool as_float) {
    size_t bytes = v.size() * (as_float ? sizeof(float) : sizeof(double));
    CK(cudaMalloc(dst, bytes ? bytes : 8));
    if (as_float) {
        std::vector<float> t(v.begin(), v.end());
        CK(cudaMemcpy(*dst, t.data(), bytes, cudaMemcpyHostToDevice));
    } else {
        CK(cudaMemcpy(*dst, v.data(), bytes, cudaMemcpyHostToDevice));
    }
    return LB_OK;
}

lb_status reduce(lb_grid* G, double out[kRed]) {
    CK(launch_reduce(G->prec, G->d.thermal != 0, aux_args(G), G->partial, G->nred, G->red, G->stream));
    CK(cudaMemcpyAsync(out, G->red, sizeof(double) * kRed, cudaMemcpyDeviceToHost, G->stream));
    CK(cudaStreamSynchronize(G->stream));
    return LB_OK;
}

// Capture n steps of `one` on the grid's private stream into an executable
// graph.  The state flips buffers n times (n even), so it is back where it
// started and the captured buffer pointers hold for every replay.  False,
// with nothing launched, where capture is unavailable: the grid's stream is
// itself being captured, or a call inside the capture is refused.
template <typename F>
bool capture_steps(lb_grid* G, int n, F& one, cudaGraphExec_t* exec, unsigned long long* per) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(G->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return false;
    }
    if (!G->cap && cudaStreamCreateWithFlags(&G->cap, cudaStreamNonBlocking) != cudaSuccess) {
        G->cap = nullptr;
        cudaGetLastError();
        return false;
    }
    const cudaStream_t user = G->stream;
    const int cur0 = G->cur;
    unsigned long long count = 0;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(G->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        G->stream = G->cap;
        t_captured = &count;
        for (int j = 0; j < n && e == cudaSuccess; ++j) {
            e = one();
            G->cur ^= 1;
        }
        t_captured = nullptr;
        G->stream = user;
        const cudaError_t e2 = cudaStreamEndCapture(G->cap, &graph);
        if (e == cudaSuccess) e = e2;
    }
    G->cur = cur0;
    *exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *exec = nullptr;
        return false;
    }
    *per = count;
    return true;
}

// nsteps steps, each one call of `one` on G->stream followed by a buffer
// flip.  A run of more than 2 graph_steps steps takes its first step
// directly (first-use function attributes and buffers are set outside any
// capture), then replays a graph of graph_steps captured steps on the
// grid's stream and launches the remainder one by one.  The replays run the
// same kernels with the same arguments as the direct launches; the graph
// only takes the per-launch host and front-end cost off each step.
template <typename F>
lb_status run_steps(lb_grid* G, int nsteps, F one) {
    int k = 0;
    const int n = G->graph_steps;
    if (n > 0 && nsteps > 2 * n) {
        CK(one());
        G->cur ^= 1;
        ++k;
        cudaGraphExec_t exec = nullptr;
        unsigned long long per = 0;
        if (capture_steps(G, n, one, &exec, &per)) {
            cudaError_t e = cudaSuccess;
            for (; k + n <= nsteps; k += n) {
                e = cudaGraphLaunch(exec, G->stream);
                if (e != cudaSuccess) break;
                g_launches.fetch_add(per, std::memory_order_relaxed);
                ++G->graph_replays;
            }
            cudaGraphExecDestroy(exec);  // released once its queued replays have run
            CK(e);
        }
    }
    for (; k < nsteps; ++k) {
        CK(one());
        G->cur ^= 1;
    }
    return LB_OK;
}

}  // namespace

extern "C" {

const char* lb_last_error(void) { return g_err.c_str(); }

unsigned long long lb_kernel_launches(void) { return g_launches.load(); }

lb_status lb_create_grid(const lb_grid_desc* d, lb_grid** out) {
    if (!d || !out) return fail(LB_ERR_ARG, "NULL description or output");
    if (d->nx < 1 || d->ny < 1) return fail(LB_ERR_ARG, "nx, ny must be >= 1 (got %d, %d)", d->nx, d->ny);
    if ((long long)d->nx * d->ny > (1LL << 31))
        return fail(LB_ERR_ARG, "grid of %d x %d cells is larger than supported", d->nx, d->ny);
    if (d->bcx < LB_BC_PERIODIC || d->bcx > LB_BC_DENSITY) return fail(LB_ERR_ARG, "bad bcx");
    if (d->bcy < LB_BC_PERIODIC || d->bcy > LB_BC_DENSITY) return fail(LB_ERR_ARG, "bad bcy");
    if ((d->bcx != LB_BC_PERIODIC && d->nx < 2) || (d->bcy != LB_BC_PERIODIC && d->ny < 2))
        return fail(LB_ERR_ARG, "a wall or density axis needs at least 2 cells (two ghost layers)");
    if (d->thermal && d->bcx != LB_BC_PERIODIC)
        return fail(LB_ERR_ARG, "thermal grids have their isothermal plates on y; x must be periodic");
    if (d->thermal && d->bcy == LB_BC_DENSITY)
        return fail(LB_ERR_ARG, "thermal grids have isothermal plates on y, not a density boundary");
    if (d->store < LB_STORE_F64 || d->store > LB_STORE_BF16DEV) return fail(LB_ERR_ARG, "bad store");
    for (int k = 0; k < 2; ++k) {
        const int sp = k ? d->sy : d->sx, n = k ? d->ny : d->nx;
        const double L = k ? d->ly : d->lx, st = k ? d->stretch_y : d->stretch_x;
        if (sp < LB_AXIS_UNIFORM || sp > LB_AXIS_CHEB) return fail(LB_ERR_ARG, "bad spacing");
        if (!(L > 0)) return fail(LB_ERR_ARG, "domain length must be > 0");
        if ((sp == LB_AXIS_TANH || sp == LB_AXIS_SINH) && !(st > 0)) return fail(LB_ERR_ARG, "stretch must be > 0");
        if (sp == LB_AXIS_SINH && (n % 2)) return fail(LB_ERR_ARG, "sinh spacing needs an even cell count");
    }
    lb_grid* G = new lb_grid();
    G->d = *d;
    G->nx = d->nx;
    G->ny = d->ny;
    G->pitch = ((d->nx + 31) / 32) * 32;
    G->plane = (long long)G->pitch * d->ny;
    G->prec = prec_of(d->store);
    G->stream = static_cast<cudaStream_t>(d->cuda_stream);
    G->ax = make_axis(d->nx, d->lx, d->sx, d->stretch_x, d->bcx);
    G->ay = make_axis(d->ny, d->ly, d->sy, d->stretch_y, d->bcy);
    G->dmin = 1e300;
    for (double v : G->ax.d) G->dmin = std::fmin(G->dmin, v);
    for (double v : G->ay.d) G->dmin = std::fmin(G->dmin, v);
    for (int k = 0; k < 2; ++k) {
        const Axis& a = k ? G->ay : G->ax;
        for (double v : a.d)
            if (!(v > 0)) {
                delete G;
                return fail(LB_ERR_ARG, "degenerate cell width on axis %c", k ? 'y' : 'x');
            }
    }
    cudaGetDevice(&G->device);
    cudaDeviceGetAttribute(&G->sms, cudaDevAttrMultiProcessorCount, G->device);
    if (G->sms <= 0) G->sms = 152;
    const size_t pop_bytes = (size_t)Q * G->plane * elem_size(d->store);
    const bool as_float = G->prec != Prec::F64;
    G->nred = reduce_blocks(G->nx, G->ny);
    lb_status st = LB_OK;
    auto alloc = [&](void** p, size_t bytes) {
        if (st != LB_OK) return;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            *p = nullptr;
            cudaGetLastError();
            st = fail(e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,
                      "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
        }
    };
    for (int b = 0; b < 2; ++b) {
        alloc(&G->f[b], pop_bytes);
        if (d->thermal) alloc(&G->g[b], pop_bytes);
    }
    alloc((void**)&G->fields, sizeof(double) * 4 * (size_t)G->nx * G->ny);
    alloc((void**)&G->toff, sizeof(double) * G->ny);
    alloc(&G->toff_r, (as_float ? sizeof(float) : sizeof(double)) * G->ny);
    alloc((void**)&G->roff, sizeof(double) * G->ny);
    alloc(&G->roff_r, (as_float ? sizeof(float) : sizeof(double)) * G->ny);
    alloc(&G->dref_r, (as_float ? sizeof(float) : sizeof(double)) * 4 * G->ny);
    alloc((void**)&G->rowtab, sizeof(float) * 20 * G->ny);
    alloc((void**)&G->coltab, sizeof(float) * 20 * G->nx);
    if (st == LB_OK && as_float) {
        // x data of the column pair starting at each column (the right column wraps)
        const int nx = G->nx;
        const std::vector<double> mxv = G->ax.metric();
        auto wpv = [&](int r, int k) { return (float)mxv[r * (nx + 1) + k]; };
        auto wmv = [&](int r, int k) { return (float)mxv[(3 + r) * (nx + 1) + k]; };
        std::vector<float> tab(20 * (size_t)nx, 0.0f);
        for (int c = 0; c < nx; ++c) {
            const int cr = (c + 1) % nx;
            float* e = &tab[20 * (size_t)c];
            for (int r = 0; r < 3; ++r) {
                e[r] = wpv(r, c);
                e[3 + r] = wpv(r, c + 1);
                e[6 + r] = wpv(r, cr + 1);
                e[9 + r] = wmv(r, c);
                e[12 + r] = wmv(r, c + 1);
                e[15 + r] = wmv(r, cr + 1);
            }
            e[18] = (float)mxv[6 * (nx + 1) + c];
            e[19] = (float)mxv[6 * (nx + 1) + cr];
        }
        if (cudaMemcpy(G->coltab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            st = fail(LB_ERR_CUDA, "coltab upload failed");
    }
    alloc((void**)&G->partial, sizeof(double) * kRed * G->nred);
    alloc((void**)&G->red, sizeof(double) * kRed);
    if (st == LB_OK) st = upload(&G->mx, G->ax.metric(), as_float);
    if (st == LB_OK) st = upload(&G->my, G->ay.metric(), as_float);
    if (st == LB_OK) st = upload((void**)&G->dxv, G->ax.d, false);
    if (st == LB_OK) st = upload((void**)&G->dyv, G->ay.d, false);
    if (st == LB_OK) st = upload((void**)&G->xc, G->ax.c, false);
    if (st == LB_OK) st = upload((void**)&G->yc, G->ay.c, false);
    if (st != LB_OK) {
        release(G);
        delete G;
        return st;
    }
    *out = G;
    return LB_OK;
}

lb_status lb_destroy(lb_grid* G) {
    if (!G) return LB_OK;
    DeviceGuard dg(G->device);
    cudaStreamSynchronize(G->stream);
    release(G);
    delete G;
    return LB_OK;
}

lb_status lb_sync(lb_grid* G) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    DeviceGuard dg(G->device);
    CK(cudaStreamSynchronize(G->stream));
    return LB_OK;
}

lb_status lb_init(lb_grid* G, const lb_params* p, const lb_init_desc* in) {
    if (!G || !p || !in) return fail(LB_ERR_ARG, "NULL argument");
    if (!(p->tau > 0) || !(p->dt > 0)) return fail(LB_ERR_ARG, "tau and dt must be > 0");
    if (G->d.thermal && !(p->tau_g > 0)) return fail(LB_ERR_ARG, "tau_g must be > 0 on a thermal grid");
    if (in->kind < LB_INIT_TGV || in->kind > LB_INIT_FIELDS) return fail(LB_ERR_ARG, "bad init kind");
    if (in->kind == LB_INIT_RB && !G->d.thermal) return fail(LB_ERR_ARG, "RB preset needs a thermal grid");
    DeviceGuard dg(G->device);
    // Reference state of the storage: the barometric density and conductive
    // temperature of the RB base state on a grid with plates, else 1 and T0.
    double rho_norm = 1.0;
    const double dTp = p->T_bot - p->T_top, bgp = p->beta * p->grav, Hy = G->d.ly;
    auto baro = [&](double y) { return std::exp(3.0 * bgp * dTp * (0.5 * y - 0.5 * y * y / Hy)); };
    if (in->kind == LB_INIT_RB) {
        double s = 0.0;
        for (int j = 0; j < G->ny; ++j) s += G->ay.d[j] * baro(G->ay.c[j]);
        rho_norm = Hy / s;  // sum V rho = sum V
    }
    {
        std::vector<double> to(G->ny, 0.0), ro(G->ny, 0.0);
        const bool plates = G->d.thermal && G->d.bcy == LB_BC_WALLS;
        for (int j = 0; j < G->ny; ++j) {
            if (plates) to[j] = dTp * (0.5 - G->ay.c[j] / Hy) + 0.5 * (p->T_bot + p->T_top) - p->T0;
            if (in->kind == LB_INIT_RB) ro[j] = rho_norm * baro(G->ay.c[j]) - 1.0;
        }
        // y flux divergence of the base state per row and upwind sign, with
        // the same QUICK weights as the kernels; ghost rows extend rho_r
        // evenly and T_r oddly about the plate temperature.
        const int ny = G->ny;
        const bool wall = G->d.bcy == LB_BC_WALLS;
        auto ext = [&](const std::vector<double>& v, int i, double wall_lo, double wall_hi, bool odd) {
            if (i >= 0 && i < ny) return v[i];
            if (!wall) return v[((i % ny) + ny) % ny];
            if (i < 0) return odd ? 2.0 * wall_lo - v[-i - 1] : v[-i - 1];
            return odd ? 2.0 * wall_hi - v[2 * ny - 1 - i] : v[2 * ny - 1 - i];
        };
        std::vector<double> dref(4 * (size_t)ny, 0.0);
        for (int q = 0; q < 2; ++q) {
            const std::vector<double>& v = q ? to : ro;
            const double lo = q ? p->T_bot - p->T0 : 0.0, hi = q ? p->T_top - p->T0 : 0.0;
            bool any = false;
            for (double x : v) any = any || x != 0.0;
            if (!any) continue;
            for (int sgn = 0; sgn < 2; ++sgn) {
                auto face = [&](int kf) {
                    const int k0 = sgn == 0 ? kf - 2 : kf - 1;
                    double w[3];
                    G->ay.quick(k0, kf, w);
                    double phi = 0.0;
                    for (int m = 0; m < 3; ++m) phi += w[m] * ext(v, k0 + m, lo, hi, q == 1);
                    return phi;
                };
                for (int j = 0; j < ny; ++j) dref[(2 * q + sgn) * ny + j] = (face(j + 1) - face(j)) / G->ay.d[j];
            }
        }
        CK(cudaMemcpy(G->toff, to.data(), sizeof(double) * G->ny, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(G->roff, ro.data(), sizeof(double) * G->ny, cudaMemcpyHostToDevice));
        if (G->prec == Prec::F64) {
            CK(cudaMemcpy(G->toff_r, to.data(), sizeof(double) * G->ny, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(G->roff_r, ro.data(), sizeof(double) * G->ny, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(G->dref_r, dref.data(), sizeof(double) * dref.size(), cudaMemcpyHostToDevice));
        } else {
            std::vector<float> tf(to.begin(), to.end()), rf(ro.begin(), ro.end()), df(dref.begin(), dref.end());
            CK(cudaMemcpy(G->toff_r, tf.data(), sizeof(float) * G->ny, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(G->roff_r, rf.data(), sizeof(float) * G->ny, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(G->dref_r, df.data(), sizeof(float) * df.size(), cudaMemcpyHostToDevice));
            // per-row table of the paired kernel: one 80-byte entry per row
            const std::vector<double> my = G->ay.metric();
            std::vector<float> tab(20 * (size_t)ny, 0.0f);
            for (int j = 0; j < ny; ++j) {
                float* e = &tab[20 * (size_t)j];
                for (int q = 0; q < 3; ++q) {
                    e[q] = (float)my[q * (ny + 1) + j];            // c > 0, south face j
                    e[3 + q] = (float)my[q * (ny + 1) + j + 1];    // c > 0, north face j + 1
                    e[6 + q] = (float)my[(3 + q) * (ny + 1) + j];  // c < 0, south
                    e[9 + q] = (float)my[(3 + q) * (ny + 1) + j + 1];
                }
                e[12] = (float)my[6 * (ny + 1) + j];
                e[13] = (float)ro[j];
                e[14] = (float)to[j];
                for (int q = 0; q < 4; ++q) e[15 + q] = (float)dref[q * ny + j];
            }
            CK(cudaMemcpy(G->rowtab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice));
        }
    }
    InitArgs a{};
    a.f = G->f[0];
    a.g = G->g[0];
    a.nx = G->nx;
    a.ny = G->ny;
    a.pitch = G->pitch;
    a.plane = G->plane;
    a.kind = in->kind;
    a.mode = in->mode;
    a.u0 = in->u0;
    a.amp = in->amp;
    a.seed = in->seed;
    a.lx = G->d.lx;
    a.ly = G->d.ly;
    a.dt = G->fv_scheme == LB_FV_EULER ? 0.0 : p->dt;  // f~ = f_eq - dt/2 F; Euler starts at f_eq
    a.ax = p->ax;
    a.ay = p->ay;
    a.bg = p->beta * p->grav;
    a.T0 = p->T0;
    a.Tb = p->T_bot;
    a.Tt = p->T_top;
    a.xc = G->xc;
    a.yc = G->yc;
    a.toff = G->toff;
    a.roff = G->roff;
    a.fields = G->fields;
    a.rho_norm = rho_norm;
    if (in->kind == LB_INIT_FIELDS) {
        // each host field straight into the staging buffer (a DMA when the
        // caller's memory is pinned); absent fields filled on the device
        const long long n = (long long)G->nx * G->ny;
        const double* src[4] = {in->rho, in->ux, in->uy, in->T};
        const double fill[4] = {1.0, 0.0, 0.0, p->T0};
        for (int k = 0; k < 4; ++k) {
            if (src[k])
                CK(cudaMemcpyAsync(G->fields + k * n, src[k], sizeof(double) * n, cudaMemcpyHostToDevice, G->stream));
            else
                CK(launch_fill(G->fields + k * n, n, fill[k], G->stream));
        }
        // the density is checked before the populations are touched, so a
        // rejected call leaves the grid's state as it was
        unsigned long long* first = reinterpret_cast<unsigned long long*>(G->red);
        unsigned long long bad = ~0ULL;
        CK(launch_first_nonpositive(G->fields, n, first, G->stream));
        CK(cudaMemcpyAsync(&bad, first, sizeof(bad), cudaMemcpyDeviceToHost, G->stream));
        CK(cudaStreamSynchronize(G->stream));  // the host arrays are read before return
        if (bad != ~0ULL) return fail(LB_ERR_ARG, "density must be > 0 (cell %llu)", bad);
        CK(launch_init(G->prec, G->d.thermal != 0, a, G->stream));
    } else {
        CK(launch_init(G->prec, G->d.thermal != 0, a, G->stream));
    }
    G->p = *p;
    G->has_params = true;
    G->poisoned = false;
    G->cur = 0;
    return LB_OK;
}

lb_status lb_step_fv(lb_grid* G, int nsteps) {
    lb_status s = check_ready(G);
    if (s != LB_OK) return s;
    if (nsteps < 0) return fail(LB_ERR_ARG, "nsteps must be >= 0");
    DeviceGuard dg(G->device);
    return run_steps(G, nsteps,
                     [G] { return G->prec == Prec::F64 ? launch_fv_step<double>(G) : launch_fv_step<float>(G); });
}

lb_status lb_set_graph_steps(lb_grid* G, int n) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    if (n < 0 || n % 2 != 0 || n > 4096) return fail(LB_ERR_ARG, "graph length must be even, 0..4096 (got %d)", n);
    G->graph_steps = n;
    return LB_OK;
}

lb_status lb_get_graph_steps(lb_grid* G, int* n, unsigned long long* replays) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    if (n) *n = G->graph_steps;
    if (replays) *replays = G->graph_replays;
    return LB_OK;
}

lb_status lb_set_fv_schedule(lb_grid* G, int kernel, int chunk) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    if (kernel < LB_FV_AUTO || kernel > LB_FV_SPLIT) return fail(LB_ERR_ARG, "unknown FV kernel %d", kernel);
    if (chunk < 0) return fail(LB_ERR_ARG, "chunk must be >= 0");
    if (kernel == LB_FV_TILE && chunk != 0 && chunk != 8 && chunk != 16)
        return fail(LB_ERR_ARG, "tile shape must be 0 (32 x 16), 16 (16 x 16) or 8 (16 x 8)");
    if (kernel == LB_FV_PTILE && chunk != 0 && chunk != 14 && chunk != 16 && chunk != 512 && chunk != 526)
        return fail(LB_ERR_ARG, "paired tile shape must be 0 (32 x 16), 14 (32 x 14), 16 (16 x 16), 512 (32 x 16, "
                                "512 threads) or 526 (32 x 14, 512 threads)");
    if (kernel == LB_FV_SPLIT && chunk != 0 && chunk != 16)
        return fail(LB_ERR_ARG, "split tile shape must be 0 (32 x 16) or 16 (16 x 16)");
    if ((kernel == LB_FV_PAIR || kernel == LB_FV_PTILE || kernel == LB_FV_SPLIT) && !pair_ok(G))
        return fail(LB_ERR_ARG, "the paired FV kernel needs FP32/FP16/BF16 storage and a periodic x axis");
    G->fv_kernel = kernel;
    G->fv_chunk = chunk;
    return LB_OK;
}

lb_status lb_set_fv_scheme(lb_grid* G, int scheme) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    if (scheme < LB_FV_HEUN || scheme > LB_FV_EULER) return fail(LB_ERR_ARG, "unknown FV scheme %d", scheme);
    if (scheme != G->fv_scheme) {
        G->fv_scheme = scheme;
        G->has_params = false;  // the state's meaning changed: lb_init again
    }
    return LB_OK;
}

lb_status lb_set_boundary_density(lb_grid* G, double rho_x0, double rho_x1, double rho_y0, double rho_y1) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    if (!(rho_x0 > 0) || !(rho_x1 > 0) || !(rho_y0 > 0) || !(rho_y1 > 0))
        return fail(LB_ERR_ARG, "boundary densities must be > 0");
    G->rho_bc[0] = rho_x0;
    G->rho_bc[1] = rho_x1;
    G->rho_bc[2] = rho_y0;
    G->rho_bc[3] = rho_y1;
    return LB_OK;
}

lb_status lb_get_fv_scheme(lb_grid* G, int* scheme) {
    if (!G || !scheme) return fail(LB_ERR_ARG, "NULL argument");
    *scheme = G->fv_scheme;
    return LB_OK;
}

lb_status lb_get_fv_schedule(lb_grid* G, int* kernel, int* chunk) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    if (kernel) *kernel = resolved_kernel(G);
    if (chunk) {
        const int k = resolved_kernel(G);
        *chunk = (k == LB_FV_TILE || k == LB_FV_PTILE || k == LB_FV_SPLIT) ? (G->fv_kernel == k ? G->fv_chunk : 0)
                                                                            : resolved_chunk(G);
    }
    return LB_OK;
}

lb_status lb_autotune_fv(lb_grid* G, int steps) {
    lb_status s = check_ready(G);
    if (s != LB_OK) return s;
    if (steps < 1) return fail(LB_ERR_ARG, "steps must be >= 1");
    DeviceGuard dg(G->device);
    const size_t bytes = (size_t)Q * G->plane * elem_size(G->d.store);
    void *sf = nullptr, *sg = nullptr;
    CK(cudaMalloc(&sf, bytes));
    if (G->d.thermal && cudaMalloc(&sg, bytes) != cudaSuccess) {
        cudaFree(sf);
        return fail(LB_ERR_OOM, "autotune: no memory for the state copy");
    }
    const int cur0 = G->cur;
    cudaMemcpyAsync(sf, G->f[cur0], bytes, cudaMemcpyDeviceToDevice, G->stream);
    if (sg) cudaMemcpyAsync(sg, G->g[cur0], bytes, cudaMemcpyDeviceToDevice, G->stream);
    const int k0 = G->fv_kernel, c0 = G->fv_chunk;
    std::vector<std::pair<int, int>> cands = {{LB_FV_TILE, 0}, {LB_FV_TILE, 16}, {LB_FV_TILE, 8}};
    if (pair_ok(G)) {
        cands.push_back({LB_FV_PTILE, 0});
        cands.push_back({LB_FV_PTILE, 16});
        cands.push_back({LB_FV_PTILE, 512});
        cands.push_back({LB_FV_PTILE, 14});
        cands.push_back({LB_FV_PTILE, 526});
        if (ensure_split_buffers(G) == cudaSuccess) {
            cands.push_back({LB_FV_SPLIT, 0});
            cands.push_back({LB_FV_SPLIT, 16});
        }
    }
    for (int kern : {(int)LB_FV_MARCH, (int)LB_FV_PAIR}) {
        if (kern == LB_FV_PAIR && !pair_ok(G)) continue;
        G->fv_kernel = kern;
        G->fv_chunk = 0;
        const int base = resolved_chunk(G);
        for (int ch : {base / 2, base, base * 2, 32, 64, 128})
            if (ch >= 16 && ch <= 4 * G->ny) cands.push_back({kern, ch});
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    std::pair<int, int> pick = {LB_FV_TILE, 0};
    lb_status st = LB_OK;
    for (auto& c : cands) {
        G->fv_kernel = c.first;
        G->fv_chunk = c.second;
        G->cur = cur0;
        // warm-up step, then the timed ones
        cudaError_t e = G->prec == Prec::F64 ? launch_fv_step<double>(G) : launch_fv_step<float>(G);
        G->cur ^= 1;
        cudaEventRecord(e0, G->stream);
        for (int k = 0; k < steps && e == cudaSuccess; ++k) {
            e = G->prec == Prec::F64 ? launch_fv_step<double>(G) : launch_fv_step<float>(G);
            G->cur ^= 1;
        }
        cudaEventRecord(e1, G->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            st = fail(LB_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            pick = c;
        }
    }
    // restore the state into the buffer it started in
    G->cur = cur0;
    cudaMemcpyAsync(G->f[cur0], sf, bytes, cudaMemcpyDeviceToDevice, G->stream);
    if (sg) cudaMemcpyAsync(G->g[cur0], sg, bytes, cudaMemcpyDeviceToDevice, G->stream);
    cudaStreamSynchronize(G->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sf);
    if (sg) cudaFree(sg);
    if (st != LB_OK) {
        G->fv_kernel = k0;
        G->fv_chunk = c0;
        return st;
    }
    G->fv_kernel = pick.first;
    G->fv_chunk = pick.second;
    return LB_OK;
}

lb_status lb_step_st(lb_grid* G, int nsteps) {
    lb_status s = check_ready(G);
    if (s != LB_OK) return s;
    if (nsteps < 0) return fail(LB_ERR_ARG, "nsteps must be >= 0");
    if (G->fv_scheme == LB_FV_EULER) return fail(LB_ERR_STATE, "ST steps tilded populations, not an Euler grid");
    if (has_density_axis(G)) return fail(LB_ERR_ARG, "the fixed-density boundary is an FV boundary (no ST form)");
    for (int k = 0; k < 2; ++k) {
        const int sp = k ? G->d.sy : G->d.sx, n = k ? G->ny : G->nx;
        const double L = k ? G->d.ly : G->d.lx;
        if (sp != LB_AXIS_UNIFORM || std::fabs(L / n - 1.0) > 1e-12)
            return fail(LB_ERR_ARG, "ST needs uniform axes with unit spacing (axis %c: L/n = %g)",
                        k ? 'y' : 'x', L / n);
    }
    if (std::fabs(G->p.dt - 1.0) > 1e-12) return fail(LB_ERR_ARG, "ST needs dt = 1 (got %g)", G->p.dt);
    DeviceGuard dg(G->device);
    const bool th = G->d.thermal != 0;
    return run_steps(G, nsteps, [G, th] {
        if (G->prec == Prec::F64) {
            StepArgs<double> A = step_args<double>(G, 1.0);
            return launch_st(G->prec, th, &A, G->stream);
        }
        StepArgs<float> A = step_args<float>(G, 1.0);
        if (st16_applies(G->prec, th, G->nx, G->d.bcx)) return launch_st16(G->prec, &A, G->stream);
        if (st_quad_applies(G->prec, th, G->nx, G->d.bcx)) return launch_st_quad(&A, G->stream);
        return launch_st(G->prec, th, &A, G->stream);
    });
}

lb_status lb_moments(lb_grid* G, double* rho, double* ux, double* uy, double* T) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    if (!G->has_params) return fail(LB_ERR_STATE, "grid has no parameters: call lb_init first");
    DeviceGuard dg(G->device);
    CK(launch_moments(G->prec, G->d.thermal != 0, aux_args(G), G->fields, G->stream));
    const size_t n = (size_t)G->nx * G->ny;
    double* outs[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k)
        if (outs[k])
            CK(cudaMemcpyAsync(outs[k], G->fields + k * n, sizeof(double) * n, cudaMemcpyDeviceToHost,
                               G->stream));
    CK(cudaStreamSynchronize(G->stream));
    return LB_OK;
}

lb_status lb_conservation(lb_grid* G, double* mass, double* momx, double* momy, double* heat) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    if (!G->has_params) return fail(LB_ERR_STATE, "grid has no parameters: call lb_init first");
    DeviceGuard dg(G->device);
    double v[kRed];
    lb_status s = reduce(G, v);
    if (s != LB_OK) return s;
    if (mass) *mass = v[0];
    if (momx) *momx = v[1];
    if (momy) *momy = v[2];
    if (heat) *heat = v[3];
    for (int q = 0; q < 4; ++q)
        if (!std::isfinite(v[q])) {
            G->poisoned = true;
            return fail(LB_ERR_UNSTABLE, "non-finite conservation sum: the run diverged (dt too large "
                                         "for tau or the grid)");
        }
    return LB_OK;
}

lb_status lb_nusselt(lb_grid* G, double* nu_vol, double* nu_bot, double* nu_top) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    if (!G->d.thermal) return fail(LB_ERR_STATE, "Nusselt numbers need a thermal grid");
    if (!G->has_params) return fail(LB_ERR_STATE, "grid has no parameters: call lb_init first");
    DeviceGuard dg(G->device);
    double v[kRed];
    lb_status s = reduce(G, v);
    if (s != LB_OK) return s;
    const lb_params& p = G->p;
    const double H = G->d.ly, dT = p.T_bot - p.T_top, kappa = p.tau_g / 3.0, Lx = G->d.lx;
    if (nu_vol) *nu_vol = 1.0 + H * (v[4] / v[5]) / (kappa * dT);
    // plate gradients: quadratic through the wall value and the first two
    // x-averaged nodes, differentiated at the wall
    const double t0 = v[6] / Lx, t1 = v[7] / Lx, tn2 = v[8] / Lx, tn1 = v[9] / Lx;
    const double y0 = G->ay.c[0], y1 = G->ay.c[1];
    const double gb = -(y0 + y1) / (y0 * y1) * p.T_bot + y1 / (y0 * (y1 - y0)) * t0 - y0 / (y1 * (y1 - y0)) * t1;
    const double s0 = H - G->ay.c[G->ny - 1], s1 = H - G->ay.c[G->ny - 2];
    const double gt = -(s0 + s1) / (s0 * s1) * p.T_top + s1 / (s0 * (s1 - s0)) * tn1 - s0 / (s1 * (s1 - s0)) * tn2;
    if (nu_bot) *nu_bot = -H * gb / dT;
    if (nu_top) *nu_top = H * gt / dT;
    for (double x : v)
        if (!std::isfinite(x)) {
            G->poisoned = true;
            return fail(LB_ERR_UNSTABLE, "non-finite reduction: the run diverged");
        }
    return LB_OK;
}

lb_status lb_set_populations(lb_grid* G, const double* f, const double* g) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    if (!G->has_params) return fail(LB_ERR_STATE, "set parameters with lb_init before setting populations");
    if (g && !G->d.thermal) return fail(LB_ERR_STATE, "thermal populations on a flow-only grid");
    DeviceGuard dg(G->device);
    const size_t n = (size_t)Q * G->nx * G->ny;
    double* tmp = nullptr;
    CK(cudaMalloc(&tmp, sizeof(double) * n));
    lb_status st = LB_OK;
    const double* srcs[2] = {f, g};
    void* dsts[2] = {G->f[G->cur], G->g[G->cur]};
    const double offs[2] = {1.0, G->p.T0};
    const double* rowoffs[2] = {G->roff, G->toff};
    for (int k = 0; k < 2 && st == LB_OK; ++k) {
        if (!srcs[k]) continue;
        cudaError_t e = cudaMemcpy(tmp, srcs[k], sizeof(double) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = launch_pack(G->prec, tmp, dsts[k], G->nx, G->ny, G->pitch, G->plane, offs[k], rowoffs[k],
                            G->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
        if (e != cudaSuccess) st = fail(LB_ERR_CUDA, "set_populations: %s", cudaGetErrorString(e));
    }
    cudaFree(tmp);
    return st;
}

lb_status lb_get_window(lb_grid* G, int x0, int y0, int w, int h, double* f, double* g) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    if (!G->has_params) return fail(LB_ERR_STATE, "grid has no parameters: call lb_init first");
    if (g && !G->d.thermal) return fail(LB_ERR_STATE, "thermal populations on a flow-only grid");
    if (w < 1 || h < 1 || w > G->nx || h > G->ny)
        return fail(LB_ERR_ARG, "window %d x %d does not fit a %d x %d grid", w, h, G->nx, G->ny);
    DeviceGuard dg(G->device);
    x0 = ((x0 % G->nx) + G->nx) % G->nx;
    y0 = ((y0 % G->ny) + G->ny) % G->ny;
    const size_t n = (size_t)Q * w * h;
    double* tmp = nullptr;
    CK(cudaMalloc(&tmp, sizeof(double) * n));
    lb_status st = LB_OK;
    double* dsts[2] = {f, g};
    const void* srcs[2] = {G->f[G->cur], G->g[G->cur]};
    const double offs[2] = {1.0, G->p.T0};
    const double* rowoffs[2] = {G->roff, G->toff};
    for (int k = 0; k < 2 && st == LB_OK; ++k) {
        if (!dsts[k]) continue;
        cudaError_t e = launch_unpack(G->prec, srcs[k], tmp, G->nx, G->ny, G->pitch, G->plane, offs[k],
                                      rowoffs[k], x0, y0, w, h, G->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dsts[k], tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, G->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
        if (e != cudaSuccess) st = fail(LB_ERR_CUDA, "get_window: %s", cudaGetErrorString(e));
    }
    cudaFree(tmp);
    return st;
}

lb_status lb_get_populations(lb_grid* G, double* f, double* g) {
    if (!G) return fail(LB_ERR_ARG, "grid is NULL");
    return lb_get_window(G, 0, 0, G->nx, G->ny, f, g);
}

}  // extern "C"
