// lb3_abi.cu -- host side of include/lb3.h: 3-D grid construction, presets,
// parameter checks, kernel dispatch and observables.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/lb3.h"
#include "lb3.cuh"
#include "lb_grid.cuh"

using namespace lbgb;

namespace lbgb {
lb_status set_last_error(lb_status s, const char* msg);
}

struct lb3_grid {
    lb3_grid_desc d{};
    lb3_params p{};
    bool has_params = false;
    bool poisoned = false;
    int device = 0;
    cudaStream_t stream = nullptr;
    Prec prec = Prec::F32;
    int n[3] = {0, 0, 0};
    long long N = 0;
    Axis ax[3];
    void* f[2] = {nullptr, nullptr};
    void* g[2] = {nullptr, nullptr};
    int cur = 0;
    void* work[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // H, FC, HS, HG, GC, HGS
    void* metric[3] = {nullptr, nullptr, nullptr};
    void* faces[3] = {nullptr, nullptr, nullptr};  // face-major metric
    double* width[3] = {nullptr, nullptr, nullptr};
    double* fields = nullptr;  // [5][N] staging
    double* plane = nullptr;   // [nz][8] plane sums
    int* werr = nullptr;       // set by a staged flux pass whose bounded wait ran out
    int fv_sched = LB3_FV_AUTO;
    int sshape[3] = {0, 0, 0};  // staged pass shape: rows per tile, planes per CTA, planes ahead
    int drop_copy = 0;         // test hook of the bounded waits (lb3_debug_drop_copies)
};

namespace {

lb_status fail3(lb_status s, const char* msg) { return set_last_error(s, msg); }

#define CK3(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail3(e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,               \
                         cudaGetErrorString(e_));                                                  \
    } while (0)

struct Dev3 {
    int prev = -1;
    explicit Dev3(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~Dev3() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

size_t rsize(Prec p) { return p == Prec::F64 ? 8 : 4; }

void release3(lb3_grid* G) {
    for (void* q : {G->f[0], G->f[1], G->g[0], G->g[1]})
        if (q) cudaFree(q);
    for (void* q : G->work)
        if (q) cudaFree(q);
    for (int a = 0; a < 3; ++a) {
        if (G->metric[a]) cudaFree(G->metric[a]);
        if (G->faces[a]) cudaFree(G->faces[a]);
        if (G->width[a]) cudaFree(G->width[a]);
    }
    if (G->fields) cudaFree(G->fields);
    if (G->plane) cudaFree(G->plane);
    if (G->werr) cudaFree(G->werr);
}

// Wait limits of the staged flux passes: generous in production (a copy
// group takes microseconds), short under the test hook so that the test
// ends quickly.
constexpr unsigned long long kWaitNs = 500000000ULL, kWaitTestNs = 2000000ULL;

bool staged_ok3(const lb3_grid* G) {
    const int bc[3] = {G->ax[0].bc, G->ax[1].bc, G->ax[2].bc};
    return adv3_staged_ok(G->n, bc, G->prec);
}

// the flux passes a step runs: staged (k3_staged.cu) or plain (k3_adv)
bool staged3(const lb3_grid* G) {
    return G->fv_sched == LB3_FV_STAGED || (G->fv_sched == LB3_FV_AUTO && staged_ok3(G));
}

// LB_ERR_TIMEOUT (and the grid poisoned) when a staged pass reported a wait
// that ran out; synchronises the grid's stream.
lb_status wait_status3(lb3_grid* G) {
    int flag = 0;
    CK3(cudaMemcpyAsync(&flag, G->werr, sizeof(int), cudaMemcpyDeviceToHost, G->stream));
    CK3(cudaStreamSynchronize(G->stream));
    if (flag) {
        G->poisoned = true;
        return fail3(LB_ERR_TIMEOUT, "a bounded wait of a staged flux pass ran out: the step is incomplete and the "
                                     "grid is poisoned until lb3_init");
    }
    return LB_OK;
}

template <typename R>
Args3<R> args3(const lb3_grid* G, bool st) {
    Args3<R> A{};
    A.fin = G->f[G->cur];
    A.fout = G->f[1 - G->cur];
    A.gin = G->g[G->cur];
    A.gout = G->g[1 - G->cur];
    A.H = static_cast<R*>(G->work[0]);
    A.FC = static_cast<R*>(G->work[1]);
    A.HS = static_cast<R*>(G->work[2]);
    A.HG = static_cast<R*>(G->work[3]);
    A.GC = static_cast<R*>(G->work[4]);
    A.HGS = static_cast<R*>(G->work[5]);
    for (int a = 0; a < 3; ++a) {
        A.n[a] = G->n[a];
        A.bc[a] = G->ax[a].bc;
        A.m[a] = AxisMetric<R>{static_cast<const R*>(G->metric[a]), G->n[a] + 1};
        A.ft[a] = static_cast<const R*>(G->faces[a]);
    }
    A.N = G->N;
    A.NP = (long long)G->n[0] * G->n[1] * (G->n[2] + 4);
    const lb3_params& p = G->p;
    const double dt = st ? 1.0 : p.dt;
    const double taut = p.tau + 0.5 * dt, taugt = p.tau_g + 0.5 * dt;  // tau~ = tau + dt/2
    A.dt = (R)dt;
    A.om = (R)(dt / taut);
    A.omh = (R)(dt / (2.0 * taut));
    A.cf = (R)(dt * (1.0 - dt / (2.0 * taut)));
    A.hf = (R)(0.5 * dt);
    A.hF = (R)(0.5 * dt * (1.0 - dt / (2.0 * taut)));
    A.omg = (R)(dt / taugt);
    A.omgh = (R)(dt / (2.0 * taugt));
    A.ax = (R)p.ax;
    A.ay = (R)p.ay;
    A.az = (R)p.az;
    A.bg = (R)(p.beta * p.grav);
    A.T0 = (R)p.T0;
    A.dTb = (R)(p.T_bot - p.T0);
    A.dTt = (R)(p.T_top - p.T0);
    A.werr = G->werr;
    A.drop_copy = G->drop_copy;
    A.wait_ns = G->drop_copy ? kWaitTestNs : kWaitNs;
    for (int q = 0; q < 3; ++q) A.sshape[q] = G->sshape[q];
    return A;
}

Aux3 aux3(const lb3_grid* G) {
    Aux3 a{};
    a.f = G->f[G->cur];
    a.g = G->g[G->cur];
    for (int k = 0; k < 3; ++k) a.n[k] = G->n[k];
    a.N = G->N;
    a.dt = G->p.dt;
    a.ax = G->p.ax;
    a.ay = G->p.ay;
    a.az = G->p.az;
    a.bg = G->p.beta * G->p.grav;
    a.T0 = G->p.T0;
    return a;
}

lb_status ready3(lb3_grid* G) {
    if (!G) return fail3(LB_ERR_ARG, "grid is NULL");
    if (!G->has_params) return fail3(LB_ERR_STATE, "grid has no parameters: call lb3_init first");
    if (G->poisoned) return fail3(LB_ERR_STATE, "grid diverged (LB_ERR_UNSTABLE); call lb3_init again");
    return LB_OK;
}

// SplitMix64 (Steele, Lea & Flood 2014): one step from seed ^ counter, the
// top 53 bits as a uniform number in [0, 1).
double splitmix64_u01(unsigned long long seed, unsigned long long counter) {
    unsigned long long z = (seed ^ counter) + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
}

}  // namespace

extern "C" {

lb_status lb3_create_grid(const lb3_grid_desc* d, lb3_grid** out) {
    if (!d || !out) return fail3(LB_ERR_ARG, "NULL description or output");
    *out = nullptr;
    const int n[3] = {d->nx, d->ny, d->nz}, bc[3] = {d->bcx, d->bcy, d->bcz}, sp[3] = {d->sx, d->sy, d->sz};
    const double L[3] = {d->lx, d->ly, d->lz}, st[3] = {d->stretch_x, d->stretch_y, d->stretch_z};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1) return fail3(LB_ERR_ARG, "cell counts must be >= 1");
        if (bc[a] != LB_BC_PERIODIC && bc[a] != LB_BC_WALLS) return fail3(LB_ERR_ARG, "3-D axes are periodic or walls");
        if (bc[a] == LB_BC_WALLS && n[a] < 2) return fail3(LB_ERR_ARG, "a wall axis needs at least 2 cells");
        if (sp[a] < LB_AXIS_UNIFORM || sp[a] > LB_AXIS_CHEB) return fail3(LB_ERR_ARG, "bad spacing");
        if (sp[a] == LB_AXIS_SINH && (n[a] % 2)) return fail3(LB_ERR_ARG, "sinh spacing needs an even cell count");
        if ((sp[a] == LB_AXIS_TANH || sp[a] == LB_AXIS_SINH) && !(st[a] > 0))
            return fail3(LB_ERR_ARG, "stretch must be > 0");
        if (!(L[a] > 0)) return fail3(LB_ERR_ARG, "domain lengths must be > 0");
    }
    if ((long long)n[0] * n[1] * n[2] > (1LL << 31)) return fail3(LB_ERR_ARG, "grid larger than supported");
    if (d->thermal && (bc[0] != LB_BC_PERIODIC || bc[1] != LB_BC_PERIODIC))
        return fail3(LB_ERR_ARG, "thermal 3-D grids have their plates on z; x and y must be periodic");
    if (d->store != LB_STORE_F64 && d->store != LB_STORE_F32)
        return fail3(LB_ERR_ARG, "3-D grids store FP64 or FP32 populations");
    if (n[2] > 65535) return fail3(LB_ERR_ARG, "nz must be <= 65535");
    lb3_grid* G = new lb3_grid();
    G->d = *d;
    G->prec = d->store == LB_STORE_F64 ? Prec::F64 : Prec::F32;
    G->stream = static_cast<cudaStream_t>(d->cuda_stream);
    cudaGetDevice(&G->device);
    G->N = (long long)n[0] * n[1] * n[2];
    for (int a = 0; a < 3; ++a) {
        G->n[a] = n[a];
        G->ax[a] = make_axis(n[a], L[a], sp[a], st[a], bc[a]);
    }
    auto bail = [&](cudaError_t e) {
        release3(G);
        delete G;
        return fail3(e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, cudaGetErrorString(e));
    };
    const size_t pop = (size_t)Q3 * G->N * rsize(G->prec);
    const int sets = d->thermal ? 2 : 1;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaMalloc(&G->f[b], pop);
        if (e == cudaSuccess && d->thermal) e = cudaMalloc(&G->g[b], pop);
    }
    // h, h* (and hg, hg*) carry two ghost planes on each side in z; f + Coll does not
    const size_t padded = (size_t)Q3 * n[0] * n[1] * (n[2] + 4) * rsize(G->prec);
    for (int w = 0; w < 3 * sets && e == cudaSuccess; ++w) e = cudaMalloc(&G->work[w], w % 3 == 1 ? pop : padded);
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        const std::vector<double> m = G->ax[a].metric();
        const int n1 = n[a] + 1;
        std::vector<double> fm((size_t)kFaceRow * n1, 0.0);
        for (int k = 0; k < n1; ++k) {
            for (int r = 0; r < 6; ++r) fm[(size_t)kFaceRow * k + r] = m[(size_t)r * n1 + k];
            if (k < n[a]) fm[(size_t)kFaceRow * k + 6] = m[(size_t)6 * n1 + k];
        }
        if (G->prec == Prec::F64) {
            e = cudaMalloc(&G->metric[a], sizeof(double) * m.size());
            if (e == cudaSuccess) e = cudaMemcpy(G->metric[a], m.data(), sizeof(double) * m.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMalloc(&G->faces[a], sizeof(double) * fm.size());
            if (e == cudaSuccess) e = cudaMemcpy(G->faces[a], fm.data(), sizeof(double) * fm.size(), cudaMemcpyHostToDevice);
        } else {
            std::vector<float> mf(m.begin(), m.end()), ff(fm.begin(), fm.end());
            e = cudaMalloc(&G->metric[a], sizeof(float) * mf.size());
            if (e == cudaSuccess) e = cudaMemcpy(G->metric[a], mf.data(), sizeof(float) * mf.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMalloc(&G->faces[a], sizeof(float) * ff.size());
            if (e == cudaSuccess) e = cudaMemcpy(G->faces[a], ff.data(), sizeof(float) * ff.size(), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) e = cudaMalloc(&G->width[a], sizeof(double) * n[a]);
        if (e == cudaSuccess)
            e = cudaMemcpy(G->width[a], G->ax[a].d.data(), sizeof(double) * n[a], cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&G->fields, sizeof(double) * 5 * G->N);
    if (e == cudaSuccess) e = cudaMalloc(&G->plane, sizeof(double) * 8 * n[2]);
    if (e == cudaSuccess) e = cudaMalloc(&G->werr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(G->werr, 0, sizeof(int));
    if (e != cudaSuccess) return bail(e);
    *out = G;
    return LB_OK;
}

lb_status lb3_init(lb3_grid* G, const lb3_params* p, const lb3_init_desc* in) {
    if (!G || !p || !in) return fail3(LB_ERR_ARG, "NULL argument");
    if (!(p->tau > 0) || !(p->dt > 0)) return fail3(LB_ERR_ARG, "tau and dt must be > 0");
    if (G->d.thermal && !(p->tau_g > 0)) return fail3(LB_ERR_ARG, "tau_g must be > 0 on a thermal grid");
    if (in->kind != LB_INIT_TGV && in->kind != LB_INIT_SHEAR && in->kind != LB_INIT_RB && in->kind != LB_INIT_FIELDS)
        return fail3(LB_ERR_ARG, "3-D presets: TGV, SHEAR, RB or FIELDS");
    if (in->kind == LB_INIT_RB && !G->d.thermal) return fail3(LB_ERR_ARG, "RB preset needs a thermal grid");
    Dev3 dg(G->device);
    const int nx = G->n[0], ny = G->n[1], nz = G->n[2];
    const long long N = G->N;
    std::vector<double> h(5 * (size_t)N);
    const double twopi = 6.283185307179586476925286766559;
    const double Lx = G->d.lx, Ly = G->d.ly, Lz = G->d.lz, dT = p->T_bot - p->T_top, bg = p->beta * p->grav;
    double norm = 1.0;
    auto baro = [&](double z) { return std::exp(3.0 * bg * dT * (0.5 * z - 0.5 * z * z / Lz)); };
    if (in->kind == LB_INIT_RB) {
        double s = 0.0;
        for (int k = 0; k < nz; ++k) s += G->ax[2].d[k] * baro(G->ax[2].c[k]);
        norm = Lz / s;  // volume mean of rho = 1
    }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long long c = ((long long)k * ny + j) * nx + i;
                const double x = G->ax[0].c[i], y = G->ax[1].c[j], z = G->ax[2].c[k];
                double rho = 1.0, ux = 0.0, uy = 0.0, uz = 0.0, T = p->T0;
                if (in->kind == LB_INIT_TGV) {
                    const double kx = twopi / Lx, ky = twopi / Ly, kz = twopi / Lz;
                    ux = in->u0 * std::sin(kx * x) * std::cos(ky * y) * std::cos(kz * z);
                    uy = -in->u0 * (kx / ky) * std::cos(kx * x) * std::sin(ky * y) * std::cos(kz * z);
                    rho = 1.0 + 3.0 * (in->u0 * in->u0 / 16.0) * (std::cos(2.0 * kx * x) + std::cos(2.0 * ky * y)) *
                                    (std::cos(2.0 * kz * z) + 2.0);
                } else if (in->kind == LB_INIT_SHEAR) {
                    ux = in->amp * std::sin(twopi * in->mode * z / Lz);
                } else if (in->kind == LB_INIT_RB) {
                    const double U = splitmix64_u01(in->seed, (unsigned long long)c);
                    T = p->T0 + dT * (0.5 - z / Lz) + in->amp * dT * (2.0 * U - 1.0);
                    rho = norm * baro(z);
                } else {
                    if (in->rho) rho = in->rho[c];
                    if (in->ux) ux = in->ux[c];
                    if (in->uy) uy = in->uy[c];
                    if (in->uz) uz = in->uz[c];
                    if (in->T) T = in->T[c];
                    if (!(rho > 0)) return fail3(LB_ERR_ARG, "density must be > 0");
                }
                h[c] = rho;
                h[N + c] = ux;
                h[2 * N + c] = uy;
                h[3 * N + c] = uz;
                h[4 * N + c] = T;
            }
    G->p = *p;
    CK3(cudaMemcpyAsync(G->fields, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, G->stream));
    G->cur = 0;
    Aux3 a = aux3(G);
    CK3(launch3_init(G->prec, G->d.thermal != 0, a, G->fields, G->f[0], G->g[0], G->stream));
    CK3(cudaMemsetAsync(G->werr, 0, sizeof(int), G->stream));
    CK3(cudaStreamSynchronize(G->stream));  // h is released on return
    G->has_params = true;
    G->poisoned = false;
    return LB_OK;
}

// one FV step on the grid's stream with its current schedule; flips cur
static cudaError_t fv3_step(lb3_grid* G) {
    const bool staged = staged3(G);
    cudaError_t e;
    if (G->prec == Prec::F64) {
        Args3<double> A = args3<double>(G, false);
        e = launch3_fv(G->prec, G->d.thermal != 0, staged, &A, G->stream);
    } else {
        Args3<float> A = args3<float>(G, false);
        e = launch3_fv(G->prec, G->d.thermal != 0, staged, &A, G->stream);
    }
    G->cur ^= 1;
    return e;
}

lb_status lb3_step_fv(lb3_grid* G, int nsteps) {
    lb_status s = ready3(G);
    if (s != LB_OK) return s;
    if (nsteps < 0) return fail3(LB_ERR_ARG, "nsteps must be >= 0");
    Dev3 dg(G->device);
    for (int k = 0; k < nsteps; ++k) CK3(fv3_step(G));
    return LB_OK;
}

lb_status lb3_autotune_fv(lb3_grid* G, int steps) {
    lb_status s = ready3(G);
    if (s != LB_OK) return s;
    if (steps < 1) return fail3(LB_ERR_ARG, "steps must be >= 1");
    Dev3 dg(G->device);
    const size_t bytes = (size_t)Q3 * G->N * rsize(G->prec);
    void *sf = nullptr, *sg = nullptr;
    CK3(cudaMalloc(&sf, bytes));
    if (G->d.thermal && cudaMalloc(&sg, bytes) != cudaSuccess) {
        cudaFree(sf);
        return fail3(LB_ERR_OOM, "autotune: no memory for the state copy");
    }
    const int cur0 = G->cur, sched0 = G->fv_sched, shape0[3] = {G->sshape[0], G->sshape[1], G->sshape[2]};
    cudaMemcpyAsync(sf, G->f[cur0], bytes, cudaMemcpyDeviceToDevice, G->stream);
    if (sg) cudaMemcpyAsync(sg, G->g[cur0], bytes, cudaMemcpyDeviceToDevice, G->stream);
    struct Cand {
        int sched, rows, planes, ahead;
    };
    std::vector<Cand> cands = {{LB3_FV_PLAIN, 0, 0, 0}};
    if (staged_ok3(G)) {
        int ty = 0, kc = 0, ah = 0;
        adv3_staged_resolve(G->n, G->prec, &ty, &kc, &ah);
        for (int rows : {ty, ty / 2})
            for (int planes : {16, 32})
                for (int ahead : {2, 3})
                    if (rows >= 1 && adv3_staged_shape_ok(G->n, G->prec, rows, planes, ahead))
                        cands.push_back({LB3_FV_STAGED, rows, planes, ahead});
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Cand pick = cands[0];
    lb_status st = LB_OK;
    for (const Cand& c : cands) {
        G->fv_sched = c.sched;
        G->sshape[0] = c.rows;
        G->sshape[1] = c.planes;
        G->sshape[2] = c.ahead;
        G->cur = cur0;
        cudaError_t e = fv3_step(G);  // warm-up, then the timed steps
        cudaEventRecord(e0, G->stream);
        for (int k = 0; k < steps && e == cudaSuccess; ++k) e = fv3_step(G);
        cudaEventRecord(e1, G->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            st = fail3(LB_ERR_CUDA, cudaGetErrorString(e));
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
    if (st == LB_OK) st = wait_status3(G);  // a timed step whose wait ran out
    if (st != LB_OK) {
        G->fv_sched = sched0;
        for (int q = 0; q < 3; ++q) G->sshape[q] = shape0[q];
        return st;
    }
    G->fv_sched = pick.sched;
    G->sshape[0] = pick.rows;
    G->sshape[1] = pick.planes;
    G->sshape[2] = pick.ahead;
    return LB_OK;
}

lb_status lb3_step_st(lb3_grid* G, int nsteps) {
    lb_status s = ready3(G);
    if (s != LB_OK) return s;
    if (nsteps < 0) return fail3(LB_ERR_ARG, "nsteps must be >= 0");
    for (int a = 0; a < 3; ++a)
        if ((a == 0 ? G->d.sx : a == 1 ? G->d.sy : G->d.sz) != LB_AXIS_UNIFORM ||
            std::fabs(G->ax[a].L / G->n[a] - 1.0) > 1e-12)
            return fail3(LB_ERR_ARG, "ST needs uniform axes with unit spacing");
    if (std::fabs(G->p.dt - 1.0) > 1e-12) return fail3(LB_ERR_ARG, "ST needs dt = 1");
    Dev3 dg(G->device);
    for (int k = 0; k < nsteps; ++k) {
        if (G->prec == Prec::F64) {
            Args3<double> A = args3<double>(G, true);
            CK3(launch3_st(G->prec, G->d.thermal != 0, &A, G->stream));
        } else {
            Args3<float> A = args3<float>(G, true);
            CK3(launch3_st(G->prec, G->d.thermal != 0, &A, G->stream));
        }
        G->cur ^= 1;
    }
    return LB_OK;
}

lb_status lb3_moments(lb3_grid* G, double* rho, double* ux, double* uy, double* uz, double* T) {
    lb_status s = ready3(G);
    if (s != LB_OK) return s;
    Dev3 dg(G->device);
    if ((s = wait_status3(G)) != LB_OK) return s;
    CK3(launch3_moments(G->prec, G->d.thermal != 0, aux3(G), G->fields, G->stream));
    double* outs[5] = {rho, ux, uy, uz, T};
    for (int q = 0; q < 5; ++q)
        if (outs[q])
            CK3(cudaMemcpyAsync(outs[q], G->fields + q * G->N, sizeof(double) * G->N, cudaMemcpyDeviceToHost,
                                G->stream));
    CK3(cudaStreamSynchronize(G->stream));
    return LB_OK;
}

// Per-plane sums on the device, then a fixed-order sum over planes here.
static lb_status plane_sums3(lb3_grid* G, std::vector<double>& ps) {
    Dev3 dg(G->device);
    const lb_status s = wait_status3(G);
    if (s != LB_OK) return s;
    CK3(launch3_moments(G->prec, G->d.thermal != 0, aux3(G), G->fields, G->stream));
    CK3(launch3_plane_sums(G->fields, G->width[0], G->width[1], G->width[2], G->n[0], G->n[1], G->n[2],
                           G->p.T0, G->plane, G->stream));
    ps.assign(8 * (size_t)G->n[2], 0.0);
    CK3(cudaMemcpyAsync(ps.data(), G->plane, sizeof(double) * ps.size(), cudaMemcpyDeviceToHost, G->stream));
    CK3(cudaStreamSynchronize(G->stream));
    return LB_OK;
}

lb_status lb3_conservation(lb3_grid* G, double* mass, double* mx, double* my, double* mz, double* heat) {
    lb_status s = ready3(G);
    if (s != LB_OK) return s;
    std::vector<double> ps;
    s = plane_sums3(G, ps);
    if (s != LB_OK) return s;
    double t[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < G->n[2]; ++k)
        for (int q = 0; q < 5; ++q) t[q] += ps[8 * k + q];
    for (double v : t)
        if (!std::isfinite(v)) {
            G->poisoned = true;
            return fail3(LB_ERR_UNSTABLE, "non-finite conservation sums: the run has diverged");
        }
    if (mass) *mass = t[0];
    if (mx) *mx = t[1];
    if (my) *my = t[2];
    if (mz) *mz = t[3];
    if (heat) *heat = t[4];
    return LB_OK;
}

lb_status lb3_nusselt(lb3_grid* G, double* nu_vol, double* nu_bot, double* nu_top) {
    lb_status s = ready3(G);
    if (s != LB_OK) return s;
    if (!G->d.thermal) return fail3(LB_ERR_STATE, "Nusselt numbers need a thermal grid");
    std::vector<double> ps;
    s = plane_sums3(G, ps);
    if (s != LB_OK) return s;
    const int nz = G->n[2];
    const double H = G->d.lz, dT = G->p.T_bot - G->p.T_top, kappa = G->p.tau_g / 3.0;
    const double area = G->d.lx * G->d.ly;
    double flux = 0.0, vol = 0.0;
    std::vector<double> Tm(nz);
    for (int k = 0; k < nz; ++k) {
        flux += ps[8 * k + 5];
        vol += ps[8 * k + 7];
        Tm[k] = ps[8 * k + 6] / area;
    }
    if (nu_vol) *nu_vol = 1.0 + H * (flux / vol) / (kappa * dT);
    if (nz >= 2) {
        const double z0 = G->ax[2].c[0], z1 = G->ax[2].c[1];
        const double d = -(z0 + z1) / (z0 * z1) * G->p.T_bot + z1 / (z0 * (z1 - z0)) * Tm[0] -
                         z0 / (z1 * (z1 - z0)) * Tm[1];
        if (nu_bot) *nu_bot = -H * d / dT;
        const double s0 = H - G->ax[2].c[nz - 1], s1 = H - G->ax[2].c[nz - 2];
        const double e = -(s0 + s1) / (s0 * s1) * G->p.T_top + s1 / (s0 * (s1 - s0)) * Tm[nz - 1] -
                         s0 / (s1 * (s1 - s0)) * Tm[nz - 2];
        if (nu_top) *nu_top = H * e / dT;
    }
    return LB_OK;
}

lb_status lb3_set_populations(lb3_grid* G, const double* f, const double* g) {
    if (!G || !f) return fail3(LB_ERR_ARG, "NULL argument");
    if (!G->has_params) return fail3(LB_ERR_STATE, "set parameters with lb3_init before setting populations");
    Dev3 dg(G->device);
    double* tmp = nullptr;
    const size_t bytes = sizeof(double) * Q3 * G->N;
    CK3(cudaMalloc(&tmp, bytes));
    // copies and packing in order on the grid's stream
    cudaError_t e = cudaMemcpyAsync(tmp, f, bytes, cudaMemcpyHostToDevice, G->stream);
    if (e == cudaSuccess) e = launch3_pack(G->prec, tmp, G->f[G->cur], G->N, 1.0, G->stream);
    if (e == cudaSuccess && g && G->d.thermal) {
        e = cudaMemcpyAsync(tmp, g, bytes, cudaMemcpyHostToDevice, G->stream);
        if (e == cudaSuccess) e = launch3_pack(G->prec, tmp, G->g[G->cur], G->N, G->p.T0, G->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail3(LB_ERR_CUDA, cudaGetErrorString(e));
    G->poisoned = false;
    return LB_OK;
}

lb_status lb3_get_populations(lb3_grid* G, double* f, double* g) {
    if (!G) return fail3(LB_ERR_ARG, "NULL grid");
    if (!G->has_params) return fail3(LB_ERR_STATE, "grid has no parameters: call lb3_init first");
    Dev3 dg(G->device);
    double* tmp = nullptr;
    const size_t bytes = sizeof(double) * Q3 * G->N;
    CK3(cudaMalloc(&tmp, bytes));
    cudaError_t e = cudaSuccess;
    if (f) {
        e = launch3_unpack(G->prec, G->f[G->cur], tmp, G->N, 1.0, G->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(f, tmp, bytes, cudaMemcpyDeviceToHost, G->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
    }
    if (e == cudaSuccess && g && G->d.thermal) {
        e = launch3_unpack(G->prec, G->g[G->cur], tmp, G->N, G->p.T0, G->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g, tmp, bytes, cudaMemcpyDeviceToHost, G->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
    }
    cudaFree(tmp);
    if (e != cudaSuccess) return fail3(LB_ERR_CUDA, cudaGetErrorString(e));
    return LB_OK;
}

lb_status lb3_sync(lb3_grid* G) {
    if (!G) return fail3(LB_ERR_ARG, "NULL grid");
    Dev3 dg(G->device);
    CK3(cudaStreamSynchronize(G->stream));
    return wait_status3(G);
}

lb_status lb3_set_fv_schedule(lb3_grid* G, int schedule) {
    if (!G) return fail3(LB_ERR_ARG, "NULL grid");
    if (schedule != LB3_FV_AUTO && schedule != LB3_FV_PLAIN && schedule != LB3_FV_STAGED)
        return fail3(LB_ERR_ARG, "schedule must be LB3_FV_AUTO, LB3_FV_PLAIN or LB3_FV_STAGED");
    if (schedule == LB3_FV_STAGED && !staged_ok3(G))
        return fail3(LB_ERR_ARG, "the staged flux passes need x and y periodic and nx a power of two <= 256 "
                                 "with rows a multiple of 16 bytes");
    G->fv_sched = schedule;
    return LB_OK;
}

lb_status lb3_set_fv_staged_shape(lb3_grid* G, int rows, int planes, int ahead) {
    if (!G) return fail3(LB_ERR_ARG, "NULL grid");
    if (!adv3_staged_shape_ok(G->n, G->prec, rows, planes, ahead))
        return fail3(LB_ERR_ARG, "staged shape out of range: rows per tile 0..(1024 cells / nx, FP64 512), "
                                 "planes per CTA 0..256, planes ahead 0..12, within the shared memory");
    G->sshape[0] = rows;
    G->sshape[1] = planes;
    G->sshape[2] = ahead;
    return LB_OK;
}

lb_status lb3_get_fv_schedule(lb3_grid* G, int* resolved) {
    if (!G || !resolved) return fail3(LB_ERR_ARG, "NULL argument");
    *resolved = staged3(G) ? LB3_FV_STAGED : LB3_FV_PLAIN;
    return LB_OK;
}

lb_status lb3_get_fv_staged_shape(lb3_grid* G, int* rows, int* planes, int* ahead) {
    if (!G || !rows || !planes || !ahead) return fail3(LB_ERR_ARG, "NULL argument");
    int r = G->sshape[0], p = G->sshape[1], a = G->sshape[2];
    adv3_staged_resolve(G->n, G->prec, &r, &p, &a);
    *rows = r;
    *planes = p;
    *ahead = a;
    return LB_OK;
}

lb_status lb3_debug_drop_copies(lb3_grid* G, int on) {
    if (!G) return fail3(LB_ERR_ARG, "NULL grid");
    G->drop_copy = on != 0;
    return LB_OK;
}

lb_status lb3_destroy(lb3_grid* G) {
    if (!G) return LB_OK;
    Dev3 dg(G->device);
    cudaStreamSynchronize(G->stream);
    release3(G);
    delete G;
    return LB_OK;
}

}  // extern "C"
