// lb_grid.cuh -- the library's grid object and the 1-D grid metric
// (private to the library; the C ABI sees lb_grid as an opaque type).
#pragma once

#include <cmath>
#include <vector>

#include "lb_internal.cuh"

namespace lbgb {

// Face coordinates of one axis, Eq. (grids) of Sec. III B.
inline std::vector<double> axis_faces(int n, double L, int sp, double st) {
    std::vector<double> xi(n + 1);
    for (int i = 0; i <= n; ++i) {
        const double s = (double)i / n;
        if (sp == LB_AXIS_TANH) {
            xi[i] = 0.5 * L * (1.0 + std::tanh((2.0 * s - 1.0) * st) / std::tanh(st));
        } else if (sp == LB_AXIS_SINH) {
            const double amp = 0.5 * L / std::sinh(0.5 * st);
            xi[i] = 2 * i <= n ? amp * std::sinh(st * s) : L - amp * std::sinh(st * (double)(n - i) / n);
        } else if (sp == LB_AXIS_CHEB) {
            xi[i] = 0.5 * L * (1.0 - std::cos(3.14159265358979323846 * s));
        } else {
            xi[i] = L * s;
        }
    }
    xi[0] = 0.0;
    xi[n] = L;
    return xi;
}

struct Axis {
    int n = 0;
    double L = 0;
    int bc = 0;
    std::vector<double> xi, c, d;
    // centre of any integer cell index: periodic repeats shifted by L, walls
    // mirror the fluid centres about the wall face (ghost centres, Sec. II B 5)
    double pos(int i) const {
        if (i >= 0 && i < n) return c[i];
        if (bc == LB_BC_PERIODIC) {
            int q = i >= 0 ? i / n : -((-i + n - 1) / n);
            return c[i - q * n] + q * L;
        }
        return i < 0 ? 2.0 * xi[0] - c[-i - 1] : 2.0 * xi[n] - c[2 * n - 1 - i];
    }
    // Lagrange weights of the parabola through cells (k0, k0+1, k0+2) at face k:
    // the QUICK coefficients of Sec. II B 3 (gamma_1 = weight of the
    // downstream node, gamma_2 = -weight of the far upstream node).
    void quick(int k0, int k, double w[3]) const {
        const double p[3] = {pos(k0), pos(k0 + 1), pos(k0 + 2)};
        const double x = xi[k];
        w[0] = (x - p[1]) * (x - p[2]) / ((p[0] - p[1]) * (p[0] - p[2]));
        w[1] = (x - p[0]) * (x - p[2]) / ((p[1] - p[0]) * (p[1] - p[2]));
        w[2] = (x - p[0]) * (x - p[1]) / ((p[2] - p[0]) * (p[2] - p[1]));
    }
    // [6][n+1] weights then [n] inverse widths
    std::vector<double> metric() const {
        std::vector<double> m(7 * (n + 1), 0.0);
        for (int k = 0; k <= n; ++k) {
            double w[3];
            quick(k - 2, k, w);
            for (int r = 0; r < 3; ++r) m[r * (n + 1) + k] = w[r];
            quick(k - 1, k, w);
            for (int r = 0; r < 3; ++r) m[(3 + r) * (n + 1) + k] = w[r];
        }
        for (int i = 0; i < n; ++i) m[6 * (n + 1) + i] = 1.0 / d[i];
        return m;
    }
};

inline Axis make_axis(int n, double L, int sp, double st, int bc) {
    Axis a;
    a.n = n;
    a.L = L;
    a.bc = bc;
    a.xi = axis_faces(n, L, sp, st);
    a.c.resize(n);
    a.d.resize(n);
    for (int i = 0; i < n; ++i) {
        a.c[i] = 0.5 * (a.xi[i] + a.xi[i + 1]);
        a.d[i] = a.xi[i + 1] - a.xi[i];
    }
    return a;
}

inline Prec prec_of(int store) {
    switch (store) {
        case LB_STORE_F64: return Prec::F64;
        case LB_STORE_F16DEV: return Prec::F16;
        case LB_STORE_BF16DEV: return Prec::BF16;
        default: return Prec::F32;
    }
}

inline size_t elem_size(int store) {
    return store == LB_STORE_F64 ? 8 : (store == LB_STORE_F32 ? 4 : 2);
}

}  // namespace lbgb

struct lb_grid {
    lb_grid_desc d{};
    lb_params p{};
    bool has_params = false;
    bool poisoned = false;
    int device = 0;
    cudaStream_t stream = nullptr;
    lbgb::Prec prec = lbgb::Prec::F32;
    int nx = 0, ny = 0, pitch = 0;
    long long plane = 0;
    lbgb::Axis ax, ay;
    double dmin = 0;
    void* f[2] = {nullptr, nullptr};
    void* g[2] = {nullptr, nullptr};
    int cur = 0;
    void* mx = nullptr;  // metric in compute precision
    void* my = nullptr;
    double *dxv = nullptr, *dyv = nullptr, *xc = nullptr, *yc = nullptr;
    double* toff = nullptr;     // per-row storage offset of g, FP64 (ny)
    void* toff_r = nullptr;     // the same in compute precision
    double* roff = nullptr;     // per-row storage offset of f, FP64 (ny)
    void* roff_r = nullptr;
    void* dref_r = nullptr;     // [4][ny] y flux divergence of the base state, compute precision
    float* rowtab = nullptr;    // [ny][20] y weights, 1/dy, offsets, base-state fluxes (paired kernels)
    float* coltab = nullptr;    // [nx][20] x weights of a column pair and its 1/dx (paired tile kernel)
    float* xh = nullptr;        // split schedule: h*, [NQ][ny][pitch] FP32 (allocated on first use)
    float* xfc = nullptr;       // split schedule: f~ + Coll - dt/2 A[h^n]
    double* fields = nullptr;   // [4][ny][nx] staging for init/moments
    double* partial = nullptr;  // reduction partials
    double* red = nullptr;      // reduction totals
    int nred = 0;
    int fv_scheme = LB_FV_HEUN;  // time integration of lb_step_fv
    double rho_bc[4] = {1.0, 1.0, 1.0, 1.0};  // imposed densities of LB_BC_DENSITY axes
    int fv_kernel = LB_FV_AUTO;  // requested schedule
    int fv_chunk = 0;
    int sms = 0;                 // streaming multiprocessors of the device
    int graph_steps = 32;        // steps per captured graph of long step runs (0: launch step by step)
    cudaStream_t cap = nullptr;  // private stream the step graphs are captured on (created on first use)
    unsigned long long graph_replays = 0;
};


namespace lbgb {

template <typename R>
inline StepArgs<R> step_args(const lb_grid* G, double dt) {
    StepArgs<R> A{};
    A.fin = G->f[G->cur];
    A.fout = G->f[1 - G->cur];
    A.gin = G->g[G->cur];
    A.gout = G->g[1 - G->cur];
    A.nx = G->nx;
    A.ny = G->ny;
    A.pitch = G->pitch;
    A.plane = G->plane;
    A.bcx = G->d.bcx;
    A.bcy = G->d.bcy;
    A.mx = AxisMetric<R>{static_cast<const R*>(G->mx), G->nx + 1};
    A.my = AxisMetric<R>{static_cast<const R*>(G->my), G->ny + 1};
    const lb_params& p = G->p;
    const double taut = p.tau + 0.5 * dt, taugt = p.tau_g + 0.5 * dt;  // tau~ = tau + dt/2
    A.dt = (R)dt;
    A.om = (R)(dt / taut);
    A.omh = (R)(dt / (2.0 * taut));
    A.cf = (R)(dt * (1.0 - dt / (2.0 * taut)));
    A.hf = (R)(0.5 * dt);
    // the advected field is the plain population f (Appendix A inverts the
    // tilde transformation): its force part is dt/2 (1 - dt/(2 tau~)) F
    A.hF = (R)(0.5 * dt * (1.0 - dt / (2.0 * taut)));
    A.omg = (R)(dt / taugt);
    A.omgh = (R)(dt / (2.0 * taugt));
    A.stages = G->fv_scheme == LB_FV_HEUN ? 2 : 1;
    if (G->fv_scheme == LB_FV_EULER) {
        // Eq. (euler): h = f, source dt/tau (f_eq - f) + dt F, u = sum c f / rho
        A.om = (R)(dt / p.tau);
        A.omh = (R)0;
        A.cf = (R)dt;
        A.hf = (R)0;
        A.hF = (R)0;
        A.omg = (R)(dt / p.tau_g);
        A.omgh = (R)0;
    }
    A.ax = (R)p.ax;
    A.ay = (R)p.ay;
    A.bg = (R)(p.beta * p.grav);
    A.dTb = (R)(p.T_bot - p.T0);
    A.dTt = (R)(p.T_top - p.T0);
    A.T0 = (R)p.T0;
    for (int k = 0; k < 4; ++k) A.rhobd[k] = (R)(G->rho_bc[k] - 1.0);
    A.toff = static_cast<const R*>(G->toff_r);
    A.roff = static_cast<const R*>(G->roff_r);
    A.dref = static_cast<const R*>(G->dref_r);
    A.rowtab = G->rowtab;
    A.coltab = G->coltab;
    A.xh = G->xh;
    A.xfc = G->xfc;
    return A;
}

}  // namespace lbgb
