/*
 * lbref3.c -- plain FP64 CPU oracle of the D3Q19 step (see lbref3.h).
 *
 * TEST INFRASTRUCTURE ONLY.  The same algorithm as lbref.c, written out for
 * three dimensions: one cell and one population at a time, in the paper's
 * order (Sec. II: equilibrium and Guo force, Eq. (F2); Eq. (ST); Eqs. (semi)
 * and (semi-heun) with QUICK faces, Sec. II B 3; double-reflection walls,
 * Sec. II B 5).  Faces of a diagonal population are taken dimension by
 * dimension, each from the nodes on its own grid line, and the isothermal
 * plates anti-reflect the thermal advected field, as in two dimensions.
 * OpenMP (if enabled) splits only the outer loop over z planes of the
 * per-cell loops; no floating-point sum changes order.
 */
#include "lbref3.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q3 19

/* D3Q19: rest, six axis neighbours (w = 1/18), twelve edge neighbours
 * (w = 1/36); opposite velocities are adjacent, inv(a) = a +- 1. */
static const int CX3[Q3] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY3[Q3] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ3[Q3] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double W3[Q3] = {1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                              1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int INV3[Q3] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};

struct ref3_grid {
    ref3_desc d;
    ref3_params p;
    int has_params;
    int n[3];
    double L[3];
    int bc[3];
    double *xi[3], *c[3], *w[3], *pos[3]; /* faces, centres, widths, centres incl. 2 ghosts */
    double *f, *g, *h, *hg, *coll, *collg, *adv, *advg, *adv2, *advg2, *fs, *gs, *fn, *gn;
};

#define I3(G, a, i, j, k) ((((size_t)(a) * (G)->n[2] + (k)) * (G)->n[1] + (j)) * (G)->n[0] + (i))
#define P3(G, a, i, j, k) \
    ((((size_t)(a) * ((G)->n[2] + 4) + (k) + 2) * ((G)->n[1] + 4) + (j) + 2) * ((G)->n[0] + 4) + (i) + 2)

/* The D3Q19 velocities, weights and opposite-velocity map (Sec. II). */
void ref3_lattice(int* cx, int* cy, int* cz, double* w, int* inv) {
    for (int a = 0; a < Q3; ++a) {
        if (cx) cx[a] = CX3[a];
        if (cy) cy[a] = CY3[a];
        if (cz) cz[a] = CZ3[a];
        if (w) w[a] = W3[a];
        if (inv) inv[a] = INV3[a];
    }
}

/* Second-order BGK equilibrium on D3Q19 (c_s^2 = 1/3). */
void ref3_equilibrium(double rho, double ux, double uy, double uz, double* feq) {
    double uu = ux * ux + uy * uy + uz * uz;
    for (int a = 0; a < Q3; ++a) {
        double cu = CX3[a] * ux + CY3[a] * uy + CZ3[a] * uz;
        feq[a] = W3[a] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* Guo force, Eq. (F2): w [ (c - u)/cs^2 + (c.u) c / cs^4 ] . rho a. */
void ref3_guo_force(double rho, double ux, double uy, double uz, double ax, double ay, double az,
                    double* F) {
    for (int a = 0; a < Q3; ++a) {
        double cu = CX3[a] * ux + CY3[a] * uy + CZ3[a] * uz;
        double ex = 3.0 * (CX3[a] - ux) + 9.0 * cu * CX3[a];
        double ey = 3.0 * (CY3[a] - uy) + 9.0 * cu * CY3[a];
        double ez = 3.0 * (CZ3[a] - uz) + 9.0 * cu * CZ3[a];
        F[a] = W3[a] * rho * (ex * ax + ey * ay + ez * az);
    }
}

static double* zalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

/* centre of any cell index of an axis (periodic images or mirrored ghosts) */
static double axis_pos3(const ref3_grid* G, int ax, int i) {
    const int n = G->n[ax];
    if (i >= 0 && i < n) return G->c[ax][i];
    if (G->bc[ax] == REF_PERIODIC) {
        int q = (i >= 0) ? i / n : -((-i + n - 1) / n);
        return G->c[ax][i - q * n] + q * G->L[ax];
    }
    if (i < 0) return 2.0 * G->xi[ax][0] - G->c[ax][-i - 1];
    return 2.0 * G->xi[ax][n] - G->c[ax][2 * n - 1 - i];
}

ref3_grid* ref3_create(const ref3_desc* d) {
    if (!d || d->nx < 1 || d->ny < 1 || d->nz < 1) return NULL;
    const int n[3] = {d->nx, d->ny, d->nz}, bc[3] = {d->bcx, d->bcy, d->bcz};
    const int sp[3] = {d->sx, d->sy, d->sz};
    for (int a = 0; a < 3; ++a) {
        if (bc[a] != REF_PERIODIC && bc[a] != REF_WALLS) return NULL;
        if (bc[a] == REF_WALLS && n[a] < 2) return NULL;
        if (sp[a] == REF_SINH && (n[a] % 2)) return NULL;
    }
    if (d->thermal && (d->bcx != REF_PERIODIC || d->bcy != REF_PERIODIC)) return NULL;
    ref3_grid* G = (ref3_grid*)calloc(1, sizeof(ref3_grid));
    G->d = *d;
    const double L[3] = {d->lx, d->ly, d->lz}, st[3] = {d->stretch_x, d->stretch_y, d->stretch_z};
    for (int a = 0; a < 3; ++a) {
        G->n[a] = n[a];
        G->L[a] = L[a];
        G->bc[a] = bc[a];
        G->xi[a] = zalloc(n[a] + 1);
        G->c[a] = zalloc(n[a]);
        G->w[a] = zalloc(n[a]);
        G->pos[a] = zalloc(n[a] + 4);
        ref_faces(n[a], L[a], sp[a], st[a], G->xi[a]);
        for (int i = 0; i < n[a]; ++i) {
            G->c[a][i] = 0.5 * (G->xi[a][i] + G->xi[a][i + 1]);
            G->w[a][i] = G->xi[a][i + 1] - G->xi[a][i];
        }
    }
    for (int a = 0; a < 3; ++a)
        for (int i = -2; i < n[a] + 2; ++i) G->pos[a][i + 2] = axis_pos3(G, a, i);
    const size_t N = (size_t)Q3 * n[0] * n[1] * n[2];
    const size_t NP = (size_t)Q3 * (n[0] + 4) * (n[1] + 4) * (n[2] + 4);
    double** bufs[] = {&G->f, &G->g, &G->coll, &G->collg, &G->adv, &G->advg, &G->adv2,
                       &G->advg2, &G->fs, &G->gs, &G->fn, &G->gn};
    for (size_t k = 0; k < sizeof(bufs) / sizeof(bufs[0]); ++k) *bufs[k] = zalloc(N);
    G->h = zalloc(NP);
    G->hg = zalloc(NP);
    return G;
}

void ref3_destroy(ref3_grid* G) {
    if (!G) return;
    for (int a = 0; a < 3; ++a) {
        free(G->xi[a]);
        free(G->c[a]);
        free(G->w[a]);
        free(G->pos[a]);
    }
    double* bufs[] = {G->f, G->g, G->h, G->hg, G->coll, G->collg, G->adv, G->advg, G->adv2,
                      G->advg2, G->fs, G->gs, G->fn, G->gn};
    for (size_t k = 0; k < sizeof(bufs) / sizeof(bufs[0]); ++k) free(bufs[k]);
    free(G);
}

int ref3_set_params(ref3_grid* G, const ref3_params* p) {
    if (!G || !p || !(p->dt > 0) || !(p->tau > 0)) return -1;
    if (G->d.thermal && !(p->tau_g > 0)) return -1;
    G->p = *p;
    G->has_params = 1;
    return 0;
}

/* rho = sum f~, T = sum g~, a = (ax, ay, az + beta g (T - T0)),
 * u = sum c f~ / rho + dt/2 a (Sec. II B 4). */
static void macro3(const ref3_grid* G, const double* fc, const double* gc, double* rho, double* u,
                   double* T, double* acc) {
    const ref3_params* p = &G->p;
    double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0, t = 0.0;
    for (int a = 0; a < Q3; ++a) {
        r += fc[a];
        jx += CX3[a] * fc[a];
        jy += CY3[a] * fc[a];
        jz += CZ3[a] * fc[a];
    }
    acc[0] = p->ax;
    acc[1] = p->ay;
    acc[2] = p->az;
    if (G->d.thermal) {
        for (int a = 0; a < Q3; ++a) t += gc[a];
        acc[2] += p->beta * p->grav * (t - p->T0);
    }
    *rho = r;
    *T = t;
    u[0] = jx / r + 0.5 * p->dt * acc[0];
    u[1] = jy / r + 0.5 * p->dt * acc[1];
    u[2] = jz / r + 0.5 * p->dt * acc[2];
}

static void gather3(const ref3_grid* G, const double* src, int i, int j, int k, double* out) {
    for (int a = 0; a < Q3; ++a) out[a] = src[I3(G, a, i, j, k)];
}

/* f~ = f_eq - dt/2 F and g~ = (T / rho) f_eq (Appendix A). */
int ref3_init_fields(ref3_grid* G, const double* rho, const double* ux, const double* uy,
                     const double* uz, const double* T) {
    if (!G || !G->has_params) return -1;
    const ref3_params* p = &G->p;
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                size_t c = ((size_t)k * G->n[1] + j) * G->n[0] + i;
                double r = rho ? rho[c] : 1.0, t = T ? T[c] : p->T0;
                double vx = ux ? ux[c] : 0.0, vy = uy ? uy[c] : 0.0, vz = uz ? uz[c] : 0.0;
                double az = p->az + (G->d.thermal ? p->beta * p->grav * (t - p->T0) : 0.0);
                double feq[Q3], F[Q3];
                ref3_equilibrium(r, vx, vy, vz, feq);
                ref3_guo_force(r, vx, vy, vz, p->ax, p->ay, az, F);
                for (int a = 0; a < Q3; ++a) {
                    G->f[I3(G, a, i, j, k)] = feq[a] - 0.5 * p->dt * F[a];
                    G->g[I3(G, a, i, j, k)] = G->d.thermal ? (t / r) * feq[a] : 0.0;
                }
            }
    return 0;
}

/* The 3-D workloads' initial fields (Taylor-Green, shear wave, and the Rayleigh-Benard
 * conduction state between the z plates with its seeded perturbation,
 * Sec. IV), set through ref3_init_fields. */
int ref3_init_preset(ref3_grid* G, int kind, double u0, double amp, int mode, unsigned long long seed) {
    if (!G || !G->has_params) return -1;
    if (kind == REF_INIT_RB && !G->d.thermal) return -1;
    const ref3_params* p = &G->p;
    const size_t n = (size_t)G->n[0] * G->n[1] * G->n[2];
    double *rho = zalloc(n), *ux = zalloc(n), *uy = zalloc(n), *uz = zalloc(n), *T = zalloc(n);
    const double PI = 3.14159265358979323846, Lz = G->L[2], dT = p->T_bot - p->T_top;
    /* barometric density of the conductive state along z, normalised so that
     * the volume mean is 1 (Sec. IV) */
    double norm = 1.0;
    if (kind == REF_INIT_RB) {
        double s = 0.0;
        for (int k = 0; k < G->n[2]; ++k) {
            double z = G->c[2][k];
            s += G->w[2][k] * exp(3.0 * p->beta * p->grav * dT * (0.5 * z - 0.5 * z * z / Lz));
        }
        norm = Lz / s;
    }
    int rc = 0;
    for (int k = 0; k < G->n[2] && rc == 0; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                size_t c = ((size_t)k * G->n[1] + j) * G->n[0] + i;
                double x = G->c[0][i], y = G->c[1][j], z = G->c[2][k];
                rho[c] = 1.0;
                T[c] = p->T0;
                if (kind == REF_INIT_TGV) {
                    /* Taylor-Green vortex in a periodic box, pressure from
                     * the incompressible solution, rho = 1 + 3 p' */
                    double kx = 2.0 * PI / G->L[0], ky = 2.0 * PI / G->L[1], kz = 2.0 * PI / G->L[2];
                    ux[c] = u0 * sin(kx * x) * cos(ky * y) * cos(kz * z);
                    uy[c] = -u0 * (kx / ky) * cos(kx * x) * sin(ky * y) * cos(kz * z);
                    rho[c] = 1.0 + 3.0 * (u0 * u0 / 16.0) * (cos(2.0 * kx * x) + cos(2.0 * ky * y)) *
                                       (cos(2.0 * kz * z) + 2.0);
                } else if (kind == REF_INIT_SHEAR) {
                    ux[c] = amp * sin(2.0 * PI * mode * z / Lz);
                } else if (kind == REF_INIT_RB) {
                    double U = ref_splitmix_uniform(seed, (unsigned long long)c);
                    T[c] = p->T0 + dT * (0.5 - z / Lz) + amp * dT * (2.0 * U - 1.0);
                    rho[c] = norm * exp(3.0 * p->beta * p->grav * dT * (0.5 * z - 0.5 * z * z / Lz));
                } else {
                    rc = -1;
                }
            }
    if (rc == 0) rc = ref3_init_fields(G, rho, ux, uy, uz, T);
    free(rho); free(ux); free(uy); free(uz); free(T);
    return rc;
}

int ref3_set_pops(ref3_grid* G, const double* f, const double* gg) {
    if (!G) return -1;
    const size_t N = (size_t)Q3 * G->n[0] * G->n[1] * G->n[2];
    if (f) memcpy(G->f, f, N * sizeof(double));
    if (gg && G->d.thermal) memcpy(G->g, gg, N * sizeof(double));
    return 0;
}

int ref3_get_pops(const ref3_grid* G, double* f, double* gg) {
    if (!G) return -1;
    const size_t N = (size_t)Q3 * G->n[0] * G->n[1] * G->n[2];
    if (f) memcpy(f, G->f, N * sizeof(double));
    if (gg) memcpy(gg, G->g, N * sizeof(double));
    return 0;
}

/* Eq. (ST) with dt = dx = 1: collide, then push to the neighbour; walls use
 * half-way bounce-back (f) and, on the z plates, anti-bounce-back (g). */
int ref3_step_st(ref3_grid* G, int nsteps) {
    if (!G || !G->has_params) return -1;
    const ref3_params* p = &G->p;
    if (fabs(p->dt - 1.0) > 1e-12) return -1;
    if (G->d.sx != REF_UNIFORM || G->d.sy != REF_UNIFORM || G->d.sz != REF_UNIFORM) return -1;
    for (int a = 0; a < 3; ++a)
        if (fabs(G->L[a] - G->n[a]) > 1e-12) return -1; /* unit spacing */
    const int th = G->d.thermal, nx = G->n[0], ny = G->n[1], nz = G->n[2];
    const double taut = p->tau + 0.5, taugt = p->tau_g + 0.5;
    for (int s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double fc[Q3], gc[Q3], feq[Q3], F[Q3], rho, u[3], T, acc[3];
                    gather3(G, G->f, i, j, k, fc);
                    if (th) gather3(G, G->g, i, j, k, gc);
                    macro3(G, fc, gc, &rho, u, &T, acc);
                    ref3_equilibrium(rho, u[0], u[1], u[2], feq);
                    ref3_guo_force(rho, u[0], u[1], u[2], acc[0], acc[1], acc[2], F);
                    for (int a = 0; a < Q3; ++a) {
                        double post = fc[a] + (feq[a] - fc[a]) / taut + (1.0 - 0.5 / taut) * F[a];
                        double gpost = th ? gc[a] + ((T / rho) * feq[a] - gc[a]) / taugt : 0.0;
                        int t[3] = {i + CX3[a], j + CY3[a], k + CZ3[a]};
                        int out = 0;
                        double Twall = 0.0;
                        for (int ax = 0; ax < 3; ++ax) {
                            if (t[ax] >= 0 && t[ax] < G->n[ax]) continue;
                            if (G->bc[ax] == REF_PERIODIC) {
                                t[ax] = (t[ax] + G->n[ax]) % G->n[ax];
                            } else {
                                out = 1;
                                if (ax == 2) Twall = t[2] < 0 ? p->T_bot : p->T_top;
                            }
                        }
                        if (out) {
                            G->fn[I3(G, INV3[a], i, j, k)] = post;
                            if (th) G->gn[I3(G, INV3[a], i, j, k)] = -gpost + 2.0 * W3[a] * Twall;
                        } else {
                            G->fn[I3(G, a, t[0], t[1], t[2])] = post;
                            if (th) G->gn[I3(G, a, t[0], t[1], t[2])] = gpost;
                        }
                    }
                }
        double* t = G->f; G->f = G->fn; G->fn = t;
        t = G->g; G->g = G->gn; G->gn = t;
    }
    return 0;
}

/* h = f~ + dt/(2 tau~)(f_eq - f~) + dt/2 (1 - dt/(2 tau~)) F (the plain
 * population of Appendix A's inversion) and coll = dt/tau~ (f_eq - f~)
 * + dt (1 - dt/(2 tau~)) F; thermal hg, collg with g_eq = (T/rho) f_eq. */
static void fv_eval3(ref3_grid* G, const double* f, const double* gsrc, double* coll, double* collg) {
    const ref3_params* p = &G->p;
    const double dt = p->dt, taut = p->tau + 0.5 * dt, taugt = p->tau_g + 0.5 * dt;
    const int th = G->d.thermal;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                double fc[Q3], gc[Q3], feq[Q3], F[Q3], rho, u[3], T, acc[3];
                gather3(G, f, i, j, k, fc);
                if (th) gather3(G, gsrc, i, j, k, gc);
                macro3(G, fc, gc, &rho, u, &T, acc);
                ref3_equilibrium(rho, u[0], u[1], u[2], feq);
                ref3_guo_force(rho, u[0], u[1], u[2], acc[0], acc[1], acc[2], F);
                for (int a = 0; a < Q3; ++a) {
                    G->h[P3(G, a, i, j, k)] =
                        fc[a] + dt / (2.0 * taut) * (feq[a] - fc[a]) + 0.5 * dt * (1.0 - dt / (2.0 * taut)) * F[a];
                    coll[I3(G, a, i, j, k)] = dt / taut * (feq[a] - fc[a]) + dt * (1.0 - dt / (2.0 * taut)) * F[a];
                    if (th) {
                        double geq = (T / rho) * feq[a];
                        G->hg[P3(G, a, i, j, k)] = gc[a] + dt / (2.0 * taugt) * (geq - gc[a]);
                        collg[I3(G, a, i, j, k)] = dt / taugt * (geq - gc[a]);
                    }
                }
            }
}

/* Two ghost layers per side on every axis, each over the fluid range of the
 * other two axes (the flux stencil never reaches an edge or corner ghost).
 * Periodic axes copy the opposite side; walls reflect, h_a(x_-m) =
 * h_inv(a)(x_m); the z plates anti-reflect hg. */
static void fv_ghosts3(ref3_grid* G) {
    const int th = G->d.thermal;
    const double Tw[2] = {G->p.T_bot, G->p.T_top};
    for (int ax = 0; ax < 3; ++ax) {
        const int n = G->n[ax];
        const int o1 = ax == 0 ? 1 : 0, o2 = ax == 2 ? 1 : 2;  /* the other two axes */
        for (int u = 0; u < G->n[o1]; ++u)
            for (int v = 0; v < G->n[o2]; ++v)
                for (int m = 1; m <= 2; ++m)
                    for (int side = 0; side < 2; ++side) {
                        int ghost = side == 0 ? -m : n - 1 + m;
                        int src;
                        if (G->bc[ax] == REF_PERIODIC) src = side == 0 ? ((-m) % n + n) % n : (n - 1 + m) % n;
                        else src = side == 0 ? m - 1 : n - m;
                        int gi[3], si[3];
                        gi[ax] = ghost;
                        si[ax] = src;
                        gi[o1] = si[o1] = u;
                        gi[o2] = si[o2] = v;
                        for (int a = 0; a < Q3; ++a) {
                            const int b = G->bc[ax] == REF_PERIODIC ? a : INV3[a];
                            G->h[P3(G, a, gi[0], gi[1], gi[2])] = G->h[P3(G, b, si[0], si[1], si[2])];
                            if (th) {
                                double v2 = G->hg[P3(G, b, si[0], si[1], si[2])];
                                if (G->bc[ax] != REF_PERIODIC) v2 = 2.0 * W3[a] * Tw[side] - v2;
                                G->hg[P3(G, a, gi[0], gi[1], gi[2])] = v2;
                            }
                        }
                    }
    }
}

/* QUICK value of population a on face fc of axis ax, on the grid line
 * through (i, j, k): parabola through the two bracketing nodes and the
 * upstream one (Sec. II B 3). */
static double face3(const ref3_grid* G, const double* hp, int a, int ax, int fc, int sgn, int i, int j, int k) {
    int n0 = sgn > 0 ? fc - 2 : fc - 1;
    double pos[3], wts[3], v = 0.0;
    for (int m = 0; m < 3; ++m) pos[m] = G->pos[ax][n0 + m + 2];
    ref_lagrange3(pos, G->xi[ax][fc], wts);
    for (int m = 0; m < 3; ++m) {
        int idx[3] = {i, j, k};
        idx[ax] = n0 + m;
        v += wts[m] * hp[P3(G, a, idx[0], idx[1], idx[2])];
    }
    return v;
}

/* Flux divergence sum over axes of c_a (Phi_+ - Phi_-) / width, Eq. (fv). */
static void fv_advect3(const ref3_grid* G, const double* hp, double* A) {
    const int* cv[3] = {CX3, CY3, CZ3};
#pragma omp parallel for schedule(static)
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                const int cell[3] = {i, j, k};
                for (int a = 0; a < Q3; ++a) {
                    double v = 0.0;
                    for (int ax = 0; ax < 3; ++ax) {
                        int c = cv[ax][a];
                        if (c == 0) continue;
                        int m = cell[ax];
                        v += c * (face3(G, hp, a, ax, m + 1, c, i, j, k) - face3(G, hp, a, ax, m, c, i, j, k)) /
                             G->w[ax][m];
                    }
                    A[I3(G, a, i, j, k)] = v;
                }
            }
}

/* nsteps FV steps: Eq. (semi) as the predictor and the Heun corrector of
 * Eq. (semi-heun) (Sec. II B 2), QUICK faces along each axis line
 * (Sec. II B 3), double-reflection walls (Sec. II B 5). */
int ref3_step_fv(ref3_grid* G, int nsteps) {
    if (!G || !G->has_params || nsteps < 0) return -1;
    const double dt = G->p.dt;
    const int th = G->d.thermal;
    const size_t N = (size_t)Q3 * G->n[0] * G->n[1] * G->n[2];
    for (int s = 0; s < nsteps; ++s) {
        fv_eval3(G, G->f, G->g, G->coll, G->collg);
        fv_ghosts3(G);
        fv_advect3(G, G->h, G->adv);
        if (th) fv_advect3(G, G->hg, G->advg);
        for (size_t q = 0; q < N; ++q) {
            G->fs[q] = G->f[q] - dt * G->adv[q] + G->coll[q];
            if (th) G->gs[q] = G->g[q] - dt * G->advg[q] + G->collg[q];
        }
        fv_eval3(G, G->fs, G->gs, G->fn, G->gn); /* fn, gn: scratch for the unused starred collision */
        fv_ghosts3(G);
        fv_advect3(G, G->h, G->adv2);
        if (th) fv_advect3(G, G->hg, G->advg2);
        for (size_t q = 0; q < N; ++q) {
            G->fn[q] = G->f[q] - 0.5 * dt * (G->adv[q] + G->adv2[q]) + G->coll[q];
            if (th) G->gn[q] = G->g[q] - 0.5 * dt * (G->advg[q] + G->advg2[q]) + G->collg[q];
        }
        double* t = G->f; G->f = G->fn; G->fn = t;
        t = G->g; G->g = G->gn; G->gn = t;
    }
    return 0;
}

/* Cell moments rho, force-corrected u and T (Sec. II B 4, Eq. (LBg)). */
int ref3_moments(const ref3_grid* G, double* rho, double* ux, double* uy, double* uz, double* T) {
    if (!G || !G->has_params) return -1;
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                double fc[Q3], gc[Q3], r, u[3], t, acc[3];
                gather3(G, G->f, i, j, k, fc);
                if (G->d.thermal) gather3(G, G->g, i, j, k, gc);
                macro3(G, fc, gc, &r, u, &t, acc);
                size_t c = ((size_t)k * G->n[1] + j) * G->n[0] + i;
                if (rho) rho[c] = r;
                if (ux) ux[c] = u[0];
                if (uy) uy[c] = u[1];
                if (uz) uz[c] = u[2];
                if (T) T[c] = t;
            }
    return 0;
}

/* Volume integrals sum V rho, sum V rho u (force-corrected u), sum V T. */
int ref3_conservation(const ref3_grid* G, double* mass, double* mx, double* my, double* mz, double* heat) {
    if (!G || !G->has_params) return -1;
    double m = 0.0, px = 0.0, py = 0.0, pz = 0.0, e = 0.0;
    for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                double fc[Q3], gc[Q3], r, u[3], t, acc[3];
                gather3(G, G->f, i, j, k, fc);
                if (G->d.thermal) gather3(G, G->g, i, j, k, gc);
                macro3(G, fc, gc, &r, u, &t, acc);
                double V = G->w[0][i] * G->w[1][j] * G->w[2][k];
                m += V * r;
                px += V * r * u[0];
                py += V * r * u[1];
                pz += V * r * u[2];
                e += V * t;
            }
    if (mass) *mass = m;
    if (mx) *mx = px;
    if (my) *my = py;
    if (mz) *mz = pz;
    if (heat) *heat = e;
    return 0;
}

/* Nu_vol = 1 + H <u_z (T - T0)>_V / (kappa dT); plate values from the
 * second-order one-sided gradient of the plane-averaged T through the
 * plate value and the first two nodes (Sec. IV). */
int ref3_nusselt(const ref3_grid* G, double* nu_vol, double* nu_bot, double* nu_top) {
    if (!G || !G->has_params || !G->d.thermal) return -1;
    const ref3_params* p = &G->p;
    const int nz = G->n[2];
    const double H = G->L[2], dT = p->T_bot - p->T_top, kappa = p->tau_g / 3.0;
    const double area = G->L[0] * G->L[1];
    double s = 0.0, sv = 0.0;
    double* Tm = zalloc(nz);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < G->n[1]; ++j)
            for (int i = 0; i < G->n[0]; ++i) {
                double fc[Q3], gc[Q3], r, u[3], t, acc[3];
                gather3(G, G->f, i, j, k, fc);
                gather3(G, G->g, i, j, k, gc);
                macro3(G, fc, gc, &r, u, &t, acc);
                double A = G->w[0][i] * G->w[1][j], V = A * G->w[2][k];
                s += V * u[2] * (t - p->T0);
                sv += V;
                Tm[k] += A * t / area;
            }
    if (nu_vol) *nu_vol = 1.0 + H * (s / sv) / (kappa * dT);
    if (nz >= 2) {
        double z0 = G->c[2][0], z1 = G->c[2][1];
        double d = -(z0 + z1) / (z0 * z1) * p->T_bot + z1 / (z0 * (z1 - z0)) * Tm[0] -
                   z0 / (z1 * (z1 - z0)) * Tm[1];
        if (nu_bot) *nu_bot = -H * d / dT;
        double s0 = H - G->c[2][nz - 1], s1 = H - G->c[2][nz - 2];
        double e = -(s0 + s1) / (s0 * s1) * p->T_top + s1 / (s0 * (s1 - s0)) * Tm[nz - 1] -
                   s0 / (s1 * (s1 - s0)) * Tm[nz - 2];
        if (nu_top) *nu_top = H * e / dT;
    }
    free(Tm);
    return 0;
}
