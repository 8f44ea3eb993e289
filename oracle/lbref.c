/*
 * lbref.c -- plain FP64 CPU oracle for the lattice Boltzmann time step of
 * Shrestha, Mompean & Calzavarini (arXiv:1505.03271).
 *
 * TEST INFRASTRUCTURE ONLY: the slow, obviously-correct definition against
 * which the CUDA library is checked.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code with the CUDA
 * library and never calls it.
 *
 * Every routine follows the paper's equations in the paper's order, one cell
 * and one population at a time.  OpenMP (if enabled) only splits the outer
 * loop over rows; it never changes the order of any floating-point sum.
 *
 * Readings of points the paper leaves open (each one is listed, with its
 * justification, in the project's design notes):
 *   - The equilibrium is the standard second-order D2Q9 BGK equilibrium the
 *     paper cites from Succi's book (Sec. II, below Eq. (LB)).
 *   - The "tilded equilibrium" in Eqs. (ST), (semi), (semi-heun) is evaluated
 *     as f_eq(rho, u) with the force-corrected velocity u (Sec. II B 4).
 *   - Lagrange quadratic through the three node centres gives the four QUICK
 *     gamma coefficients on any grid (Sec. II B 3).
 *   - The isothermal wall for g (Sec. IV says only "isothermal") extends the
 *     advected field linearly through the wall value:
 *     hg_a(x_-k) = 2 w_a T_wall - hg_inv(a)(x_k), so that the ghost
 *     temperature is 2 T_wall - T(x_k) for the equilibrium and the diffusive
 *     part alike (the FV counterpart of anti-bounce-back).
 *   - Streaming walls use half-way bounce-back (f) and anti-bounce-back (g).
 *
 *   - The FV advected field is the plain population f of Appendix A, which
 *     inverts the tilde transformation as f = f~ + dt/(2 tau + dt)(f~_eq -
 *     f~) + dt/2 F with the tilded equilibrium f~_eq = f_eq - dt/2 F: its
 *     force part is (dt/2)(1 - dt/(2 tau~)) F, so that sum c h = rho u and a
 *     fluid at rest in hydrostatic balance stays at rest.
 * Every routine has a pin in the oracle tests.
 */
#include "lbref.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9

/* D2Q9 lattice (Sec. II; D3Q19 reduces to D2Q9 in two dimensions). */
static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* inv(a): the population moving opposite to c_a (Sec. II B 5). */
static const int INV[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

struct ref_grid {
    ref_desc d;
    ref_params p;
    int has_params;
    int nx, ny;
    double *xi_x, *xi_y;   /* face coordinates, n+1 each                  */
    double *xc, *yc;       /* cell centres y_i = (xi_i + xi_{i+1}) / 2    */
    double *dx, *dy;       /* cell widths                                 */
    double *posx, *posy;   /* centres incl. two ghost/periodic cells each side, index i+2 */
    double *f, *g;         /* state: tilded populations                   */
    double *h, *hg;        /* advected field on the grid padded by two    */
    double *coll, *collg;  /* time-n collision + force terms              */
    double *adv, *advg;    /* time-n advection                            */
    double *adv2, *advg2;  /* starred advection                           */
    double *fs, *gs;       /* starred (predictor) state                   */
    double *fn, *gn;       /* next state                                  */
    double *scr, *scrg;    /* collision of the starred state (unused)     */
    int scheme;            /* REF_FV_HEUN / REF_FV_SEMI / REF_FV_EULER     */
    double rho_bc[4];      /* imposed densities: x0, x1, y0, y1             */
};

/* ------------------------------------------------------------------ */
/* building blocks                                                     */
/* ------------------------------------------------------------------ */

/* The D2Q9 velocities, weights and opposite-velocity map (Sec. II). */
void ref_lattice(int* cx, int* cy, double* w, int* inv) {
    for (int a = 0; a < Q; ++a) {
        if (cx) cx[a] = CX[a];
        if (cy) cy[a] = CY[a];
        if (w) w[a] = W[a];
        if (inv) inv[a] = INV[a];
    }
}

/* Face coordinates xi_0..xi_n of one axis, Eq. (grids) of Sec. III B.
 * tanh: xi_i = L/2 (1 + tanh[(2i/n - 1) delta] / tanh(delta)), which is the
 * paper's formula with s1 = tanh(delta); "stretch" is delta.
 * sinh: the paper's two branches with s2 = stretch (n even).
 * Chebyshev: xi_i = L/2 (1 - cos(i pi / n)).  The paper's formula, with
 * (i - 1/2) in place of i, puts neither xi_0 nor xi_n on a wall; these are
 * the Chebyshev-Gauss-Lobatto points, which do. */
void ref_faces(int n, double L, int spacing, double stretch, double* xi) {
    for (int i = 0; i <= n; ++i) {
        double v;
        if (spacing == REF_TANH) {
            v = 0.5 * L * (1.0 + tanh((2.0 * i / n - 1.0) * stretch) / tanh(stretch));
        } else if (spacing == REF_SINH) {
            double A = 0.5 * L / sinh(0.5 * stretch);
            if (2 * i <= n)
                v = A * sinh(stretch * i / n);
            else
                v = L - A * sinh(stretch * (double)(n - i) / n);
        } else if (spacing == REF_CHEB) {
            v = 0.5 * L * (1.0 - cos(3.14159265358979323846 * i / n));
        } else {
            v = L * i / n;
        }
        xi[i] = v;
    }
    xi[0] = 0.0;
    xi[n] = L;
}

/* Lagrange weights of the parabola through pos[0..2], evaluated at x: the
 * QUICK gamma coefficients of Sec. II B 3 on any node spacing. */
void ref_lagrange3(const double* pos, double x, double* wts) {
    for (int k = 0; k < 3; ++k) {
        double num = 1.0, den = 1.0;
        for (int m = 0; m < 3; ++m) {
            if (m == k) continue;
            num *= (x - pos[m]);
            den *= (pos[k] - pos[m]);
        }
        wts[k] = num / den;
    }
}

/* Second-order BGK equilibrium (Sec. II, cited to Succi's book). */
void ref_equilibrium(double rho, double ux, double uy, double* feq) {
    double uu = ux * ux + uy * uy;
    for (int a = 0; a < Q; ++a) {
        double cu = CX[a] * ux + CY[a] * uy;
        feq[a] = W[a] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* Guo force term, Eq. (F2): w [ (c-u)/cs^2 + (c.u) c / cs^4 ] . rho a. */
void ref_guo_force(double rho, double ux, double uy, double ax, double ay, double* F) {
    for (int a = 0; a < Q; ++a) {
        double cu = CX[a] * ux + CY[a] * uy;
        double ex = 3.0 * (CX[a] - ux) + 9.0 * cu * CX[a];
        double ey = 3.0 * (CY[a] - uy) + 9.0 * cu * CY[a];
        F[a] = W[a] * rho * (ex * ax + ey * ay);
    }
}

/* SplitMix64 (Steele, Lea & Flood 2014) used as a counter-based generator:
 * one step from state (seed ^ counter), top 53 bits mapped to [0,1). */
double ref_splitmix_uniform(unsigned long long seed, unsigned long long counter) {
    unsigned long long z = (seed ^ counter) + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------ */
/* grid                                                                */
/* ------------------------------------------------------------------ */

static int g_threads = 1;

void ref_set_threads(int n) {
    g_threads = n < 1 ? 1 : n;
#ifdef _OPENMP
    omp_set_num_threads(g_threads);
#endif
}

int ref_get_threads(void) {
#ifdef _OPENMP
    return g_threads;
#else
    return 1;
#endif
}

static double* alloc0(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

/* Centre of cell i on an axis, for any integer i: periodic axes repeat the
 * cells shifted by L, wall axes mirror the first two cells at the wall
 * (ghost centres of Sec. II B 5). */
static double axis_pos(const double* c, const double* xi, int n, double L, int bc, int i) {
    if (i >= 0 && i < n) return c[i];
    if (bc == REF_PERIODIC) {
        int q = (i >= 0) ? i / n : -((-i + n - 1) / n);
        int r = i - q * n;
        return c[r] + q * L;
    }
    if (i < 0) return 2.0 * xi[0] - c[-i - 1];
    return 2.0 * xi[n] - c[2 * n - 1 - i];
}

static void build_axis(int n, double L, int sp, double st, int bc, double** xi, double** c,
                       double** d, double** pos) {
    *xi = alloc0(n + 1);
    *c = alloc0(n);
    *d = alloc0(n);
    *pos = alloc0(n + 4);
    ref_faces(n, L, sp, st, *xi);
    for (int i = 0; i < n; ++i) {
        (*c)[i] = 0.5 * ((*xi)[i] + (*xi)[i + 1]);
        (*d)[i] = (*xi)[i + 1] - (*xi)[i];
    }
    for (int i = -2; i < n + 2; ++i) (*pos)[i + 2] = axis_pos(*c, *xi, n, L, bc, i);
}

ref_grid* ref_create(const ref_desc* d) {
    if (!d || d->nx < 1 || d->ny < 1) return NULL;
    if (d->bcx != REF_PERIODIC && d->nx < 2) return NULL;
    if (d->bcy != REF_PERIODIC && d->ny < 2) return NULL;
    if (d->bcx < REF_PERIODIC || d->bcx > REF_DENSITY || d->bcy < REF_PERIODIC || d->bcy > REF_DENSITY) return NULL;
    if (d->thermal && d->bcx != REF_PERIODIC) return NULL; /* isothermal walls are on y only */
    if (d->thermal && d->bcy == REF_DENSITY) return NULL;
    if (d->sx == REF_SINH && (d->nx % 2)) return NULL;
    if (d->sy == REF_SINH && (d->ny % 2)) return NULL;
    ref_grid* G = (ref_grid*)calloc(1, sizeof(ref_grid));
    G->d = *d;
    for (int k = 0; k < 4; ++k) G->rho_bc[k] = 1.0;
    G->nx = d->nx;
    G->ny = d->ny;
    build_axis(d->nx, d->lx, d->sx, d->stretch_x, d->bcx, &G->xi_x, &G->xc, &G->dx, &G->posx);
    build_axis(d->ny, d->ly, d->sy, d->stretch_y, d->bcy, &G->xi_y, &G->yc, &G->dy, &G->posy);
    size_t N = (size_t)G->nx * G->ny * Q;
    size_t NP = (size_t)(G->nx + 4) * (G->ny + 4) * Q;
    G->f = alloc0(N); G->g = alloc0(N);
    G->h = alloc0(NP); G->hg = alloc0(NP);
    G->coll = alloc0(N); G->collg = alloc0(N);
    G->adv = alloc0(N); G->advg = alloc0(N);
    G->adv2 = alloc0(N); G->advg2 = alloc0(N);
    G->fs = alloc0(N); G->gs = alloc0(N);
    G->fn = alloc0(N); G->gn = alloc0(N);
    G->scr = alloc0(N); G->scrg = alloc0(N);
    return G;
}

void ref_destroy(ref_grid* G) {
    if (!G) return;
    double* bufs[] = {G->xi_x, G->xi_y, G->xc, G->yc, G->dx, G->dy, G->posx, G->posy,
                      G->f, G->g, G->h, G->hg, G->coll, G->collg, G->adv, G->advg,
                      G->adv2, G->advg2, G->fs, G->gs, G->fn, G->gn, G->scr, G->scrg};
    for (size_t k = 0; k < sizeof(bufs) / sizeof(bufs[0]); ++k) free(bufs[k]);
    free(G);
}

int ref_set_params(ref_grid* G, const ref_params* p) {
    if (!G || !p || !(p->dt > 0) || !(p->tau > 0)) return -1;
    if (G->d.thermal && !(p->tau_g > 0)) return -1;
    G->p = *p;
    G->has_params = 1;
    return 0;
}

void ref_centers(const ref_grid* G, double* xc, double* yc) {
    if (xc) memcpy(xc, G->xc, sizeof(double) * G->nx);
    if (yc) memcpy(yc, G->yc, sizeof(double) * G->ny);
}

void ref_face_coords(const ref_grid* G, double* a, double* b) {
    if (a) memcpy(a, G->xi_x, sizeof(double) * (G->nx + 1));
    if (b) memcpy(b, G->xi_y, sizeof(double) * (G->ny + 1));
}

#define IDX(G, a, i, j) (((size_t)(a) * (G)->ny + (j)) * (G)->nx + (i))
#define PIDX(G, a, i, j) (((size_t)(a) * ((G)->ny + 4) + (j) + 2) * ((G)->nx + 4) + (i) + 2)

/* Macroscopic fields of one cell from its tilded populations:
 * rho = sum f~, T = sum g~, a = a_ext + beta g (T - T0) y^ (Boussinesq,
 * Sec. IV), u = sum c f~ / rho + dt/2 a (Sec. II B 4). */
static void macro(const ref_grid* G, const double* fc, const double* gc, double* rho, double* ux,
                  double* uy, double* T, double* ax, double* ay) {
    const ref_params* p = &G->p;
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < Q; ++a) {
        r += fc[a];
        jx += CX[a] * fc[a];
        jy += CY[a] * fc[a];
    }
    double t = 0.0;
    double fx = p->ax, fy = p->ay;
    if (G->d.thermal) {
        for (int a = 0; a < Q; ++a) t += gc[a];
        fy += p->beta * p->grav * (t - p->T0);
    }
    *rho = r;
    *T = t;
    *ax = fx;
    *ay = fy;
    /* the plain populations of the Euler scheme carry the momentum itself */
    const double shift = G->scheme == REF_FV_EULER ? 0.0 : 0.5 * p->dt;
    *ux = jx / r + shift * fx;
    *uy = jy / r + shift * fy;
}

static void gather(const ref_grid* G, const double* src, int i, int j, double* out) {
    for (int a = 0; a < Q; ++a) out[a] = src[IDX(G, a, i, j)];
}

/* ------------------------------------------------------------------ */
/* initialisation                                                      */
/* ------------------------------------------------------------------ */

/* f~ = f_eq(rho,u) - dt/2 F(rho,u,a) and g~ = g_eq = (T/rho) f_eq, the
 * equilibrium expressed in tilded variables (Appendix A). */
int ref_init_fields(ref_grid* G, const double* rho, const double* ux, const double* uy,
                    const double* T) {
    if (!G || !G->has_params) return -1;
    const ref_params* p = &G->p;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < G->ny; ++j)
        for (int i = 0; i < G->nx; ++i) {
            size_t c = (size_t)j * G->nx + i;
            double r = rho ? rho[c] : 1.0;
            double vx = ux ? ux[c] : 0.0, vy = uy ? uy[c] : 0.0;
            double t = T ? T[c] : p->T0;
            double fx = p->ax, fy = p->ay;
            if (G->d.thermal) fy += p->beta * p->grav * (t - p->T0);
            double feq[Q], F[Q];
            ref_equilibrium(r, vx, vy, feq);
            ref_guo_force(r, vx, vy, fx, fy, F);
            const double shift = G->scheme == REF_FV_EULER ? 0.0 : 0.5 * p->dt;
            for (int a = 0; a < Q; ++a) {
                G->f[IDX(G, a, i, j)] = feq[a] - shift * F[a];
                G->g[IDX(G, a, i, j)] = G->d.thermal ? (t / r) * feq[a] : 0.0;
            }
        }
    return 0;
}

/* The workloads' initial fields (Taylor-Green, shear wave, the Poiseuille
 * parabola of Sec. III B, and the Rayleigh-Benard conduction state with its
 * seeded perturbation, Sec. IV), set through ref_init_fields. */
int ref_init_preset(ref_grid* G, int kind, double u0, double amp, int mode,
                    unsigned long long seed) {
    if (!G || !G->has_params) return -1;
    const ref_params* p = &G->p;
    int nx = G->nx, ny = G->ny;
    double Lx = G->d.lx, Ly = G->d.ly;
    size_t n = (size_t)nx * ny;
    double* rho = alloc0(n);
    double* ux = alloc0(n);
    double* uy = alloc0(n);
    double* T = alloc0(n);
    const double PI = 3.14159265358979323846;
    int rc = 0;
    if (kind == REF_INIT_RB && !G->d.thermal) rc = -1;
    if (kind != REF_INIT_TGV && kind != REF_INIT_SHEAR && kind != REF_INIT_POISEUILLE && kind != REF_INIT_RB)
        rc = -1;
    /* barometric density of the conductive state (Sec. IV): c_s^2 d(rho)/dy =
     * rho * beta g (T_c - T0), normalised so that sum V rho = sum V. */
    double dT = p->T_bot - p->T_top;
    double norm = 1.0;
    if (kind == REF_INIT_RB && rc == 0) {
        double s = 0.0;
        for (int j = 0; j < ny; ++j) {
            double y = G->yc[j];
            s += G->dy[j] * exp(3.0 * p->beta * p->grav * dT * (0.5 * y - 0.5 * y * y / Ly));
        }
        norm = Ly / s;
    }
    const int rows = rc == 0 ? ny : 0; /* nothing to fill for a rejected kind */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < rows; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = (size_t)j * nx + i;
            double x = G->xc[i], y = G->yc[j];
            rho[c] = 1.0;
            T[c] = p->T0;
            if (kind == REF_INIT_TGV) {
                double kx = 2.0 * PI / Lx, ky = 2.0 * PI / Ly, r = kx / ky;
                ux[c] = -u0 * cos(kx * x) * sin(ky * y);
                uy[c] = u0 * r * sin(kx * x) * cos(ky * y);
                rho[c] = 1.0 - 3.0 * (u0 * u0 / 4.0) * (cos(2.0 * kx * x) + r * r * cos(2.0 * ky * y));
                if (amp != 0.0) ux[c] += amp * sin(2.0 * PI * mode * y / Ly);
            } else if (kind == REF_INIT_SHEAR) {
                ux[c] = amp * sin(2.0 * PI * mode * y / Ly);
            } else if (kind == REF_INIT_POISEUILLE) {
                ux[c] = 4.0 * u0 * y * (Ly - y) / (Ly * Ly);
            } else if (kind == REF_INIT_RB) {
                double U = ref_splitmix_uniform(seed, (unsigned long long)c);
                T[c] = p->T0 + dT * (0.5 - y / Ly) + amp * dT * (2.0 * U - 1.0);
                rho[c] = norm * exp(3.0 * p->beta * p->grav * dT * (0.5 * y - 0.5 * y * y / Ly));
            }
        }
    if (rc == 0) rc = ref_init_fields(G, rho, ux, uy, T);
    free(rho); free(ux); free(uy); free(T);
    return rc;
}

int ref_set_pops(ref_grid* G, const double* f, const double* gg) {
    size_t N = (size_t)G->nx * G->ny * Q;
    if (f) memcpy(G->f, f, N * sizeof(double));
    if (gg && G->d.thermal) memcpy(G->g, gg, N * sizeof(double));
    return 0;
}

int ref_get_pops(const ref_grid* G, double* f, double* gg) {
    size_t N = (size_t)G->nx * G->ny * Q;
    if (f) memcpy(f, G->f, N * sizeof(double));
    if (gg) memcpy(gg, G->g, N * sizeof(double));
    return 0;
}

/* ------------------------------------------------------------------ */
/* streaming (ST) step, Eq. (ST) with dt = dx = 1                      */
/* ------------------------------------------------------------------ */

static int axis_uniform_unit(int sp, int n, double L) {
    return sp == REF_UNIFORM && fabs(L / n - 1.0) < 1e-12;
}

/* nsteps ST steps, Eq. (ST) with dt = dx = 1 (Sec. II A): collide each
 * cell and push each population to its neighbour; walls use half-way
 * bounce-back (f) and anti-bounce-back through T_wall (g). */
int ref_step_st(ref_grid* G, int nsteps) {
    if (!G || !G->has_params || nsteps < 0) return -1;
    const ref_params* p = &G->p;
    if (fabs(p->dt - 1.0) > 1e-12) return -1;
    if (G->scheme == REF_FV_EULER) return -1;
    if (G->d.bcx == REF_DENSITY || G->d.bcy == REF_DENSITY) return -1; /* FV boundary only */
    if (!axis_uniform_unit(G->d.sx, G->nx, G->d.lx) || !axis_uniform_unit(G->d.sy, G->ny, G->d.ly))
        return -1;
    const int nx = G->nx, ny = G->ny, th = G->d.thermal;
    const double taut = p->tau + 0.5;       /* tau~ = tau + dt/2 */
    const double taugt = p->tau_g + 0.5;
    for (int s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double fc[Q], gc[Q], feq[Q], F[Q];
                double rho, ux, uy, T, ax, ay;
                gather(G, G->f, i, j, fc);
                if (th) gather(G, G->g, i, j, gc);
                macro(G, fc, gc, &rho, &ux, &uy, &T, &ax, &ay);
                ref_equilibrium(rho, ux, uy, feq);
                ref_guo_force(rho, ux, uy, ax, ay, F);
                for (int a = 0; a < Q; ++a) {
                    /* right-hand side of Eq. (ST) */
                    double post = fc[a] + (feq[a] - fc[a]) / taut + (1.0 - 0.5 / taut) * F[a];
                    double gpost = 0.0;
                    if (th) gpost = gc[a] + ((T / rho) * feq[a] - gc[a]) / taugt;
                    int ti = i + CX[a], tj = j + CY[a];
                    int out = 0;
                    double Twall = 0.0;
                    if (ti < 0 || ti >= nx) {
                        if (G->d.bcx == REF_PERIODIC) ti = (ti + nx) % nx;
                        else out = 1;
                    }
                    if (tj < 0 || tj >= ny) {
                        if (G->d.bcy == REF_PERIODIC) tj = (tj + ny) % ny;
                        else { out = 1; Twall = (tj < 0) ? p->T_bot : p->T_top; }
                    }
                    if (out) {
                        /* half-way bounce-back: the population returns to
                         * its cell reversed; g uses anti-bounce-back for a
                         * fixed wall temperature. */
                        G->fn[IDX(G, INV[a], i, j)] = post;
                        if (th) G->gn[IDX(G, INV[a], i, j)] = -gpost + 2.0 * W[a] * Twall;
                    } else {
                        G->fn[IDX(G, a, ti, tj)] = post;
                        if (th) G->gn[IDX(G, a, ti, tj)] = gpost;
                    }
                }
            }
        double* t = G->f; G->f = G->fn; G->fn = t;
        t = G->g; G->g = G->gn; G->gn = t;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* finite-volume (FV) step: semi-implicit collision + Heun advection,  */
/* Eqs. (semi) and (semi-heun), QUICK faces, double-reflection walls   */
/* ------------------------------------------------------------------ */

/* For every fluid cell: the advected field
 *   h = f~ + dt/(2 tau~) (f_eq - f~) + dt/2 (1 - dt/(2 tau~)) F
 * (the bracket of Eq. (semi), i.e. the plain population of Appendix A's
 * inversion with f~_eq = f_eq - dt/2 F)
 * and the collision + force term
 *   coll = dt/tau~ (f_eq - f~) + dt (1 - dt/(2 tau~)) F.
 * Thermal: hg = g~ + dt/(2 tau~_g)(g_eq - g~), collg = dt/tau~_g (g_eq - g~),
 * g_eq = (T/rho) f_eq (Eq. (LBg)). */
static void fv_eval(ref_grid* G, const double* f, const double* gsrc, double* coll,
                    double* collg) {
    const ref_params* p = &G->p;
    const double dt = p->dt, taut = p->tau + 0.5 * dt, taugt = p->tau_g + 0.5 * dt;
    const int th = G->d.thermal;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < G->ny; ++j)
        for (int i = 0; i < G->nx; ++i) {
            double fc[Q], gc[Q], feq[Q], F[Q];
            double rho, ux, uy, T, ax, ay;
            gather(G, f, i, j, fc);
            if (th) gather(G, gsrc, i, j, gc);
            macro(G, fc, gc, &rho, &ux, &uy, &T, &ax, &ay);
            ref_equilibrium(rho, ux, uy, feq);
            ref_guo_force(rho, ux, uy, ax, ay, F);
            for (int a = 0; a < Q; ++a) {
                G->h[PIDX(G, a, i, j)] =
                    fc[a] + dt / (2.0 * taut) * (feq[a] - fc[a]) + 0.5 * dt * (1.0 - dt / (2.0 * taut)) * F[a];
                coll[IDX(G, a, i, j)] =
                    dt / taut * (feq[a] - fc[a]) + dt * (1.0 - dt / (2.0 * taut)) * F[a];
                if (th) {
                    double geq = (T / rho) * feq[a];
                    G->hg[PIDX(G, a, i, j)] = gc[a] + dt / (2.0 * taugt) * (geq - gc[a]);
                    collg[IDX(G, a, i, j)] = dt / taugt * (geq - gc[a]);
                }
            }
        }
}

/* Explicit Euler, Eq. (euler): the advected field is the population
 * itself, h = f and hg = g, and the source is
 *   coll = dt/tau (f_eq - f) + dt F,   collg = dt/tau_g (g_eq - g)
 * with the physical relaxation times and the moments of the plain
 * populations. */
static void fv_eval_euler(ref_grid* G, const double* f, const double* gsrc, double* coll,
                          double* collg) {
    const ref_params* p = &G->p;
    const double dt = p->dt;
    const int th = G->d.thermal;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < G->ny; ++j)
        for (int i = 0; i < G->nx; ++i) {
            double fc[Q], gc[Q], feq[Q], F[Q];
            double rho, ux, uy, T, ax, ay;
            gather(G, f, i, j, fc);
            if (th) gather(G, gsrc, i, j, gc);
            macro(G, fc, gc, &rho, &ux, &uy, &T, &ax, &ay);
            ref_equilibrium(rho, ux, uy, feq);
            ref_guo_force(rho, ux, uy, ax, ay, F);
            for (int a = 0; a < Q; ++a) {
                G->h[PIDX(G, a, i, j)] = fc[a];
                coll[IDX(G, a, i, j)] = dt / p->tau * (feq[a] - fc[a]) + dt * F[a];
                if (th) {
                    G->hg[PIDX(G, a, i, j)] = gc[a];
                    collg[IDX(G, a, i, j)] = dt / p->tau_g * ((T / rho) * feq[a] - gc[a]);
                }
            }
        }
}

/* Fixed-density ghost (Sec. II B 5): the density at the ghost centre is
 * extrapolated linearly through the imposed face value rho_S from the fluid
 * node it mirrors, rho_g = 2 rho_S - rho_k, and the ghost takes that node's
 * populations rescaled, h_a(ghost) = (rho_g / rho_k) h_a(node). */
static void density_ghost(ref_grid* G, int i, int j, int gi, int gj, double rho_s) {
    double rk = 0.0;
    for (int a = 0; a < Q; ++a) rk += G->h[PIDX(G, a, i, j)];
    const double s = (2.0 * rho_s - rk) / rk;
    for (int a = 0; a < Q; ++a) G->h[PIDX(G, a, gi, gj)] = s * G->h[PIDX(G, a, i, j)];
}

/* Ghost cells of the padded advected fields (two per side, Sec. II B 5).
 * Periodic axes copy the opposite side.  Wall axes apply the double
 * reflection h_a(x_-k) = h_inv(a)(x_k); the thermal field is anti-reflected,
 * hg_a(x_-k) = 2 w_a T_wall - hg_inv(a)(x_k). */
static void fv_ghosts(ref_grid* G) {
    const int nx = G->nx, ny = G->ny, th = G->d.thermal;
    for (int j = 0; j < ny; ++j)
        for (int k = 1; k <= 2; ++k)
            for (int a = 0; a < Q; ++a) {
                if (G->d.bcx == REF_PERIODIC) {
                    int il = ((-k) % nx + nx) % nx, ir = (nx - 1 + k) % nx;
                    G->h[PIDX(G, a, -k, j)] = G->h[PIDX(G, a, il, j)];
                    G->h[PIDX(G, a, nx - 1 + k, j)] = G->h[PIDX(G, a, ir, j)];
                    if (th) {
                        G->hg[PIDX(G, a, -k, j)] = G->hg[PIDX(G, a, il, j)];
                        G->hg[PIDX(G, a, nx - 1 + k, j)] = G->hg[PIDX(G, a, ir, j)];
                    }
                } else if (G->d.bcx == REF_WALLS) {
                    G->h[PIDX(G, a, -k, j)] = G->h[PIDX(G, INV[a], k - 1, j)];
                    G->h[PIDX(G, a, nx - 1 + k, j)] = G->h[PIDX(G, INV[a], nx - k, j)];
                }
            }
    if (G->d.bcx == REF_DENSITY)
        for (int j = 0; j < ny; ++j)
            for (int k = 1; k <= 2; ++k) {
                density_ghost(G, k - 1, j, -k, j, G->rho_bc[0]);
                density_ghost(G, nx - k, j, nx - 1 + k, j, G->rho_bc[1]);
            }
    for (int i = 0; i < nx; ++i)
        for (int k = 1; k <= 2; ++k) {
            if (G->d.bcy == REF_PERIODIC) {
                int jl = ((-k) % ny + ny) % ny, jr = (ny - 1 + k) % ny;
                for (int a = 0; a < Q; ++a) {
                    G->h[PIDX(G, a, i, -k)] = G->h[PIDX(G, a, i, jl)];
                    G->h[PIDX(G, a, i, ny - 1 + k)] = G->h[PIDX(G, a, i, jr)];
                    if (th) {
                        G->hg[PIDX(G, a, i, -k)] = G->hg[PIDX(G, a, i, jl)];
                        G->hg[PIDX(G, a, i, ny - 1 + k)] = G->hg[PIDX(G, a, i, jr)];
                    }
                }
            } else if (G->d.bcy == REF_DENSITY) {
                density_ghost(G, i, k - 1, i, -k, G->rho_bc[2]);
                density_ghost(G, i, ny - k, i, ny - 1 + k, G->rho_bc[3]);
            } else {
                int jb = k - 1, jt = ny - k;
                for (int a = 0; a < Q; ++a) {
                    G->h[PIDX(G, a, i, -k)] = G->h[PIDX(G, INV[a], i, jb)];
                    G->h[PIDX(G, a, i, ny - 1 + k)] = G->h[PIDX(G, INV[a], i, jt)];
                    if (th) {
                        G->hg[PIDX(G, a, i, -k)] = 2.0 * W[a] * G->p.T_bot - G->hg[PIDX(G, INV[a], i, jb)];
                        G->hg[PIDX(G, a, i, ny - 1 + k)] = 2.0 * W[a] * G->p.T_top - G->hg[PIDX(G, INV[a], i, jt)];
                    }
                }
            }
        }
}

/* QUICK value of one population on the x face xi_x[fc] (between cells fc-1
 * and fc of row j): parabola through the two bracketing nodes and the
 * upstream one, chosen by the sign of c_x (Sec. II B 3). */
static double face_x(const ref_grid* G, const double* hp, int a, int j, int fc, int sgn) {
    int n0 = (sgn > 0) ? fc - 2 : fc - 1;
    double pos[3], w[3];
    for (int k = 0; k < 3; ++k) pos[k] = G->posx[n0 + k + 2];
    ref_lagrange3(pos, G->xi_x[fc], w);
    double v = 0.0;
    for (int k = 0; k < 3; ++k) v += w[k] * hp[PIDX(G, a, n0 + k, j)];
    return v;
}

static double face_y(const ref_grid* G, const double* hp, int a, int i, int fc, int sgn) {
    int n0 = (sgn > 0) ? fc - 2 : fc - 1;
    double pos[3], w[3];
    for (int k = 0; k < 3; ++k) pos[k] = G->posy[n0 + k + 2];
    ref_lagrange3(pos, G->xi_y[fc], w);
    double v = 0.0;
    for (int k = 0; k < 3; ++k) v += w[k] * hp[PIDX(G, a, i, n0 + k)];
    return v;
}

/* Flux divergence (S_j/V) c.n_j [h]_j of Eq. (fv) on the Cartesian cell:
 * c_x (Phi_e - Phi_w)/dx_i + c_y (Phi_n - Phi_s)/dy_j. */
static void fv_advect(const ref_grid* G, const double* hp, double* A) {
#pragma omp parallel for schedule(static)
    for (int j = 0; j < G->ny; ++j)
        for (int i = 0; i < G->nx; ++i)
            for (int a = 0; a < Q; ++a) {
                double v = 0.0;
                if (CX[a] != 0)
                    v += CX[a] * (face_x(G, hp, a, j, i + 1, CX[a]) - face_x(G, hp, a, j, i, CX[a])) /
                         G->dx[i];
                if (CY[a] != 0)
                    v += CY[a] * (face_y(G, hp, a, i, j + 1, CY[a]) - face_y(G, hp, a, i, j, CY[a])) /
                         G->dy[j];
                A[IDX(G, a, i, j)] = v;
            }
}

int ref_set_boundary_density(ref_grid* G, double rho_x0, double rho_x1, double rho_y0, double rho_y1) {
    if (!G || !(rho_x0 > 0) || !(rho_x1 > 0) || !(rho_y0 > 0) || !(rho_y1 > 0)) return -1;
    G->rho_bc[0] = rho_x0;
    G->rho_bc[1] = rho_x1;
    G->rho_bc[2] = rho_y0;
    G->rho_bc[3] = rho_y1;
    return 0;
}

int ref_set_scheme(ref_grid* G, int scheme) {
    if (!G || scheme < REF_FV_HEUN || scheme > REF_FV_EULER) return -1;
    G->scheme = scheme;
    return 0;
}

/* nsteps FV steps (Sec. II B 2): Eq. (semi) as the predictor, and the Heun
 * corrector of Eq. (semi-heun) for the default scheme; the single-stage
 * schemes stop after the first update (Eq. (semi) alone, or Eq. (euler) on
 * plain populations). */
int ref_step_fv(ref_grid* G, int nsteps) {
    if (!G || !G->has_params || nsteps < 0) return -1;
    const double dt = G->p.dt;
    const int th = G->d.thermal;
    const size_t N = (size_t)G->nx * G->ny * Q;
    for (int s = 0; s < nsteps; ++s) {
        /* time level n: h^n, Coll^n, A^n */
        if (G->scheme == REF_FV_EULER)
            fv_eval_euler(G, G->f, G->g, G->coll, G->collg);
        else
            fv_eval(G, G->f, G->g, G->coll, G->collg);
        fv_ghosts(G);
        fv_advect(G, G->h, G->adv);
        if (th) fv_advect(G, G->hg, G->advg);
        /* predictor f~* of Eq. (semi); for Eq. (euler) the same update of
         * the plain populations.  Both single-stage schemes end here. */
        for (size_t k = 0; k < N; ++k) {
            G->fs[k] = G->f[k] - dt * G->adv[k] + G->coll[k];
            if (th) G->gs[k] = G->g[k] - dt * G->advg[k] + G->collg[k];
        }
        if (G->scheme != REF_FV_HEUN) {
            double* t = G->f; G->f = G->fs; G->fs = t;
            t = G->g; G->g = G->gs; G->gs = t;
            continue;
        }
        /* starred advected field h*, with its own moments and force */
        fv_eval(G, G->fs, G->gs, G->scr, G->scrg);
        fv_ghosts(G);
        fv_advect(G, G->h, G->adv2);
        if (th) fv_advect(G, G->hg, G->advg2);
        /* corrector, Eq. (semi-heun): trapezoidal advection, time-n collision */
        for (size_t k = 0; k < N; ++k) {
            G->fn[k] = G->f[k] - 0.5 * dt * (G->adv[k] + G->adv2[k]) + G->coll[k];
            if (th) G->gn[k] = G->g[k] - 0.5 * dt * (G->advg[k] + G->advg2[k]) + G->collg[k];
        }
        double* t = G->f; G->f = G->fn; G->fn = t;
        t = G->g; G->g = G->gn; G->gn = t;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* observables                                                         */
/* ------------------------------------------------------------------ */

/* Cell moments rho, force-corrected u and T (Sec. II B 4, Eq. (LBg)). */
int ref_moments(const ref_grid* G, double* rho, double* ux, double* uy, double* T) {
    if (!G || !G->has_params) return -1;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < G->ny; ++j)
        for (int i = 0; i < G->nx; ++i) {
            double fc[Q], gc[Q];
            double r, vx, vy, t, ax, ay;
            gather(G, G->f, i, j, fc);
            if (G->d.thermal) gather(G, G->g, i, j, gc);
            macro(G, fc, gc, &r, &vx, &vy, &t, &ax, &ay);
            size_t c = (size_t)j * G->nx + i;
            if (rho) rho[c] = r;
            if (ux) ux[c] = vx;
            if (uy) uy[c] = vy;
            if (T) T[c] = t;
        }
    return 0;
}

/* Volume integrals sum V rho, sum V rho u (force-corrected u), sum V T. */
int ref_conservation(const ref_grid* G, double* mass, double* momx, double* momy, double* heat) {
    if (!G || !G->has_params) return -1;
    double m = 0.0, px = 0.0, py = 0.0, e = 0.0;
    for (int j = 0; j < G->ny; ++j)
        for (int i = 0; i < G->nx; ++i) {
            double fc[Q], gc[Q];
            double r, vx, vy, t, ax, ay;
            gather(G, G->f, i, j, fc);
            if (G->d.thermal) gather(G, G->g, i, j, gc);
            macro(G, fc, gc, &r, &vx, &vy, &t, &ax, &ay);
            double V = G->dx[i] * G->dy[j];
            m += V * r;
            px += V * r * vx;
            py += V * r * vy;
            e += V * t;
        }
    if (mass) *mass = m;
    if (momx) *momx = px;
    if (momy) *momy = py;
    if (heat) *heat = e;
    return 0;
}

/* Nusselt numbers.  Volume: Nu = 1 + H <u_y (T - T0)>_V / (kappa dT), with
 * kappa = tau_g c_s^2 (Sec. IV).  Walls: second-order one-sided gradient of
 * the x-averaged T through the wall value and the first two nodes
 * (Sec. IV, post-processing of Nu(z)). */
int ref_nusselt(const ref_grid* G, double* nu_vol, double* nu_bot, double* nu_top) {
    if (!G || !G->has_params || !G->d.thermal) return -1;
    const ref_params* p = &G->p;
    const int nx = G->nx, ny = G->ny;
    const double H = G->d.ly, dT = p->T_bot - p->T_top, kappa = p->tau_g / 3.0;
    double sv = 0.0, s = 0.0;
    double* Tm = alloc0(ny);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double fc[Q], gc[Q];
            double r, vx, vy, t, ax, ay;
            gather(G, G->f, i, j, fc);
            gather(G, G->g, i, j, gc);
            macro(G, fc, gc, &r, &vx, &vy, &t, &ax, &ay);
            double V = G->dx[i] * G->dy[j];
            s += V * vy * (t - p->T0);
            sv += V;
            Tm[j] += G->dx[i] * t / G->d.lx;
        }
    if (nu_vol) *nu_vol = 1.0 + H * (s / sv) / (kappa * dT);
    if (ny >= 2) {
        /* quadratic through (0, T_bot), (y0, Tm0), (y1, Tm1), slope at 0 */
        double y0 = G->yc[0], y1 = G->yc[1];
        double d = -(y0 + y1) / (y0 * y1) * p->T_bot + y1 / (y0 * (y1 - y0)) * Tm[0] -
                   y0 / (y1 * (y1 - y0)) * Tm[1];
        if (nu_bot) *nu_bot = -H * d / dT;
        double s0 = G->d.ly - G->yc[ny - 1], s1 = G->d.ly - G->yc[ny - 2];
        double e = -(s0 + s1) / (s0 * s1) * p->T_top + s1 / (s0 * (s1 - s0)) * Tm[ny - 1] -
                   s0 / (s1 * (s1 - s0)) * Tm[ny - 2];
        if (nu_top) *nu_top = H * e / dT;
    }
    free(Tm);
    return 0;
}
