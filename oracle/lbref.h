/*
 * lbref.h -- FP64 CPU oracle for the lattice Boltzmann (LB) time step of
 * Shrestha, Mompean & Calzavarini, "Finite Volume vs. Streaming-based Lattice
 * Boltzmann algorithm for fluid-dynamics simulations: a one-to-one accuracy
 * and performance study" (arXiv:1505.03271).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain definition that
 * the CUDA path is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * Conventions (D2Q9, Sec. II of the paper, "reduces to D2Q9 for 2-D flows"):
 *   velocity index a = 0..8, c_0=(0,0), c_1..4=(1,0),(0,1),(-1,0),(0,-1),
 *   c_5..8=(1,1),(-1,1),(-1,-1),(1,-1); weights 4/9, 1/9, 1/36; c_s^2 = 1/3.
 *   Population arrays are [a][j][i] (a slowest, i = x index fastest),
 *   nx*ny doubles per population.  All values are absolute (no offsets).
 *   "tau" is the physical relaxation time (nu = tau c_s^2); the schemes use
 *   tau~ = tau + dt/2 (Sec. II A, below Eq. (ST)).
 */
#ifndef LBREF_H
#define LBREF_H

#ifdef __cplusplus
extern "C" {
#endif

enum { REF_UNIFORM = 0, REF_TANH = 1, REF_SINH = 2, REF_CHEB = 3 };
/* Axis boundaries: periodic; no-slip walls (double reflection, Sec. II B 5);
 * fixed density at both faces of the axis (extrapolated and rescaled ghosts,
 * Sec. II B 5; flow grids only). */
enum { REF_PERIODIC = 0, REF_WALLS = 1, REF_DENSITY = 2 };
enum { REF_INIT_TGV = 0, REF_INIT_SHEAR = 1, REF_INIT_POISEUILLE = 2, REF_INIT_RB = 3 };
/* FV time integration (Sec. II B 2): the semi-implicit collision with the
 * Heun corrector on the advection (Eq. (semi-heun), the default), the same
 * without the corrector (Eq. (semi)), or explicit Euler on the plain
 * populations with the physical tau (Eq. (euler)). */
enum { REF_FV_HEUN = 0, REF_FV_SEMI = 1, REF_FV_EULER = 2 };

typedef struct {
    int nx, ny;
    double lx, ly;
    int sx, sy;                 /* REF_UNIFORM / TANH / SINH / CHEB          */
    double stretch_x, stretch_y;/* tanh: delta = atanh(s1); sinh: s2        */
    int bcx, bcy;               /* REF_PERIODIC / REF_WALLS                 */
    int thermal;                /* 1: second population set g               */
} ref_desc;

typedef struct {
    double tau, dt, tau_g;      /* physical relaxation times, time step     */
    double ax, ay;              /* external acceleration                    */
    double beta, grav;          /* Boussinesq: a_y += beta*grav*(T - T0)    */
    double T0, T_bot, T_top;    /* reference and wall temperatures          */
} ref_params;

typedef struct ref_grid ref_grid;

/* ---- building blocks, exposed so that tests can pin them one by one ---- */
void   ref_lattice(int* cx, int* cy, double* w, int* inv);
void   ref_faces(int n, double L, int spacing, double stretch, double* xi);
void   ref_lagrange3(const double* pos, double x, double* wts);
void   ref_equilibrium(double rho, double ux, double uy, double* feq);
void   ref_guo_force(double rho, double ux, double uy, double ax, double ay, double* F);
double ref_splitmix_uniform(unsigned long long seed, unsigned long long counter);

/* ---- grid state ---- */
ref_grid* ref_create(const ref_desc* d);
void      ref_destroy(ref_grid* g);
int       ref_set_params(ref_grid* g, const ref_params* p);
void      ref_set_threads(int n);
int       ref_get_threads(void);
void      ref_centers(const ref_grid* g, double* xc, double* yc);   /* nx, ny */
void      ref_face_coords(const ref_grid* g, double* xi_x, double* xi_y); /* nx+1, ny+1 */

int ref_init_fields(ref_grid* g, const double* rho, const double* ux,
                    const double* uy, const double* T);
int ref_init_preset(ref_grid* g, int kind, double u0, double amp, int mode,
                    unsigned long long seed);
int ref_set_pops(ref_grid* g, const double* f, const double* gg);
int ref_get_pops(const ref_grid* g, double* f, double* gg);

int ref_step_st(ref_grid* g, int nsteps);
int ref_step_fv(ref_grid* g, int nsteps);
/* Select the FV scheme.  It fixes what the state holds: tilded populations
 * for REF_FV_HEUN and REF_FV_SEMI, plain ones for REF_FV_EULER (whose
 * moments carry no dt/2 a shift and whose initial state is f_eq).  Call it
 * before initialising; ref_step_st refuses an Euler grid (-1). */
int ref_set_scheme(ref_grid* g, int scheme);
/* Densities imposed on the faces of REF_DENSITY axes: x = 0, x = L_x,
 * y = 0, y = L_y (default 1). */
int ref_set_boundary_density(ref_grid* g, double rho_x0, double rho_x1, double rho_y0, double rho_y1);

int ref_moments(const ref_grid* g, double* rho, double* ux, double* uy, double* T);
int ref_conservation(const ref_grid* g, double* mass, double* momx, double* momy,
                     double* heat);
int ref_nusselt(const ref_grid* g, double* nu_vol, double* nu_bot, double* nu_top);

#ifdef __cplusplus
}
#endif
#endif
