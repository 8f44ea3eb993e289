/*
 * lbref3.h -- FP64 CPU oracle of the three-dimensional (D3Q19) lattice
 * Boltzmann step of arXiv:1505.03271: the same ST and FV (semi-implicit
 * collision + Heun, QUICK faces, double-reflection walls) steps as lbref.h on
 * the D3Q19 lattice the paper uses for its 3-D Rayleigh-Benard runs (Sec. IV,
 * Table rb: x and y periodic, plates on z with a sinh grid).
 *
 * TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the
 * benchmark's CPU legs may load it.  It shares no code with the CUDA library.
 *
 * Layout: populations [19][nz][ny][nx] in the order of ref3_lattice; fields
 * [nz][ny][nx].  Gravity acts along -z: a = (ax, ay, az + beta g (T - T0)).
 */
#ifndef LBREF3_H
#define LBREF3_H

#include "lbref.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;
    int sx, sy, sz;                       /* REF_UNIFORM / TANH / SINH / CHEB        */
    double stretch_x, stretch_y, stretch_z;
    int bcx, bcy, bcz;                    /* REF_PERIODIC / REF_WALLS                */
    int thermal;                          /* plates on z; x, y periodic              */
} ref3_desc;

typedef struct {
    double tau, dt, tau_g;
    double ax, ay, az;
    double beta, grav;                    /* a_z += beta grav (T - T0)               */
    double T0, T_bot, T_top;              /* plates at z = 0 and z = L_z             */
} ref3_params;

typedef struct ref3_grid ref3_grid;

void ref3_lattice(int* cx, int* cy, int* cz, double* w, int* inv);
void ref3_equilibrium(double rho, double ux, double uy, double uz, double* feq);
void ref3_guo_force(double rho, double ux, double uy, double uz, double ax, double ay, double az,
                    double* F);

ref3_grid* ref3_create(const ref3_desc* d);
void ref3_destroy(ref3_grid* g);
int ref3_set_params(ref3_grid* g, const ref3_params* p);
/* kind: REF_INIT_TGV (3-D Taylor-Green, u0, periodic box), REF_INIT_SHEAR
 * (u_x = amp sin(2 pi mode z / L_z)), REF_INIT_RB (conductive T on z,
 * barometric rho, seeded perturbation amp dT (2U - 1), U = SplitMix64 of
 * seed ^ ((k ny + j) nx + i)). */
int ref3_init_preset(ref3_grid* g, int kind, double u0, double amp, int mode, unsigned long long seed);
int ref3_init_fields(ref3_grid* g, const double* rho, const double* ux, const double* uy,
                     const double* uz, const double* T);
int ref3_set_pops(ref3_grid* g, const double* f, const double* gg);
int ref3_get_pops(const ref3_grid* g, double* f, double* gg);
int ref3_step_st(ref3_grid* g, int nsteps);
int ref3_step_fv(ref3_grid* g, int nsteps);
int ref3_moments(const ref3_grid* g, double* rho, double* ux, double* uy, double* uz, double* T);
int ref3_conservation(const ref3_grid* g, double* mass, double* mx, double* my, double* mz, double* heat);
int ref3_nusselt(const ref3_grid* g, double* nu_vol, double* nu_bot, double* nu_top);

#ifdef __cplusplus
}
#endif
#endif
