/*
 * lb3.h -- C ABI of the three-dimensional (D3Q19) lattice Boltzmann step of
 * Shrestha, Mompean & Calzavarini, arXiv:1505.03271.
 *
 * The paper states its method for D3Q19 (Sec. II B 5) and runs it in 3-D on
 * Rayleigh-Benard convection (Sec. IV, Table rb: 128 x 128 x 64 cells, x and
 * y periodic, isothermal plates on z with a sinh grid for FV, uniform for
 * ST).  This header gives that workload the same operations as include/lb.h:
 *   - lb3_step_st: Eq. (ST), collide and stream, dt = dx = 1;
 *   - lb3_step_fv: Eqs. (semi) and (semi-heun) with QUICK faces
 *     (Sec. II B 3) taken dimension by dimension and double-reflection walls
 *     (Sec. II B 5); thermal populations anti-reflected at the z plates;
 *   - observables rho, u, T, conservation sums and Nusselt numbers (Sec. IV).
 *
 * Conventions (as in lb.h): the library owns all device memory; callers own
 * host arrays.  Steps are asynchronous on the grid's stream; getters
 * synchronise.  Every call returns an lb_status and never aborts; the
 * message of the last failure is lb_last_error().
 *
 * Lattice order (index: velocity): 0 (0,0,0); 1 (1,0,0); 2 (-1,0,0);
 * 3 (0,1,0); 4 (0,-1,0); 5 (0,0,1); 6 (0,0,-1); 7 (1,1,0); 8 (-1,-1,0);
 * 9 (1,-1,0); 10 (-1,1,0); 11 (1,0,1); 12 (-1,0,-1); 13 (1,0,-1);
 * 14 (-1,0,1); 15 (0,1,1); 16 (0,-1,-1); 17 (0,1,-1); 18 (0,-1,1).
 * Weights 1/3, 1/18 (axis), 1/36 (edges).  Populations are laid out
 * [19][nz][ny][nx] (x fastest), fields [nz][ny][nx].
 */
#ifndef LB3_H
#define LB3_H

#include "lb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb3_grid lb3_grid; /* opaque, owned by the library */

typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;             /* domain lengths                              */
    int sx, sy, sz;                /* lb_spacing per axis (Eq. (grids))           */
    double stretch_x, stretch_y, stretch_z;
    int bcx, bcy, bcz;             /* LB_BC_PERIODIC or LB_BC_WALLS per axis      */
    int thermal;                   /* g populations; plates on z, x and y periodic */
    int store;                     /* LB_STORE_F64 or LB_STORE_F32                */
    void* cuda_stream;             /* cudaStream_t (NULL: legacy default stream)  */
} lb3_grid_desc;

typedef struct {
    double tau, dt, tau_g;         /* physical relaxation times (nu = tau/3), step */
    double ax, ay, az;             /* external acceleration                       */
    double beta, grav;             /* Boussinesq: a_z += beta grav (T - T0)       */
    double T0, T_bot, T_top;       /* reference and plate temperatures (z = 0, L_z) */
} lb3_params;

typedef struct {
    int kind;                      /* LB_INIT_TGV, LB_INIT_SHEAR, LB_INIT_RB or LB_INIT_FIELDS */
    int mode;                      /* shear wave number                            */
    double u0, amp;                /* TGV amplitude; shear amplitude or RB perturbation */
    unsigned long long seed;       /* RB perturbation seed                         */
    const double *rho, *ux, *uy, *uz, *T; /* LB_INIT_FIELDS: host [nz][ny][nx], any may be NULL */
} lb3_init_desc;

/* Create a grid.  LB_ERR_ARG: a size < 1, a wall axis with < 2 cells, a sinh
 * axis with an odd count, a thermal grid whose x or y axis is not periodic,
 * or a store other than FP64/FP32.  LB_ERR_OOM when the device is full. */
lb_status lb3_create_grid(const lb3_grid_desc* desc, lb3_grid** out);

/* Parameters and initial state at equilibrium in tilded variables
 * (Appendix A): f~ = f_eq(rho, u) - dt/2 F, g~ = (T / rho) f_eq.
 * Presets: 3-D Taylor-Green u = u0 (sin x cos y cos z, -cos x sin y cos z, 0)
 * with its pressure in rho (periodic box); shear u_x = amp sin(2 pi mode z/L_z);
 * Rayleigh-Benard: conductive T on z, barometric rho (Sec. IV) and the seeded
 * perturbation amp (T_bot - T_top)(2U - 1), U = SplitMix64 of
 * seed ^ ((k ny + j) nx + i). */
lb_status lb3_init(lb3_grid* grid, const lb3_params* params, const lb3_init_desc* init);

/* nsteps FV steps, Eq. (semi-heun): four kernel launches per step (the
 * collision pass with h and its z ghost planes, the predictor's flux pass,
 * the moments of f~* with h* and its ghost planes, the corrector's flux
 * pass). */
lb_status lb3_step_fv(lb3_grid* grid, int nsteps);

/* Flux passes of lb3_step_fv (the QUICK divergence of Sec. II B 3):
 *   LB3_FV_PLAIN:  one population per CTA; stencil nodes read through the
 *                  caches; every grid;
 *   LB3_FV_STAGED: one population per CTA; its z planes staged in shared
 *                  memory by bulk asynchronous copies several planes ahead;
 *                  needs x and y periodic and nx a power of two <= 256 whose
 *                  rows are a multiple of 16 bytes (nx >= 4 for FP32, >= 2
 *                  for FP64);
 *   LB3_FV_AUTO:   STAGED where the grid allows it, else PLAIN (default).
 * Both give the same step up to the rounding of the folded face weights.
 * lb3_set_fv_schedule returns LB_ERR_ARG for STAGED on a grid it does not
 * serve; lb3_get_fv_schedule writes the passes a step runs (PLAIN or
 * STAGED). */
#define LB3_FV_AUTO 0
#define LB3_FV_PLAIN 1
#define LB3_FV_STAGED 2
lb_status lb3_set_fv_schedule(lb3_grid* grid, int schedule);
lb_status lb3_get_fv_schedule(lb3_grid* grid, int* resolved);
/* Shape of the staged passes: x rows per tile (1 .. 1024 / nx, FP64
 * 512 / nx), z planes per CTA (1 .. 256) and planes of copies in flight
 * ahead of the arithmetic (1 .. 12); 0 keeps the default of each (rows
 * min(16, 1024 / nx), 16 planes, 3 ahead).  LB_ERR_ARG when out of range or
 * beyond 200 KiB of shared memory per CTA.  Results do not depend on it. */
lb_status lb3_set_fv_staged_shape(lb3_grid* grid, int rows, int planes, int ahead);
/* The shape the staged passes use (defaults resolved for this grid). */
lb_status lb3_get_fv_staged_shape(lb3_grid* grid, int* rows, int* planes, int* ahead);
/* Times the flux schedules on the grid's current state (one warm-up step and
 * `steps` timed steps each, CUDA events on the grid's stream), keeps the
 * fastest and restores the state bit for bit.  Candidates: the plain passes,
 * and where the grid allows them the staged passes with rows per tile
 * {default, default / 2}, planes per CTA {16, 32} and planes ahead {2, 3}.
 * LB_ERR_ARG for steps < 1; LB_ERR_OOM without room for a copy of the
 * state; LB_ERR_TIMEOUT (grid poisoned) if a timed step's wait ran out. */
lb_status lb3_autotune_fv(lb3_grid* grid, int steps);

/* Every wait of the staged passes on its copies is bounded (0.5 s).  A pass
 * whose wait runs out records it on the device, and the next lb3_sync,
 * lb3_moments, lb3_conservation or lb3_nusselt returns LB_ERR_TIMEOUT; the
 * grid is then poisoned (LB_ERR_STATE) until lb3_init.
 * lb3_debug_drop_copies(grid, 1) is the test hook of that path: each CTA of
 * the staged passes announces its first copy group without starting it, so
 * its wait runs out after 2 ms and the step reports LB_ERR_TIMEOUT.  No
 * fault is raised and the context stays usable.  0 restores normal steps. */
lb_status lb3_debug_drop_copies(lb3_grid* grid, int on);

/* nsteps ST steps, Eq. (ST); needs uniform unit spacing on every axis and
 * dt = 1 (LB_ERR_ARG otherwise).  One launch per step. */
lb_status lb3_step_st(lb3_grid* grid, int nsteps);

/* rho, force-corrected u and T per cell (host, [nz][ny][nx]; any may be NULL). */
lb_status lb3_moments(lb3_grid* grid, double* rho, double* ux, double* uy, double* uz, double* T);
/* sum V rho, sum V rho u, sum V T in FP64 (fixed summation order).  Marks the
 * grid LB_ERR_UNSTABLE (until lb3_init) when any sum is not finite. */
lb_status lb3_conservation(lb3_grid* grid, double* mass, double* mx, double* my, double* mz, double* heat);
/* Nu_vol = 1 + H <u_z (T - T0)>_V / (kappa dT) and the plate values from the
 * second-order one-sided gradient of the plane-averaged T (Sec. IV).
 * LB_ERR_STATE on a grid without thermal populations. */
lb_status lb3_nusselt(lb3_grid* grid, double* nu_vol, double* nu_bot, double* nu_top);

/* Populations as FP64 host arrays [19][nz][ny][nx] (g may be NULL). */
lb_status lb3_set_populations(lb3_grid* grid, const double* f, const double* g);
lb_status lb3_get_populations(lb3_grid* grid, double* f, double* g);

lb_status lb3_sync(lb3_grid* grid);
lb_status lb3_destroy(lb3_grid* grid);

#ifdef __cplusplus
}
#endif
#endif
