/*
 * lb.h -- C ABI of the GB300 lattice Boltzmann library (libpaper_gb300.so).
 *
 * The library advances a two-dimensional D2Q9 lattice Boltzmann state by the
 * two time-integration schemes of Shrestha, Mompean & Calzavarini,
 * "Finite Volume vs. Streaming-based Lattice Boltzmann algorithm for
 * fluid-dynamics simulations: a one-to-one accuracy and performance study"
 * (arXiv:1505.03271):
 *   - the finite-volume (FV) step: QUICK face fluxes on a stretched Cartesian
 *     grid, semi-implicit BGK collision and Heun predictor-corrector
 *     advection (Sec. II B, Eqs. (fv), (semi), (semi-heun));
 *   - the streaming (ST) step: fused collide-and-stream on the uniform unit
 *     lattice (Sec. II A, Eq. (ST)),
 * for the flow populations f and, optionally, the thermal populations g of the
 * double-population model with Boussinesq buoyancy (Sec. IV, Eq. (LBg)).
 *
 * General conventions
 *   - Every call returns an lb_status and never aborts.  On failure
 *     lb_last_error() returns a message (per calling thread).  A failed call
 *     leaves the grid as it was, except LB_ERR_UNSTABLE (see lb_conservation).
 *   - The library owns all device memory of a grid; callers own every host
 *     array they pass.  Host arrays are row-major [ny][nx] (x fastest);
 *     population arrays are [9][ny][nx], population index slowest, in the
 *     D2Q9 order c_0=(0,0), c_1..4=(1,0),(0,1),(-1,0),(0,-1),
 *     c_5..8=(1,1),(-1,1),(-1,-1),(1,-1).
 *   - Step calls are asynchronous on the grid's CUDA stream; calls that return
 *     host data synchronise that stream.
 *   - Units: lattice units, c_s^2 = 1/3.  lb_params.tau is the physical
 *     relaxation time, nu = tau c_s^2 (Sec. II, below Eq. (LB)); the schemes
 *     relax with tau~ = tau + dt/2 (Sec. II A, below Eq. (ST)).
 *   - The y axis carries the plates of a thermal grid: T_bot at y = 0 and
 *     T_top at y = ly; gravity points to -y.
 */
#ifndef LB_H
#define LB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_grid lb_grid; /* opaque, owned by the library */

typedef enum {
    LB_OK = 0,
    LB_ERR_ARG = 1,      /* invalid argument or unsupported combination       */
    LB_ERR_OOM = 2,      /* device or host allocation failed                   */
    LB_ERR_CUDA = 3,     /* a CUDA call failed (message has the CUDA error)     */
    LB_ERR_STATE = 4,    /* call not valid in the grid's current state          */
    LB_ERR_UNSTABLE = 5, /* non-finite values found: the run has diverged       */
    LB_ERR_TIMEOUT = 6   /* a bounded device-side wait gave up                  */
} lb_status;

/* Face spacing of an axis, Eq. (grids) of Sec. III B: uniform; tanh with
 * stretch delta (s1 = tanh delta); sinh with stretch s2 (even n); Chebyshev
 * faces xi_i = L/2 (1 - cos(i pi / n)) (stretch unused). */
typedef enum { LB_AXIS_UNIFORM = 0, LB_AXIS_TANH = 1, LB_AXIS_SINH = 2, LB_AXIS_CHEB = 3 } lb_spacing;
/* Boundary of an axis (both ends): periodic; no-slip walls (double
 * reflection, Sec. II B 5); or fixed density, where the ghost density is
 * extrapolated linearly through the imposed face value from the node it
 * mirrors and the ghost populations are that node's rescaled by the density
 * ratio (Sec. II B 5; FV on flow grids only, see lb_set_boundary_density). */
typedef enum { LB_BC_PERIODIC = 0, LB_BC_WALLS = 1, LB_BC_DENSITY = 2 } lb_bc;
typedef enum {
    LB_STORE_F64 = 0,    /* FP64 storage, FP64 arithmetic                      */
    LB_STORE_F32 = 1,    /* FP32 storage of f - w (and g - w T0), FP32 math    */
    LB_STORE_F16DEV = 2, /* FP16 storage of f - w (and g - w T0), FP32 math    */
    LB_STORE_BF16DEV = 3 /* BF16 storage of f - w (and g - w T0), FP32 math    */
} lb_store;

/* Grid description.  Face coordinates of each axis follow Eq. (grids) of
 * Sec. III B: uniform xi_i = i L / n; tanh xi_i = L/2 (1 + tanh((2i/n - 1)
 * delta) / tanh(delta)) with stretch = delta (the paper's s1 = tanh(delta));
 * sinh with stretch = s2 and n even.  Cell centres are the face midpoints.
 * Walls (LB_BC_WALLS) sit on the first and last face of that axis.        */
typedef struct {
    int nx, ny;          /* cells per axis, >= 1 (>= 2 on a wall axis)         */
    double lx, ly;       /* domain lengths                                     */
    int sx, sy;          /* lb_spacing per axis                                */
    double stretch_x, stretch_y;
    int bcx, bcy;        /* lb_bc per axis; thermal grids need bcx periodic     */
    int thermal;         /* 0: flow only; 1: flow + thermal populations        */
    int store;           /* lb_store                                           */
    void* cuda_stream;   /* cudaStream_t to enqueue on; NULL = default stream  */
} lb_grid_desc;

/* Physical parameters (Sec. II, Eq. (LB); Sec. IV, Eq. (LBg) and buoyancy
 * a = -beta (T - T0) g with g = -grav y^).                                  */
typedef struct {
    double tau, dt, tau_g;   /* relaxation times (physical) and time step       */
    double ax, ay;           /* external acceleration                          */
    double beta, grav;       /* thermal expansion and gravity: a_y += beta grav (T - T0) */
    double T0, T_bot, T_top; /* reference temperature, plate temperatures      */
} lb_params;

typedef enum {
    LB_INIT_TGV = 0,        /* Taylor-Green vortex of amplitude u0; if amp != 0 a
                               shear wave amp sin(2 pi mode y / ly) is added to u_x */
    LB_INIT_SHEAR = 1,      /* u_x = amp sin(2 pi mode y / ly) (Sec. III A)        */
    LB_INIT_POISEUILLE = 2, /* u_x = 4 u0 y (ly - y) / ly^2 (Sec. III B)           */
    LB_INIT_RB = 3,         /* rest, linear conductive T, barometric rho, plus the
                               seeded perturbation amp (T_bot - T_top)(2U - 1) (Sec. IV) */
    LB_INIT_FIELDS = 4      /* from host arrays rho, ux, uy, T                     */
} lb_init_kind;

typedef struct {
    int kind;                 /* lb_init_kind                                   */
    int mode;                 /* shear-wave mode number                         */
    double u0, amp;
    unsigned long long seed;  /* RB perturbation: U = SplitMix64(seed ^ (j nx + i)) */
    const double *rho, *ux, *uy, *T; /* LB_INIT_FIELDS: host [ny][nx]; NULL = 1, 0, 0, T0 */
} lb_init_desc;

/* Create a grid: allocates two population buffers per population set (the
 * state and the next state), the 1-D metric of each axis (face weights of
 * the QUICK interpolation, Sec. II B 3) and reduction scratch.
 * LB_ERR_ARG on an invalid description, LB_ERR_OOM if device memory runs out.
 * *out is written only on success. */
lb_status lb_create_grid(const lb_grid_desc* desc, lb_grid** out);

/* Set parameters and initial state: f~ = f_eq(rho, u) - dt/2 F (Appendix A,
 * tilded variables at equilibrium) and g~ = (T/rho) f_eq (Eq. (LBg)).
 * Clears the poisoned flag.  LB_ERR_ARG on bad parameters (tau <= 0,
 * dt <= 0, a thermal preset on a flow-only grid, NULL arrays where needed).
 * LB_INIT_FIELDS: each given host array is copied to the device as it is
 * (a DMA when the caller's memory is page-locked), absent ones are filled on
 * the device, and rho > 0 is checked there before any population is
 * written: LB_ERR_ARG names the first cell that fails, and the populations
 * stay as they were.  The host arrays are read before the call returns. */
lb_status lb_init(lb_grid* grid, const lb_params* params, const lb_init_desc* init);

/* Advance nsteps FV time steps (Sec. II B 2, Eq. (semi-heun)): the advected
 * field h = f~ + dt/(2 tau~)(f_eq - f~) + dt/2 F of Eq. (semi) is
 * interpolated to the faces by QUICK (Sec. II B 3), walls use the double
 * reflection of Sec. II B 5 on h (thermal field: anti-reflection through
 * T_wall), the predictor f~* is Eq. (semi) and the corrector averages the
 * two flux divergences.  One fused kernel launch per step (long runs replay
 * the launches as a CUDA graph: lb_set_graph_steps).
 * LB_ERR_STATE if the grid has no parameters or is poisoned. */
lb_status lb_step_fv(lb_grid* grid, int nsteps);

/* Advance nsteps ST time steps, Eq. (ST) with dt = dx = 1: collide and push
 * each population to its neighbour; walls use half-way bounce-back (f) and
 * anti-bounce-back through the plate temperature (g).  Requires uniform axes
 * with unit spacing and dt = 1 (LB_ERR_ARG otherwise), since streaming ties
 * the mesh to the lattice (Sec. II A).  One kernel launch per step (long
 * runs replay the launches as a CUDA graph: lb_set_graph_steps). */
lb_status lb_step_st(lb_grid* grid, int nsteps);

/* Long runs.  A call of lb_step_fv or lb_step_st with more than 2 n steps,
 * n the grid's graph length, takes its first step with a plain launch,
 * captures the next n steps once into a CUDA graph (on a private stream of
 * the grid, created on first use) and replays that graph on the grid's
 * stream; the steps left over launch one by one.  The replays run the same
 * kernels with the same arguments, so the state is bitwise that of n plain
 * launches, and lb_kernel_launches counts each captured kernel once per
 * replay.  Where capture is unavailable (the grid's stream is itself being
 * captured) every step launches directly.  n must be even (the state is back
 * in its buffer after each replay), 0..4096; 0 turns replays off; the
 * default is 32.  LB_ERR_ARG otherwise.  lb_get_graph_steps returns n and
 * the number of graph replays this grid has issued (either pointer may be
 * NULL). */
lb_status lb_set_graph_steps(lb_grid* grid, int n);
lb_status lb_get_graph_steps(lb_grid* grid, int* n, unsigned long long* replays);

/* Kernel schedule of lb_step_fv.  All kernels compute the same step
 * (Eq. (semi-heun)); they differ only in how the grid is cut into CTAs:
 *   LB_FV_TILE:  32 x 16 tiles with a 4-cell halo in both axes, three
 *                shared-memory regions per tile;
 *   LB_FV_MARCH: strips of 120 columns (56 for FP64 thermal) that march up
 *                `chunk` rows each, halo only in x;
 *   LB_FV_PAIR:  the marching strips with two columns per thread and packed
 *                FP32 pair arithmetic; FP32/FP16/BF16 storage and x-periodic
 *                grids only (LB_ERR_ARG otherwise);
 *   LB_FV_PTILE: the tiles with two columns per thread-cell and packed FP32
 *                pair arithmetic (same restrictions); chunk 0 = 32 x 16,
 *                14 = 32 x 14, 16 = 16 x 16, 512 = 32 x 16 with 512 threads
 *                per CTA, 526 = 32 x 14 with 512 threads (one pass per
 *                stage; the corrector splits each cell's populations over
 *                two threads);
 *   LB_FV_SPLIT: the paired step in two launches: collision on tile + 2 and
 *                the predictor on the tile, then the corrector; h* and
 *                f~ + Coll - dt/2 A[h^n] pass through two library-owned FP32
 *                buffers allocated on first use (same restrictions as
 *                LB_FV_PAIR); chunk 0 = 32 x 16, 16 = 16 x 16.
 * LB_FV_AUTO picks by grid size.  For the marching kernels chunk = 0 lets
 * the library size the chunks to fill the GPU; for LB_FV_TILE chunk picks
 * the tile: 0 = 32 x 16, 16 = 16 x 16, 8 = 16 x 8 (smaller tiles recompute
 * more halo but suit small, latency-bound grids).  LB_ERR_ARG on an unknown
 * kernel or chunk. */
typedef enum {
    LB_FV_AUTO = 0, LB_FV_TILE = 1, LB_FV_MARCH = 2, LB_FV_PAIR = 3, LB_FV_PTILE = 4, LB_FV_SPLIT = 5
} lb_fv_kernel;
lb_status lb_set_fv_schedule(lb_grid* grid, int kernel, int chunk);
/* The schedule lb_step_fv will use now (after AUTO has been resolved). */
lb_status lb_get_fv_schedule(lb_grid* grid, int* kernel, int* chunk);

/* FV time integration (Sec. II B 2).  LB_FV_HEUN (default) is the
 * semi-implicit collision with the Heun predictor-corrector on the
 * advection, Eq. (semi-heun).  LB_FV_SEMI stops after the predictor,
 * Eq. (semi).  LB_FV_EULER is explicit Euler on the plain populations with
 * the physical tau, Eq. (euler): the advected field is f itself, the source
 * dt/tau (f_eq - f) + dt F, and the moments carry no dt/2 a shift.
 * The scheme fixes what the state holds (tilded populations, or plain ones
 * for Euler), so setting a different scheme on an initialised grid returns
 * it to the uninitialised state: steps return LB_ERR_STATE until the next
 * lb_init, which then starts from the scheme's equilibrium.  The two
 * single-stage schemes run on the scalar tile kernel whatever the schedule;
 * lb_step_st on an Euler grid returns LB_ERR_STATE.  LB_ERR_ARG on an unknown
 * scheme. */
typedef enum { LB_FV_HEUN = 0, LB_FV_SEMI = 1, LB_FV_EULER = 2 } lb_fv_scheme;

/* Densities imposed on the faces of LB_BC_DENSITY axes (Sec. II B 5):
 * x = 0, x = L_x, y = 0, y = L_y (each > 0; default 1; values for periodic
 * or wall axes are ignored).  They apply from the next FV step on; any time
 * after lb_create_grid.  Grids with a density axis step on the scalar tile
 * kernel whatever the schedule, and lb_step_st returns LB_ERR_ARG on them.
 * LB_ERR_ARG on a non-positive density. */
lb_status lb_set_boundary_density(lb_grid* grid, double rho_x0, double rho_x1, double rho_y0, double rho_y1);
lb_status lb_set_fv_scheme(lb_grid* grid, int scheme);
lb_status lb_get_fv_scheme(lb_grid* grid, int* scheme);

/* Autotuner: times `steps` FV steps for each candidate schedule (the three
 * tile shapes; march and pair with several chunk lengths; the paired tiles
 * and the split schedule where they apply) on the grid's current state,
 * restores the state after each candidate, and keeps the fastest.
 * Synchronous; uses a temporary copy of the populations (and allocates the
 * split schedule's buffers).  LB_ERR_STATE before lb_init. */
lb_status lb_autotune_fv(lb_grid* grid, int steps);

/* Macroscopic fields: rho = sum f~, u = sum c f~ / rho + dt/2 a (Sec. II B 4),
 * T = sum g~ (Eq. (LBg)).  Host outputs [ny][nx]; any may be NULL. Synchronous. */
lb_status lb_moments(lb_grid* grid, double* rho, double* ux, double* uy, double* T);

/* Volume integrals with FP64 accumulation: sum V rho, sum V rho u_x,
 * sum V rho u_y, sum V T (V = dx_i dy_j).  Synchronous.  If any is not
 * finite the grid is marked poisoned and LB_ERR_UNSTABLE is returned (the
 * stability limits of Sec. III C were exceeded); lb_init clears the mark. */
lb_status lb_conservation(lb_grid* grid, double* mass, double* momx, double* momy, double* heat);

/* Nusselt numbers of a thermal grid (Sec. IV): volume
 * Nu = 1 + H <u_y (T - T0)>_V / (kappa (T_bot - T_top)), kappa = tau_g c_s^2;
 * and at each plate from the second-order one-sided gradient of the
 * x-averaged temperature through the wall value and the first two nodes.
 * LB_ERR_STATE on a flow-only grid.  Synchronous. */
lb_status lb_nusselt(lb_grid* grid, double* nu_vol, double* nu_bot, double* nu_top);

/* Copy the tilded populations from/to host FP64 arrays [9][ny][nx]
 * (g may be NULL; it is required on lb_set_populations of a thermal grid
 * unless only f is to change).  The copy rounds to the grid's storage type.
 * Setting populations requires parameters (lb_init first). Synchronous. */
lb_status lb_set_populations(lb_grid* grid, const double* f, const double* g);
lb_status lb_get_populations(lb_grid* grid, double* f, double* g);

/* Copy a w x h window of the populations, starting at cell (x0, y0), to host
 * FP64 arrays [9][h][w] (g may be NULL).  Indices wrap modulo nx, ny, so a
 * window may cross a periodic edge.  Lets callers sample grids too large to
 * copy whole.  LB_ERR_ARG if w or h is < 1 or larger than the grid. */
lb_status lb_get_window(lb_grid* grid, int x0, int y0, int w, int h, double* f, double* g);

/* Mass, momentum and heat sums of lb_conservation (sum V rho, sum V rho u_x,
 * sum V rho u_y, sum V T) for a state held in caller-owned device buffers,
 * computed without allocating any memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, such as a
 * process whose device memory is owned by its own pool or arena (a serving
 * engine that reserves HBM at start-up, a framework's caching allocator) or
 * code on a latency-critical path where an allocation would synchronise the
 * device.  Such a caller cannot create an lb_grid, which allocates.
 *   f, g   device, FP32, [9][ny][pitch]: f - w_a and g - w_a T0 (g may be NULL
 *          for a flow-only state); pitch >= nx elements.
 *   dx, dy device, FP64 cell widths (nx and ny values).
 *   dt, ax, ay, beta_grav, T0: as in lb_params (beta_grav = beta * grav), used
 *          for the force-corrected velocity u = sum c f / rho + dt/2 a.
 *   out    device, 4 doubles, written asynchronously on cuda_stream (NULL =
 *          default stream); read it after the stream has synchronised.
 * Its scratch is a fixed array inside the library (one per GPU that loads it,
 * held until the process exits), so a call handles at most 8,388,608 cells;
 * larger grids return LB_ERR_ARG.  All calls share that array: calls that
 * overlap on the GPU race and must be serialised.  Every call looks up the
 * array's address in the calling thread's current context (so a reset device
 * or a non-primary context uses its own copy); the first call in a context
 * loads the library's module there, so make it before any stream capture
 * begins.  LB_ERR_ARG on NULL or inconsistent sizes,
 * LB_ERR_CUDA if the launch fails. */
lb_status lb_conservation_noalloc(const float* f, const float* g, int nx, int ny, int pitch,
                                  const double* dx, const double* dy, double dt, double ax,
                                  double ay, double beta_grav, double T0, double* out,
                                  void* cuda_stream);

/* ---- Serving: continuous batching of independent FV simulations ----
 * The paper's parameter studies (Sec. III, IV: many runs over grid sizes,
 * Rayleigh numbers and step counts) as a stream of requests.  A server
 * owns the requests' grids; every lb_server_pump() admits queued requests
 * in arrival order while their memory fits (the budget and the device's free
 * memory), advances all active requests together by up to
 * steps_per_launch FV steps (Eq. (semi-heun)) in one batched kernel per
 * step over a device table of (request, tile) entries, replayed from a
 * captured CUDA graph, and retires the requests that are done.  Every tile
 * is stepped by the same code whatever else is in the table, so a request's
 * result is bit-for-bit the same alone and in any batch; it is the
 * LB_FV_TILE step of lb_step_fv (equal up to FP32 rounding, since the two are
 * compiled separately). */
typedef struct lb_server lb_server;

typedef struct {
    long long id;          /* caller's tag, returned in the result            */
    lb_grid_desc grid;     /* its cuda_stream is ignored (the server's is used) */
    lb_params params;
    lb_init_desc init;     /* LB_INIT_FIELDS arrays must live until the request is admitted */
    int nsteps;            /* FV steps to take                                */
} lb_request;

typedef struct {
    long long id;
    int status;            /* LB_OK, or the failure that ended the request    */
    int steps;             /* steps taken                                     */
    long long cells;       /* nx * ny                                         */
    double nu_vol, nu_bot, nu_top; /* Nusselt numbers (thermal servers)       */
    double mass;           /* sum V rho at the end                             */
    double t_submit, t_admit, t_done; /* seconds on the server clock          */
} lb_result;

/* Which admitted requests take steps in a pump:
 *   LB_SERVE_SHARE:    all of them (equal steps for everyone);
 *   LB_SERVE_SHORTEST: least remaining work (cells x steps) first: the first
 *                      one, then as many as fit about two more waves of
 *                      CTAs; the others keep their memory and wait;
 *   LB_SERVE_ARRIVAL:  the earliest submitted first, then as many as fit
 *                      about two more waves of CTAs: first-come first-served
 *                      for the large requests, and the small ones batched,
 *                      riding along with a large one that fills the GPU. */
typedef enum { LB_SERVE_SHARE = 0, LB_SERVE_SHORTEST = 1, LB_SERVE_ARRIVAL = 2 } lb_serve_policy;

/* store/thermal: the one storage type and model all requests use.
 * hbm_budget: bytes of device memory the requests may hold at once.
 * steps_per_launch: >= 1 (steps per pump).  policy: lb_serve_policy.
 * cuda_stream: NULL lets the server create its own non-blocking stream
 * (graph capture needs a non-default stream). */
lb_status lb_server_create(int store, int thermal, unsigned long long hbm_budget, int steps_per_launch,
                           int policy, void* cuda_stream, lb_server** out);
/* Queue a request (host side only).  LB_ERR_ARG if its storage or thermal
 * flag differs from the server's or it alone exceeds the budget. */
lb_status lb_server_submit(lb_server* server, const lb_request* request);
/* Admit, advance and retire as described above.  Synchronous.  Reports how
 * many requests are active and still queued afterwards. */
lb_status lb_server_pump(lb_server* server, int* n_active, int* n_pending);
/* Move up to max finished results into out; *n receives the count. */
lb_status lb_server_results(lb_server* server, lb_result* out, int max, int* n);
/* Seconds since the server was created (the clock of lb_result). */
double lb_server_clock(lb_server* server);
lb_status lb_server_destroy(lb_server* server);

/* Wait for all work queued on the grid's stream. */
lb_status lb_sync(lb_grid* grid);

/* Free the grid and its device memory (NULL is a no-op). */
lb_status lb_destroy(lb_grid* grid);

/* Message of the calling thread's last failure ("" if none). */
const char* lb_last_error(void);

/* Number of kernels this library has launched since it was loaded. */
unsigned long long lb_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* LB_H */
