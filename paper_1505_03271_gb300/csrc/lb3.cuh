// lb3.cuh -- D3Q19 lattice and the argument blocks of the three-dimensional
// kernels (private to the library; the C ABI is include/lb3.h).
//
// Storage holds deviations from a constant reference: f - w and g - w T0
// (FP64 or FP32).  Gravity acts along -z: a = (ax, ay, az + beta g (T - T0)).
#pragma once

#include "lb_internal.cuh"

namespace lbgb {

constexpr int Q3 = 19;

// D3Q19 in the order of include/lb3.h: rest; +-x, +-y, +-z; then the twelve
// edge velocities in opposite pairs (xy, xz, yz planes).  inv(a) = a +- 1.
__host__ __device__ constexpr int c3x(int a) {
    return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1
           : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0;
}
__host__ __device__ constexpr int c3y(int a) {
    return (a == 3 || a == 7 || a == 10 || a == 15 || a == 17) ? 1
           : (a == 4 || a == 8 || a == 9 || a == 16 || a == 18) ? -1 : 0;
}
__host__ __device__ constexpr int c3z(int a) {
    return (a == 5 || a == 11 || a == 14 || a == 15 || a == 18) ? 1
           : (a == 6 || a == 12 || a == 13 || a == 16 || a == 17) ? -1 : 0;
}
__host__ __device__ constexpr int inv3(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }
template <typename R>
__host__ __device__ constexpr R w3(int a) {
    return a == 0 ? R(1) / R(3) : (a <= 6 ? R(1) / R(18) : R(1) / R(36));
}
static_assert(c3x(inv3(7)) == -c3x(7) && c3y(inv3(9)) == -c3y(9) && c3z(inv3(18)) == -c3z(18), "inv3");

// The same velocities packed 2 bits per population (value c + 1), one word
// per component, for loops over a runtime population index.
__host__ __device__ constexpr unsigned long long pack3(int ax, int a) {
    return a < 0 ? 0ULL
                 : pack3(ax, a - 1) |
                       ((unsigned long long)((ax == 0 ? c3x(a) : ax == 1 ? c3y(a) : c3z(a)) + 1) << (2 * a));
}
__host__ __device__ constexpr int c3comp(int a, int ax) {
    return (int)(((ax == 0 ? pack3(0, Q3 - 1) : ax == 1 ? pack3(1, Q3 - 1) : pack3(2, Q3 - 1)) >> (2 * a)) & 3ULL) - 1;
}
static_assert(c3comp(13, 0) == 1 && c3comp(13, 2) == -1 && c3comp(10, 1) == 1 && c3comp(0, 2) == 0, "pack");

// Face-major metric of one axis: for face k (k = 0..n) eight values
// [wp0 wp1 wp2 wm0 wm1 wm2 1/dx_k 0] (1/dx of cell k; 0 for k = n), so that a
// thread reads the weights of its two faces at fixed offsets.
constexpr int kFaceRow = 8;

// Arguments of one 3-D step in compute precision R.
template <typename R>
struct Args3 {
    const void* fin;
    void* fout;
    const void* gin;
    void* gout;
    R* H;    // [19][nz + 4][ny][nx] advected field h' (time n), two ghost planes each side in z
    R* FC;   // [19][N] f' + Coll, then f' + Coll - dt/2 A[h^n]
    R* HS;   // [19][nz + 4][ny][nx] f~*' (parked), then h*'
    R* HG;   // thermal counterparts
    R* GC;
    R* HGS;
    int n[3];           // nx, ny, nz
    int bc[3];          // LB_BC_PERIODIC / LB_BC_WALLS per axis
    long long N;        // nx ny nz
    long long NP;       // nx ny (nz + 4): population stride of the padded fields
    AxisMetric<R> m[3]; // QUICK weights and 1/width per axis
    const R* ft[3];     // the same, face-major (kFaceRow values per face)
    R dt, om, omh, cf, hf, omg, omgh;
    R hF;  // force part of the advected field: dt/2 (1 - dt/(2 tau~))
    R ax, ay, az, bg, T0, dTb, dTt;  // dTb, dTt: plate temperature - T0 (z walls)
    // staged flux passes (k3_staged.cu): status word a CTA sets when a bounded
    // wait runs out, the limit of each wait, and the test hook that leaves
    // the first copy group of every CTA unstarted
    int* werr;
    unsigned long long wait_ns;
    int drop_copy;
    int sshape[3];  // requested rows per tile, planes per CTA, planes ahead (0: default)
};

struct Aux3 {
    const void* f;
    const void* g;
    int n[3];
    long long N;
    double dt, ax, ay, az, bg, T0;
};

// One FV step.  staged: run the flux passes of k3_staged.cu (the grid must
// pass adv3_staged_ok).
cudaError_t launch3_fv(Prec p, bool th, bool staged, const void* args, cudaStream_t s);
// The staged flux pass (k3_staged.cu): whether it serves a grid, and one launch
// (corr: the corrector's pass; np: 19 or 38 populations).
bool adv3_staged_ok(const int* n, const int* bc, Prec p);
// whether a requested (rows per tile, planes per CTA, planes ahead) fits the grid (0: default)
bool adv3_staged_shape_ok(const int* n, Prec p, int ty, int kc, int ahead);
// the shape a launch uses for a request (0 entries: the defaults)
void adv3_staged_resolve(const int* n, Prec p, int* ty, int* kc, int* ahead);
cudaError_t launch3_adv_staged(Prec p, bool corr, int np, const void* args, cudaStream_t s);
cudaError_t launch3_st(Prec p, bool th, const void* args, cudaStream_t s);
// the paired FP32 ST step (k3_st_pair.cu): grids with an even nx
bool st3_pair_ok(Prec p, const int* n);
cudaError_t launch3_st_pair(bool th, const void* args, cudaStream_t s);
// fields [5][N] (rho, ux, uy, uz, T) on the device -> storage (equilibrium in tilded variables)
cudaError_t launch3_init(Prec p, bool th, const Aux3& a, const double* fields, void* f, void* g, cudaStream_t s);
// storage -> fields [5][N]
cudaError_t launch3_moments(Prec p, bool th, const Aux3& a, double* fields, cudaStream_t s);
// FP64 [19][N] <-> storage (value - w off)
cudaError_t launch3_pack(Prec p, const double* src, void* dst, long long N, double off, cudaStream_t s);
cudaError_t launch3_unpack(Prec p, const void* src, double* dst, long long N, double off, cudaStream_t s);
// per-plane sums of the observables: out[nz][8] = (sum V rho, sum V rho u (3), sum V T,
// sum V u_z (T - T0), sum A T, sum V) over the cells of plane k, fixed order
cudaError_t launch3_plane_sums(const double* fields, const double* dx, const double* dy, const double* dz,
                               int nx, int ny, int nz, double T0, double* out, cudaStream_t s);

}  // namespace lbgb
