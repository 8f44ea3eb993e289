// k_fv.cu -- one fused kernel per finite-volume time step (Sec. II B):
// semi-implicit collision + Heun predictor-corrector advection,
// Eqs. (semi) and (semi-heun), with QUICK face values (Sec. II B 3) on a
// stretched Cartesian grid and double-reflection walls (Sec. II B 5).
//
// Each CTA owns a TX x TY tile.  f~^(n+1) on the tile depends on h* two cells
// around it, and h* on h^n two cells further out, so the CTA works on three
// nested regions held in shared memory (compute precision):
//   E4 = tile + 4 halo: h^n (from f~^n, one HBM read per cell)
//   E2 = tile + 2 halo: f~^n + Coll^n, then f~* and h*
//   tile:              f~^(n+1) = f~^n + Coll^n - dt/2 (A[h^n] + A[h*])
// Ghost rows/columns of walls are formed in shared memory from the fluid
// cells next to the wall; they are never stored in HBM.  Every population
// is read from HBM once and written once per step (halo cells re-read from
// L2 by neighbouring CTAs).
#include "lb_internal.cuh"

namespace lbgb {

constexpr int kFvThreads = 256;

// Flux divergence of population a at cell (ix, iy) of a shared-memory region
// with row stride `stride`; (gx, gy) is the grid cell (wrapped) that indexes
// the metric.  c_x (Phi_e - Phi_w)/dx + c_y (Phi_n - Phi_s)/dy, Eq. (fv).
template <typename R, int a>
__device__ __forceinline__ R advect(const R* P, int stride, int ix, int iy, int gx, int gy,
                                    const StepArgs<R>& A) {
    R v = 0;
    const R* row = P + iy * stride;
    if constexpr (cx(a) > 0) {
        const R pe = A.mx.wp(0, gx + 1) * row[ix - 1] + A.mx.wp(1, gx + 1) * row[ix] +
                     A.mx.wp(2, gx + 1) * row[ix + 1];
        const R pw = A.mx.wp(0, gx) * row[ix - 2] + A.mx.wp(1, gx) * row[ix - 1] +
                     A.mx.wp(2, gx) * row[ix];
        v += (pe - pw) * A.mx.invd(gx);
    } else if constexpr (cx(a) < 0) {
        const R pe = A.mx.wm(0, gx + 1) * row[ix] + A.mx.wm(1, gx + 1) * row[ix + 1] +
                     A.mx.wm(2, gx + 1) * row[ix + 2];
        const R pw = A.mx.wm(0, gx) * row[ix - 1] + A.mx.wm(1, gx) * row[ix] +
                     A.mx.wm(2, gx) * row[ix + 1];
        v -= (pe - pw) * A.mx.invd(gx);
    }
    const R* col = P + ix;
    if constexpr (cy(a) > 0) {
        const R pn = A.my.wp(0, gy + 1) * col[(iy - 1) * stride] + A.my.wp(1, gy + 1) * col[iy * stride] +
                     A.my.wp(2, gy + 1) * col[(iy + 1) * stride];
        const R ps = A.my.wp(0, gy) * col[(iy - 2) * stride] + A.my.wp(1, gy) * col[(iy - 1) * stride] +
                     A.my.wp(2, gy) * col[iy * stride];
        v += (pn - ps) * A.my.invd(gy);
    } else if constexpr (cy(a) < 0) {
        const R pn = A.my.wm(0, gy + 1) * col[iy * stride] + A.my.wm(1, gy + 1) * col[(iy + 1) * stride] +
                     A.my.wm(2, gy + 1) * col[(iy + 2) * stride];
        const R ps = A.my.wm(0, gy) * col[(iy - 1) * stride] + A.my.wm(1, gy) * col[iy * stride] +
                     A.my.wm(2, gy) * col[(iy + 1) * stride];
        v -= (pn - ps) * A.my.invd(gy);
    }
    return v;
}

// Flux divergences of all populations: the deviations' part plus the base
// state's own y flux (a per-row constant).
template <typename R, bool TH, int a>
__device__ __forceinline__ void unroll_advect(const R* P, int plane, int stride, int ix, int iy,
                                              int gx, int gy, const StepArgs<R>& A, R* out) {
    out[a] = advect<R, a>(P + a * plane, stride, ix, iy, gx, gy, A) + ref_flux<R, a>(A, gy, false);
    if constexpr (TH)
        out[Q + a] = advect<R, a>(P + (Q + a) * plane, stride, ix, iy, gx, gy, A) + ref_flux<R, a>(A, gy, true);
    if constexpr (a + 1 < Q) unroll_advect<R, TH, a + 1>(P, plane, stride, ix, iy, gx, gy, A, out);
}

// Ghost cells of one shared-memory region W x H whose corner is the grid
// position (gx0, gy0).  Double reflection h_a(x_-k) = h_inv(a)(x_k) for f;
// for g the anti-reflection hg_a(x_-k) = 2 w_a T_wall - hg_inv(a)(x_k), which
// on base-state deviations (T_r odd about T_wall) reads h'_a = -h'_inv(a).
// Thermal grids have their plates on y only.
// Fixed density (flow grids, whose base state is rho_r = 1): the ghost
// density 2 rho_S - rho_k is extrapolated through the face value from the
// mirrored node k and h_a(ghost) = (rho_g / rho_k) h_a(k); on deviations
// h' = h - w this is h'_g = h'_k + s (h'_k + w) with
// s = rho_g / rho_k - 1 = 2 ((rho_S - 1) - sum h'_k) / (1 + sum h'_k).
template <typename R>
__device__ __forceinline__ void density_ghost(R* P, int plane, int dst, int src, R rsd) {
    R sum = 0;
#pragma unroll
    for (int a = 0; a < Q; ++a) sum += P[a * plane + src];
    const R s = R(2) * (rsd - sum) / (R(1) + sum);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const R v = P[a * plane + src];
        P[a * plane + dst] = v + s * (v + wgt<R>(a));
    }
}

template <typename R, bool TH>
__device__ void ghost_fill(R* P, int plane, int W, int H, int gx0, int gy0, const StepArgs<R>& A) {
    if (!TH && A.bcy == LB_BC_DENSITY) {
        for (int k = threadIdx.x; k < W * 4; k += blockDim.x) {
            const int ex = k % W, which = k / W;
            int gxx;
            if (!map_axis(gx0 + ex, A.nx, A.bcx, gxx)) continue;
            const int kk = (which & 1) + 1;
            const bool bot = which < 2;
            const int ey = (bot ? -kk : A.ny - 1 + kk) - gy0, eys = (bot ? kk - 1 : A.ny - kk) - gy0;
            if (ey < 0 || ey >= H) continue;
            density_ghost<R>(P, plane, ey * W + ex, eys * W + ex, bot ? A.rhobd[2] : A.rhobd[3]);
        }
    }
    if (!TH && A.bcx == LB_BC_DENSITY) {
        for (int k = threadIdx.x; k < H * 4; k += blockDim.x) {
            const int ey = k % H, which = k / H;
            int gyy;
            if (!map_axis(gy0 + ey, A.ny, A.bcy, gyy)) continue;
            const int kk = (which & 1) + 1;
            const bool lft = which < 2;
            const int ex = (lft ? -kk : A.nx - 1 + kk) - gx0, exs = (lft ? kk - 1 : A.nx - kk) - gx0;
            if (ex < 0 || ex >= W) continue;
            density_ghost<R>(P, plane, ey * W + ex, ey * W + exs, lft ? A.rhobd[0] : A.rhobd[1]);
        }
    }
    if (A.bcy == LB_BC_WALLS) {
        for (int k = threadIdx.x; k < W * 4; k += blockDim.x) {
            const int ex = k % W, which = k / W;  // 0,1: bottom ghost 1,2; 2,3: top ghost 1,2
            int gxx;
            if (!map_axis(gx0 + ex, A.nx, A.bcx, gxx)) continue;
            const int kk = (which & 1) + 1;
            const bool bot = which < 2;
            const int gy = bot ? -kk : A.ny - 1 + kk;
            const int gys = bot ? kk - 1 : A.ny - kk;
            const int ey = gy - gy0, eys = gys - gy0;
            if (ey < 0 || ey >= H) continue;
            const int dst = ey * W + ex, src = eys * W + ex;
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                P[a * plane + dst] = P[inv(a) * plane + src];
                if (TH) P[(Q + a) * plane + dst] = -P[(Q + inv(a)) * plane + src];
            }
        }
    }
    if (A.bcx == LB_BC_WALLS) {
        for (int k = threadIdx.x; k < H * 4; k += blockDim.x) {
            const int ey = k % H, which = k / H;
            int gyy;
            if (!map_axis(gy0 + ey, A.ny, A.bcy, gyy)) continue;
            const int kk = (which & 1) + 1;
            const bool lft = which < 2;
            const int gx = lft ? -kk : A.nx - 1 + kk;
            const int gxs = lft ? kk - 1 : A.nx - kk;
            const int ex = gx - gx0, exs = gxs - gx0;
            if (ex < 0 || ex >= W) continue;
            const int dst = ey * W + ex, src = ey * W + exs;
#pragma unroll
            for (int a = 0; a < Q; ++a) P[a * plane + dst] = P[inv(a) * plane + src];
        }
    }
}

// One FV step on the tile whose first cell is (x0, y0).
template <typename R, typename S, bool TH, int TX, int TY>
__device__ __forceinline__ void fv_tile(const StepArgs<R>& A, const int x0, const int y0) {
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr int EX = TX + 8, EY = TY + 8, NE = EX * EY;
    constexpr int BX = TX + 4, BY = TY + 4, NB = BX * BY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sH = reinterpret_cast<R*>(smem_raw);  // [NQ][EY][EX]  h^n
    R* sFC = sH + NQ * NE;                   // [NQ][BY][BX]  f~ + Coll, then f~ + Coll - dt/2 A^n
    R* sHs = sFC + NQ * NB;                  // [NQ][BY][BX]  h*
    const S* fin = static_cast<const S*>(A.fin);
    const S* gin = static_cast<const S*>(A.gin);

    // ---- time level n on E4: h^n, and f~ + Coll^n on E2 ----
    for (int k = threadIdx.x; k < NE; k += blockDim.x) {
        const int ex = k % EX, ey = k / EX;
        int gx, gy;
        if (!map_axis(x0 - 4 + ex, A.nx, A.bcx, gx) || !map_axis(y0 - 4 + ey, A.ny, A.bcy, gy))
            continue;
        const long long c = (long long)gy * A.pitch + gx;
        R d[Q], e[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) d[a] = Store<S>::ld(fin + a * A.plane + c);
        if constexpr (TH) {
#pragma unroll
            for (int a = 0; a < Q; ++a) e[a] = Store<S>::ld(gin + a * A.plane + c);
        }
        Cell<R, TH> m;
        m.moments(d, e, A, A.roff[gy], A.toff[gy]);
        const bool inB = ex >= 2 && ex < EX - 2 && ey >= 2 && ey < EY - 2;
        const int kb = (ey - 2) * BX + (ex - 2);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            R feqd, F, geqd = 0;
            m.eq(a, A, feqd, F, geqd);
            const R neq = feqd - d[a];
            sH[a * NE + k] = d[a] + A.omh * neq + A.hF * F;          // h, Eq. (semi) bracket
            if (inB) sFC[a * NB + kb] = d[a] + A.om * neq + A.cf * F;  // f~ + Coll
            if constexpr (TH) {
                const R neqg = geqd - e[a];
                sH[(Q + a) * NE + k] = e[a] + A.omgh * neqg;
                if (inB) sFC[(Q + a) * NB + kb] = e[a] + A.omg * neqg;
            }
        }
    }
    __syncthreads();
    ghost_fill<R, TH>(sH, NE, EX, EY, x0 - 4, y0 - 4, A);
    __syncthreads();

    // ---- predictor on E2: f~* = f~ + Coll - dt A[h^n] (Eq. (semi)), then h* ----
    for (int k = threadIdx.x; k < NB; k += blockDim.x) {
        const int bx = k % BX, by = k / BX;
        int gx, gy;
        if (!map_axis(x0 - 2 + bx, A.nx, A.bcx, gx) || !map_axis(y0 - 2 + by, A.ny, A.bcy, gy))
            continue;
        const bool tile = bx >= 2 && bx < BX - 2 && by >= 2 && by < BY - 2;
        R adv[NQ];
        unroll_advect<R, TH, 0>(sH, NE, EX, bx + 2, by + 2, gx, gy, A, adv);
        R fs[Q], es[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const R fc = sFC[a * NB + k];
            fs[a] = fc - A.dt * adv[a];
            if (tile) sFC[a * NB + k] = fc - A.hf * adv[a];
            if constexpr (TH) {
                const R gc = sFC[(Q + a) * NB + k];
                es[a] = gc - A.dt * adv[Q + a];
                if (tile) sFC[(Q + a) * NB + k] = gc - A.hf * adv[Q + a];
            }
        }
        if (A.stages == 1) {
            // single-stage schemes (Eqs. (semi), (euler)): the predictor is
            // the new state of the tile's cells
            // (a ragged tile's cells past the grid edge wrap on a periodic
            // axis; the CTA that owns them writes them)
            if (tile && x0 - 2 + bx < A.nx && y0 - 2 + by < A.ny) {
                const long long c = (long long)gy * A.pitch + gx;
                S* fout = static_cast<S*>(A.fout);
                S* gout = static_cast<S*>(A.gout);
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    Store<S>::st(fout + a * A.plane + c, fs[a]);
                    if constexpr (TH) Store<S>::st(gout + a * A.plane + c, es[a]);
                }
            }
            continue;
        }
        Cell<R, TH> m;
        m.moments(fs, es, A, A.roff[gy], A.toff[gy]);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            R feqd, F, geqd = 0;
            m.eq(a, A, feqd, F, geqd);
            sHs[a * NB + k] = fs[a] + A.omh * (feqd - fs[a]) + A.hF * F;
            if constexpr (TH) sHs[(Q + a) * NB + k] = es[a] + A.omgh * (geqd - es[a]);
        }
    }
    if (A.stages == 1) return;  // uniform over the CTA
    __syncthreads();
    ghost_fill<R, TH>(sHs, NB, BX, BY, x0 - 2, y0 - 2, A);
    __syncthreads();

    // ---- corrector on the tile, Eq. (semi-heun) ----
    S* fout = static_cast<S*>(A.fout);
    S* gout = static_cast<S*>(A.gout);
    for (int k = threadIdx.x; k < TX * TY; k += blockDim.x) {
        const int tx = k % TX, ty = k / TX;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx >= A.nx || gy >= A.ny) continue;
        const int bx = tx + 2, by = ty + 2, kb = by * BX + bx;
        R adv[NQ];
        unroll_advect<R, TH, 0>(sHs, NB, BX, bx, by, gx, gy, A, adv);
        const long long c = (long long)gy * A.pitch + gx;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            Store<S>::st(fout + a * A.plane + c, sFC[a * NB + kb] - A.hf * adv[a]);
            if constexpr (TH) Store<S>::st(gout + a * A.plane + c, sFC[(Q + a) * NB + kb] - A.hf * adv[Q + a]);
        }
    }
}

template <typename R, typename S, bool TH, int TX, int TY>
__global__ void __launch_bounds__(kFvThreads) k_fv(const StepArgs<R> A) {
    fv_tile<R, S, TH, TX, TY>(A, blockIdx.x * TX, blockIdx.y * TY);
}

// Many grids in one launch: CTA b steps tile tiles[b] = (request, tile x,
// tile y) of request reqs[tile.x], using step k of the launch sequence to
// pick that request's input buffer; requests with fewer than k + 1 steps
// left are skipped.  Each tile runs the tile code of k_fv with parameters
// read from the table, so a request gives the same bits alone and in any
// batch.
template <typename R, typename S, bool TH, int TX, int TY>
__global__ void __launch_bounds__(kFvThreads)
k_fv_batched(const BatchReq<R>* reqs, const int4* tiles, const int* ntiles, const int k) {
    if ((int)blockIdx.x >= *ntiles) return;
    const int4 t = tiles[blockIdx.x];
    const BatchReq<R>& B = reqs[t.x];
    if (k >= B.remaining) return;
    StepArgs<R> A = B.args;
    const int p = (B.parity + k) & 1;
    A.fin = B.f[p];
    A.fout = B.f[p ^ 1];
    A.gin = B.g[p];
    A.gout = B.g[p ^ 1];
    fv_tile<R, S, TH, TX, TY>(A, t.y * TX, t.z * TY);
}

template <typename R, typename S, bool TH, int TX, int TY>
static cudaError_t run_fv_batched(const void* reqs, const int4* tiles, const int* ntiles, int capacity, int k,
                                  cudaStream_t s) {
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr size_t smem = sizeof(R) * (size_t)NQ * ((TX + 8) * (TY + 8) + 2 * (TX + 4) * (TY + 4));
    {
        cudaError_t e = set_max_smem((const void*)k_fv_batched<R, S, TH, TX, TY>, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_fv_batched<R, S, TH, TX, TY><<<capacity, kFvThreads, smem, s>>>(static_cast<const BatchReq<R>*>(reqs),
                                                                      tiles, ntiles, k);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fv_batched(Prec p, bool th, const void* reqs, const int4* tiles, const int* ntiles,
                              int capacity, int k, cudaStream_t s) {
    switch (p) {
        case Prec::F64:
            return th ? run_fv_batched<double, double, true, 16, 16>(reqs, tiles, ntiles, capacity, k, s)
                      : run_fv_batched<double, double, false, 32, 16>(reqs, tiles, ntiles, capacity, k, s);
        case Prec::F32:
            return th ? run_fv_batched<float, float, true, 32, 16>(reqs, tiles, ntiles, capacity, k, s)
                      : run_fv_batched<float, float, false, 32, 16>(reqs, tiles, ntiles, capacity, k, s);
        case Prec::F16:
            return th ? run_fv_batched<float, __half, true, 32, 16>(reqs, tiles, ntiles, capacity, k, s)
                      : run_fv_batched<float, __half, false, 32, 16>(reqs, tiles, ntiles, capacity, k, s);
        case Prec::BF16:
            return th ? run_fv_batched<float, __nv_bfloat16, true, 32, 16>(reqs, tiles, ntiles, capacity, k, s)
                      : run_fv_batched<float, __nv_bfloat16, false, 32, 16>(reqs, tiles, ntiles, capacity, k, s);
    }
    return cudaErrorInvalidValue;
}

void tile_shape(Prec p, bool th, int* tx, int* ty) {
    *tx = (p == Prec::F64 && th) ? 16 : 32;
    *ty = 16;
}

template <typename R, typename S, bool TH, int TX, int TY>
static cudaError_t run_fv(const void* vargs, cudaStream_t s) {
    const StepArgs<R>& A = *static_cast<const StepArgs<R>*>(vargs);
    constexpr int NQ = TH ? 2 * Q : Q;
    constexpr size_t smem = sizeof(R) * (size_t)NQ * ((TX + 8) * (TY + 8) + 2 * (TX + 4) * (TY + 4));
    static_assert(smem <= 232448, "shared memory per CTA");
    {
        cudaError_t e = set_max_smem((const void*)k_fv<R, S, TH, TX, TY>, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((A.nx + TX - 1) / TX, (A.ny + TY - 1) / TY);
    k_fv<R, S, TH, TX, TY><<<grid, kFvThreads, smem, s>>>(A);
    count_launch();
    return cudaGetLastError();
}

// Tile shape variants: 0 = 32 x 16 (16 x 16 for FP64 thermal), 16 = 16 x 16,
// 8 = 16 x 8.  Smaller tiles recompute more halo but give more, shorter
// CTAs, which is what small grids (latency-bound) want.
template <typename R, typename S, bool TH>
static cudaError_t run_fv_shape(const void* args, int shape, cudaStream_t s) {
    if (shape == 8) return run_fv<R, S, TH, 16, 8>(args, s);
    if (shape == 16) return run_fv<R, S, TH, 16, 16>(args, s);
    if constexpr (sizeof(R) == 8 && TH) return run_fv<R, S, TH, 16, 16>(args, s);
    else return run_fv<R, S, TH, 32, 16>(args, s);
}

cudaError_t launch_fv(Prec p, bool th, const void* args, int shape, cudaStream_t s) {
    switch (p) {
        case Prec::F64:
            return th ? run_fv_shape<double, double, true>(args, shape, s)
                      : run_fv_shape<double, double, false>(args, shape, s);
        case Prec::F32:
            return th ? run_fv_shape<float, float, true>(args, shape, s)
                      : run_fv_shape<float, float, false>(args, shape, s);
        case Prec::F16:
            return th ? run_fv_shape<float, __half, true>(args, shape, s)
                      : run_fv_shape<float, __half, false>(args, shape, s);
        case Prec::BF16:
            return th ? run_fv_shape<float, __nv_bfloat16, true>(args, shape, s)
                      : run_fv_shape<float, __nv_bfloat16, false>(args, shape, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbgb
