// lb_serve.cu -- continuous-batching server for streams of independent FV
// simulations (the paper's parameter studies run as requests).
//
// A request is an ordinary lb_grid plus a step count.  lb_server_pump()
//   1. admits queued requests in arrival order while their device memory
//      fits the budget and the device's free memory (others wait),
//   2. advances every active request by up to K steps in K launches of one
//      batched FV kernel over a device table of (request, tile) entries; the
//      K launches are captured once in a CUDA graph and replayed while the
//      table's capacity is unchanged (only the table contents change),
//   3. retires requests that have taken all their steps: Nusselt numbers and
//      mass are computed, the grid is freed, the result is queued.
// Every tile is stepped by the same code whatever else is in the table, so a
// request's result does not depend on what it was batched with.
#include <algorithm>
#include <chrono>
#include <deque>
#include <string>
#include <vector>

#include "lb_grid.cuh"

using namespace lbgb;

namespace lbgb {
lb_status set_last_error(lb_status s, const char* msg);
}

namespace {

struct Active {
    lb_request req;
    lb_grid* grid = nullptr;
    int remaining = 0;
    int done = 0;
    double t_submit = 0, t_admit = 0;
    size_t bytes = 0;
};

struct Pending {
    lb_request req;
    double t_submit = 0;
};

size_t grid_bytes(const lb_grid_desc& d) {
    const size_t pitch = ((size_t)d.nx + 31) / 32 * 32;
    const size_t pops = 9 * pitch * (size_t)d.ny * elem_size(d.store) * 2 * (d.thermal ? 2 : 1);
    return pops + 4 * sizeof(double) * (size_t)d.nx * d.ny + 64 * ((size_t)d.nx + d.ny + 64);
}

lb_status fail(lb_status s, const std::string& m) { return set_last_error(s, m.c_str()); }

}  // namespace

struct lb_server {
    int store = LB_STORE_F32;
    int thermal = 0;
    Prec prec = Prec::F32;
    size_t budget = 0, used = 0;
    int K = 2;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::deque<Pending> pending;
    std::vector<Active> active;
    std::deque<lb_result> finished;
    // device tables and their host staging
    int cap_req = 0, cap_tiles = 0;
    void* d_reqs = nullptr;
    int4* d_tiles = nullptr;
    int* d_ntiles = nullptr;
    void* h_reqs = nullptr;
    int4* h_tiles = nullptr;
    int* h_ntiles = nullptr;
    cudaGraphExec_t graph = nullptr;
    // the captured launches hold the table pointers: a graph is replayed
    // only while the tables it was captured with are still the current ones
    unsigned long long table_gen = 0, graph_gen = 0;
    bool graph_paired = false;
    bool warmed = false;
    bool all_periodic_x = true;  // every active request has a periodic x axis
    int policy = LB_SERVE_SHARE;
    int sms = 152;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

size_t req_size(Prec p) { return p == Prec::F64 ? sizeof(BatchReq<double>) : sizeof(BatchReq<float>); }

lb_status ensure_capacity(lb_server* S, int nreq, int ntiles) {
    if (nreq <= S->cap_req && ntiles <= S->cap_tiles) return LB_OK;
    int cr = S->cap_req, ct = S->cap_tiles;
    while (cr < nreq) cr = cr ? 2 * cr : 64;
    while (ct < ntiles) ct = ct ? 2 * ct : 1024;
    if (S->d_reqs) cudaFree(S->d_reqs);
    if (S->d_tiles) cudaFree(S->d_tiles);
    if (S->h_reqs) cudaFreeHost(S->h_reqs);
    if (S->h_tiles) cudaFreeHost(S->h_tiles);
    S->d_reqs = nullptr;
    S->d_tiles = nullptr;
    S->h_reqs = nullptr;
    S->h_tiles = nullptr;
    ++S->table_gen;  // the old tables are gone: any captured graph is stale
    const size_t rs = req_size(S->prec);
    if (cudaMalloc(&S->d_reqs, rs * cr) != cudaSuccess || cudaMalloc((void**)&S->d_tiles, sizeof(int4) * ct) != cudaSuccess ||
        cudaMallocHost(&S->h_reqs, rs * cr) != cudaSuccess ||
        cudaMallocHost((void**)&S->h_tiles, sizeof(int4) * ct) != cudaSuccess) {
        cudaGetLastError();
        S->cap_req = S->cap_tiles = 0;
        return fail(LB_ERR_OOM, "server: no memory for the tile table");
    }
    S->cap_req = cr;
    S->cap_tiles = ct;
    return LB_OK;
}

template <typename R>
void fill_req(lb_server* S, int i, const Active& a) {
    BatchReq<R>* t = static_cast<BatchReq<R>*>(S->h_reqs) + i;
    t->args = step_args<R>(a.grid, a.grid->p.dt);
    t->f[0] = a.grid->f[0];
    t->f[1] = a.grid->f[1];
    t->g[0] = a.grid->g[0];
    t->g[1] = a.grid->g[1];
    t->parity = a.grid->cur;
    t->remaining = a.remaining;
}

// The paired tile kernel (packed FP32 arithmetic) serves FP32/FP16/BF16
// requests with periodic x; FP64 and x-wall requests use the scalar tile.
bool paired(const lb_server* S) { return S->prec != Prec::F64 && S->all_periodic_x; }

lb_status launch_steps(lb_server* S, int ncap) {
    for (int k = 0; k < S->K; ++k) {
        cudaError_t e = paired(S) ? launch_fv_ptile_batched(S->prec, S->thermal != 0, S->d_reqs, S->d_tiles,
                                                            S->d_ntiles, ncap, k, S->stream)
                                  : launch_fv_batched(S->prec, S->thermal != 0, S->d_reqs, S->d_tiles, S->d_ntiles,
                                                      ncap, k, S->stream);
        if (e != cudaSuccess) return fail(LB_ERR_CUDA, std::string("server launch: ") + cudaGetErrorString(e));
    }
    return LB_OK;
}

// K batched launches: plain launches the first time (so that per-kernel
// attributes are set outside any capture), then a captured graph replayed
// while the device tables it was captured with are still in place (both
// are reallocated when either capacity grows).
lb_status run_batch(lb_server* S) {
    const int ncap = S->cap_tiles;
    if (!S->warmed) {
        S->warmed = true;
        return launch_steps(S, ncap);
    }
    if (!S->graph || S->graph_gen != S->table_gen || S->graph_paired != paired(S)) {
        if (S->graph) cudaGraphExecDestroy(S->graph);
        S->graph = nullptr;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail(LB_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        lb_status st = launch_steps(S, ncap);
        e = cudaStreamEndCapture(S->stream, &g);
        if (st != LB_OK) return st;
        if (e != cudaSuccess) return fail(LB_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&S->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(LB_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
        S->graph_gen = S->table_gen;
        S->graph_paired = paired(S);
    }
    cudaError_t e = cudaGraphLaunch(S->graph, S->stream);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return LB_OK;
}

void retire(lb_server* S, Active& a, lb_status status) {
    lb_result r{};
    r.id = a.req.id;
    r.steps = a.done;
    r.t_submit = a.t_submit;
    r.t_admit = a.t_admit;
    r.cells = (long long)a.req.grid.nx * a.req.grid.ny;
    r.status = status;
    if (status == LB_OK) {
        double mass = 0;
        lb_status s = lb_conservation(a.grid, &mass, nullptr, nullptr, nullptr);
        r.mass = mass;
        if (s == LB_OK && S->thermal) s = lb_nusselt(a.grid, &r.nu_vol, &r.nu_bot, &r.nu_top);
        r.status = s;
    }
    r.t_done = S->now();
    lb_destroy(a.grid);
    a.grid = nullptr;
    S->used -= a.bytes;
    S->finished.push_back(r);
}

}  // namespace

extern "C" {

lb_status lb_server_create(int store, int thermal, unsigned long long hbm_budget, int steps_per_launch,
                           int policy, void* cuda_stream, lb_server** out) {
    if (!out) return fail(LB_ERR_ARG, "NULL output");
    if (policy != LB_SERVE_SHARE && policy != LB_SERVE_SHORTEST && policy != LB_SERVE_ARRIVAL)
        return fail(LB_ERR_ARG, "unknown policy");
    if (store < LB_STORE_F64 || store > LB_STORE_BF16DEV) return fail(LB_ERR_ARG, "bad store");
    if (steps_per_launch < 1) return fail(LB_ERR_ARG, "steps_per_launch must be >= 1");
    lb_server* S = new lb_server();
    S->store = store;
    S->thermal = thermal ? 1 : 0;
    S->prec = prec_of(store);
    S->budget = hbm_budget;
    S->K = steps_per_launch;
    S->policy = policy;
    S->stream = static_cast<cudaStream_t>(cuda_stream);
    if (!S->stream) {
        if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete S;
            return fail(LB_ERR_CUDA, "server: cannot create a stream");
        }
        S->own_stream = true;
    }
    S->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&S->device);
    cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device);
    if (S->sms <= 0) S->sms = 152;
    if (cudaMalloc((void**)&S->d_ntiles, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&S->h_ntiles, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return fail(LB_ERR_OOM, "server: allocation failed");
    }
    *out = S;
    return LB_OK;
}

double lb_server_clock(lb_server* S) { return S ? S->now() : 0.0; }

lb_status lb_server_submit(lb_server* S, const lb_request* r) {
    if (!S || !r) return fail(LB_ERR_ARG, "NULL argument");
    if (r->grid.store != S->store || (r->grid.thermal != 0) != (S->thermal != 0))
        return fail(LB_ERR_ARG, "request storage/thermal flags differ from the server's");
    if (r->nsteps < 0) return fail(LB_ERR_ARG, "nsteps must be >= 0");
    if (grid_bytes(r->grid) > S->budget) return fail(LB_ERR_ARG, "request larger than the server's memory budget");
    S->pending.push_back({*r, S->now()});
    return LB_OK;
}

lb_status lb_server_pump(lb_server* S, int* n_active, int* n_pending) {
    if (!S) return fail(LB_ERR_ARG, "server is NULL");
    // 1. admission in arrival order, by budget and free device memory
    while (!S->pending.empty()) {
        const Pending& p = S->pending.front();
        const size_t need = grid_bytes(p.req.grid);
        size_t free_b = 0, total_b = 0;
        cudaError_t me = cudaMemGetInfo(&free_b, &total_b);
        if (me != cudaSuccess) return fail(LB_ERR_CUDA, std::string("server admission: ") + cudaGetErrorString(me));
        if (S->used + need > S->budget || need + (64u << 20) > free_b) break;
        Active a;
        a.req = p.req;
        a.t_submit = p.t_submit;
        a.remaining = p.req.nsteps;
        a.bytes = need;
        lb_grid_desc d = p.req.grid;
        d.cuda_stream = S->stream;
        lb_status st = lb_create_grid(&d, &a.grid);
        if (st == LB_OK) st = lb_init(a.grid, &p.req.params, &p.req.init);
        if (st == LB_OK) {
            // the batched kernels use the tile decomposition
            a.grid->fv_kernel = LB_FV_TILE;
            a.t_admit = S->now();
            S->used += need;
            S->active.push_back(a);
            S->pending.pop_front();
        } else if (st == LB_ERR_OOM) {
            if (a.grid) lb_destroy(a.grid);
            break;  // wait for memory to free up
        } else {
            lb_result r{};
            r.id = p.req.id;
            r.status = st;
            r.t_submit = p.t_submit;
            r.t_admit = r.t_done = S->now();
            if (a.grid) lb_destroy(a.grid);
            S->finished.push_back(r);
            S->pending.pop_front();
        }
    }
    // requests with no steps finish at once
    for (size_t i = 0; i < S->active.size();) {
        if (S->active[i].remaining == 0) {
            retire(S, S->active[i], LB_OK);
            S->active.erase(S->active.begin() + i);
        } else {
            ++i;
        }
    }
    if (!S->active.empty()) {
        // 2. tile table of the active set and one batched launch sequence
        S->all_periodic_x = true;
        for (const Active& a : S->active) S->all_periodic_x = S->all_periodic_x && a.req.grid.bcx == LB_BC_PERIODIC;
        int tx = 32, ty = 16;
        if (!paired(S)) tile_shape(S->prec, S->thermal != 0, &tx, &ty);
        auto tiles_of = [&](const Active& a) {
            return ((a.req.grid.nx + tx - 1) / tx) * ((a.req.grid.ny + ty - 1) / ty);
        };
        // which requests take steps this pump
        std::vector<int> order(S->active.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
        std::vector<char> run(S->active.size(), 1);
        if (S->policy != LB_SERVE_SHARE) {
            // least remaining work first (SHORTEST) or the active list's
            // arrival order (ARRIVAL): the first request always steps, and
            // the next ones join while their tiles fit in about two more
            // waves of CTAs, so small requests ride along with a large one
            // that fills the GPU by itself
            if (S->policy == LB_SERVE_SHORTEST)
                std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
                    const Active &p = S->active[x], &q = S->active[y];
                    return (double)p.req.grid.nx * p.req.grid.ny * p.remaining <
                           (double)q.req.grid.nx * q.req.grid.ny * q.remaining;
                });
            const int target = 2 * S->sms * (S->thermal ? 1 : 2);
            int sum = 0;  // tiles of the requests after the first
            for (size_t j = 0; j < order.size(); ++j) {
                const int t = tiles_of(S->active[order[j]]);
                run[order[j]] = (j == 0 || sum + t <= target) ? 1 : 0;
                if (run[order[j]] && j > 0) sum += t;
            }
        }
        int ntiles = 0;
        for (size_t i = 0; i < S->active.size(); ++i)
            if (run[i]) ntiles += tiles_of(S->active[i]);
        lb_status st = ensure_capacity(S, (int)S->active.size(), ntiles);
        if (st != LB_OK) return st;
        int b = 0;
        for (int i = 0; i < (int)S->active.size(); ++i) {
            const Active& a = S->active[i];
            if (S->prec == Prec::F64) fill_req<double>(S, i, a);
            else fill_req<float>(S, i, a);
            if (!run[i]) continue;
            const int nbx = (a.req.grid.nx + tx - 1) / tx, nby = (a.req.grid.ny + ty - 1) / ty;
            for (int y = 0; y < nby; ++y)
                for (int x = 0; x < nbx; ++x) S->h_tiles[b++] = make_int4(i, x, y, 0);
        }
        *S->h_ntiles = ntiles;
        // a failed upload would leave the previous pump's tables in place: stop before stepping
        cudaError_t ue = cudaMemcpyAsync(S->d_reqs, S->h_reqs, req_size(S->prec) * S->active.size(),
                                         cudaMemcpyHostToDevice, S->stream);
        if (ue == cudaSuccess)
            ue = cudaMemcpyAsync(S->d_tiles, S->h_tiles, sizeof(int4) * ntiles, cudaMemcpyHostToDevice, S->stream);
        if (ue == cudaSuccess)
            ue = cudaMemcpyAsync(S->d_ntiles, S->h_ntiles, sizeof(int), cudaMemcpyHostToDevice, S->stream);
        if (ue != cudaSuccess) return fail(LB_ERR_CUDA, std::string("server table upload: ") + cudaGetErrorString(ue));
        st = run_batch(S);
        if (st != LB_OK) return st;
        cudaError_t e = cudaStreamSynchronize(S->stream);
        if (e != cudaSuccess) return fail(LB_ERR_CUDA, std::string("server step: ") + cudaGetErrorString(e));
        // 3. bookkeeping and retirement
        for (size_t i = 0, j = 0; i < S->active.size(); ++j) {
            Active& a = S->active[i];
            if (!run[j]) {
                ++i;
                continue;
            }
            const int taken = a.remaining < S->K ? a.remaining : S->K;
            a.remaining -= taken;
            a.done += taken;
            a.grid->cur = (a.grid->cur + taken) & 1;
            if (a.remaining == 0) {
                retire(S, a, LB_OK);
                S->active.erase(S->active.begin() + i);
            } else {
                ++i;
            }
        }
    }
    if (n_active) *n_active = (int)S->active.size();
    if (n_pending) *n_pending = (int)S->pending.size();
    return LB_OK;
}

lb_status lb_server_results(lb_server* S, lb_result* out, int max, int* n) {
    if (!S || !n || (max > 0 && !out)) return fail(LB_ERR_ARG, "NULL argument");
    int k = 0;
    while (k < max && !S->finished.empty()) {
        out[k++] = S->finished.front();
        S->finished.pop_front();
    }
    *n = k;
    return LB_OK;
}

lb_status lb_server_destroy(lb_server* S) {
    if (!S) return LB_OK;
    cudaStreamSynchronize(S->stream);
    for (Active& a : S->active)
        if (a.grid) lb_destroy(a.grid);
    if (S->graph) cudaGraphExecDestroy(S->graph);
    if (S->d_reqs) cudaFree(S->d_reqs);
    if (S->d_tiles) cudaFree(S->d_tiles);
    if (S->d_ntiles) cudaFree(S->d_ntiles);
    if (S->h_reqs) cudaFreeHost(S->h_reqs);
    if (S->h_tiles) cudaFreeHost(S->h_tiles);
    if (S->h_ntiles) cudaFreeHost(S->h_ntiles);
    if (S->own_stream) cudaStreamDestroy(S->stream);
    delete S;
    return LB_OK;
}

}  // extern "C"
