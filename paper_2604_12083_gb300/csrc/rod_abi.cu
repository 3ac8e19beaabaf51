// rod_abi.cu -- host side of rod_forces, rod_step, rot_sqrt_batch and the rod workspaces.
#include <cmath>
#include <cstring>

#include "rod_internal.h"

namespace mrs {

template <typename T>
static int dalloc(T** p, size_t n)
{
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cudaMalloc of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
        return MRS_ENOMEM;
    }
    return MRS_OK;
}

static int check_rods(int n_rods, const int64_t* rod_off)
{
    MRS_REQUIRE(n_rods >= 1, "n_rods must be >= 1 (got %d)", n_rods);
    MRS_REQUIRE(rod_off != nullptr, "rod_off is NULL");
    MRS_REQUIRE(rod_off[0] == 0, "rod_off[0] must be 0");
    for (int r = 0; r < n_rods; ++r) {
        const int64_t M = rod_off[r + 1] - rod_off[r];
        MRS_REQUIRE(M >= 2 && M <= 4096, "rod %d has %lld nodes (2..4096 allowed)", r, (long long)M);
    }
    MRS_REQUIRE(rod_off[n_rods] < (1LL << 30), "too many nodes");
    return MRS_OK;
}

static int check_params(const mrs_rod_params* p, bool need_fluid)
{
    MRS_REQUIRE(p != nullptr, "params is NULL");
    MRS_REQUIRE(std::isfinite(p->L) && p->L > 0.0, "L must be > 0");
    for (int i = 0; i < 3; ++i)
        MRS_REQUIRE(std::isfinite(p->a[i]) && std::isfinite(p->b[i]), "moduli must be finite");
    MRS_REQUIRE(std::isfinite(p->wave_A) && std::isfinite(p->wave_k) && std::isfinite(p->wave_f),
                "wave parameters must be finite");
    if (need_fluid) {
        MRS_REQUIRE(std::isfinite(p->mu) && p->mu > 0.0, "mu must be > 0");
        MRS_REQUIRE(std::isfinite(p->eps) && p->eps > 0.0, "eps must be > 0");
    }
    MRS_REQUIRE(std::isfinite(p->lj_eps) && p->lj_eps >= 0.0, "lj_eps must be >= 0");
    if (p->lj_eps > 0.0)
        MRS_REQUIRE(std::isfinite(p->lj_sigma) &&
                        (p->lj_sigma > 0.0 || (std::isfinite(p->eps) && p->eps > 0.0)),
                    "Lennard-Jones repulsion needs lj_sigma > 0, or lj_sigma = 0 and eps > 0 "
                    "(sigma = 3 eps)");
    return MRS_OK;
}

void rod_ws_free(RodWorkspace* ws)
{
    if (!ws) return;
    for (auto& g : ws->graphs) cudaGraphExecDestroy(g.exec);
    if (ws->cap) cudaStreamDestroy(ws->cap);
    if (ws->plan) plan_free(ws->plan);
    void* ptrs[] = {ws->d_node_info, ws->d_chunks, ws->d_wchunks, ws->d_t0, ws->d_step, ws->d_FN, ws->d_Xf, ws->d_gf, ws->d_mf,
                    ws->d_u, ws->d_w, ws->d_g64, ws->d_m64, ws->d_u64, ws->d_w64, ws->d_Xh, ws->d_Dh,
                    ws->d_segsc};
    for (void* q : ptrs) cudaFree(q);
    delete ws;
}

int rod_ws_get(mrs_ctx* ctx, int n_rods, const int64_t* rod_off, int n_inst, int precision,
               double mu, double eps, RodWorkspace** out, int tag)
{
    *out = nullptr;
    for (auto it = ctx->rod_ws.begin(); it != ctx->rod_ws.end(); ++it) {
        RodWorkspace* ws = *it;
        if (ws->n_inst != n_inst || ws->n_rods != n_rods || ws->precision != precision ||
            ws->tag != tag)
            continue;
        if (std::memcmp(ws->rod_off.data(), rod_off, sizeof(int64_t) * (n_rods + 1)) != 0) continue;
        if ((eps > 0.0) != (ws->plan != nullptr)) continue;
        if (ws->plan && (ws->plan->mu != mu || ws->plan->eps[0] != eps)) continue;
        ctx->rod_ws.erase(it);
        ctx->rod_ws.push_front(ws);
        *out = ws;
        return MRS_OK;
    }
    RodWorkspace* ws = new RodWorkspace();
    ws->ctx = ctx;
    ws->n_inst = n_inst;
    ws->tag = tag;
    ws->n_rods = n_rods;
    ws->precision = precision;
    ws->rod_off.assign(rod_off, rod_off + n_rods + 1);
    ws->N1 = (int)rod_off[n_rods];
    ws->N = ws->N1 * n_inst;
    const size_t N = (size_t)ws->N;
    std::vector<int2> info(N);
    std::vector<int> chunks;
    std::vector<int4> wchunks;
    for (int i = 0; i < n_inst; ++i)
        for (int r = 0; r < n_rods; ++r) {
            const int M = (int)(rod_off[r + 1] - rod_off[r]);
            for (int k = 0; k < M; ++k) info[(size_t)i * ws->N1 + rod_off[r] + k] = make_int2(k, M);
            for (int c = 0; c < M; c += kRodChunk - 1)
                chunks.push_back((int)((size_t)i * ws->N1 + rod_off[r] + c));
            for (int c = 0; c < M; c += kWNodes)
                wchunks.push_back(make_int4((int)((size_t)i * ws->N1 + rod_off[r] + c), M, c, i));
        }
    ws->n_chunks = (int)chunks.size();
    ws->n_wchunks = (int)wchunks.size();
    int st;
    if ((st = dalloc(&ws->d_node_info, N)) || (st = dalloc(&ws->d_chunks, chunks.size())) ||
        (ws->n_wchunks && (st = dalloc(&ws->d_wchunks, wchunks.size()))) ||
        (st = dalloc(&ws->d_t0, n_inst)) ||
        (st = dalloc(&ws->d_step, 1)) || (st = dalloc(&ws->d_FN, 6 * N)) ||
        (st = dalloc(&ws->d_Xh, 3 * N)) || (st = dalloc(&ws->d_Dh, 9 * N)) ||
        (st = dalloc(&ws->d_segsc, N))) {
        rod_ws_free(ws);
        return st;
    }
    if (precision == MRS_F64) {
        if ((st = dalloc(&ws->d_g64, 3 * N)) || (st = dalloc(&ws->d_m64, 3 * N)) ||
            (st = dalloc(&ws->d_u64, 3 * N)) || (st = dalloc(&ws->d_w64, 3 * N))) {
            rod_ws_free(ws);
            return st;
        }
    } else {
        if ((st = dalloc(&ws->d_Xf, 3 * N)) || (st = dalloc(&ws->d_gf, 3 * N)) ||
            (st = dalloc(&ws->d_mf, 3 * N)) || (st = dalloc(&ws->d_u, 3 * N)) ||
            (st = dalloc(&ws->d_w, 3 * N))) {
            rod_ws_free(ws);
            return st;
        }
    }
    cudaMemcpy(ws->d_node_info, info.data(), N * sizeof(int2), cudaMemcpyHostToDevice);
    cudaMemcpy(ws->d_chunks, chunks.data(), chunks.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (ws->n_wchunks)
        cudaMemcpy(ws->d_wchunks, wchunks.data(), wchunks.size() * sizeof(int4), cudaMemcpyHostToDevice);
    cudaMemset(ws->d_t0, 0, n_inst * sizeof(double));
    cudaMemset(ws->d_step, 0, sizeof(long long));
    if (eps > 0.0) {
        std::vector<int64_t> off(n_inst + 1);
        for (int i = 0; i <= n_inst; ++i) off[i] = (int64_t)i * ws->N1;
        st = plan_build(ctx, n_inst, off.data(), mu, eps, nullptr, precision, -1, &ws->plan);
        if (st) {
            rod_ws_free(ws);
            return st;
        }
    }
    cudaError_t e = cudaStreamCreateWithFlags(&ws->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        rod_ws_free(ws);
        set_error("rod workspace set-up failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    ctx->rod_ws.push_front(ws);
    while (ctx->rod_ws.size() > ctx->rod_ws_max) {
        RodWorkspace* old = ctx->rod_ws.back();
        ctx->rod_ws.pop_back();
        cudaDeviceSynchronize();
        rod_ws_free(old);
    }
    *out = ws;
    return MRS_OK;
}

RodLaunch rod_launch(const RodWorkspace* ws, const mrs_rod_params* p, double dt)
{
    RodLaunch L;
    L.N = ws->N;
    L.nodes_per_inst = ws->N1;
    L.node_info = ws->d_node_info;
    L.t0 = ws->d_t0;
    L.step = ws->d_step;
    L.dt = dt;
    L.p = *p;
    L.p.lj_sigma = lj_sigma_of(*p);
    L.FN = ws->d_FN;
    L.chunks = ws->d_chunks;
    L.n_chunks = ws->n_chunks;
    // warp-cooperative force kernel: small batches by default (mrs_ctx_set_rod_force_kernel)
    const int fk = ws->ctx ? ws->ctx->rod_force_kernel : 0;
    const bool warp_forces = fk == 2 || (fk == 0 && ws->N <= kWarpForceMaxNodes);
    L.wchunks = warp_forces && ws->n_wchunks ? ws->d_wchunks : nullptr;
    L.n_wchunks = ws->n_wchunks;
    L.inv_L = 1.0 / p->L;
    set_pack_reference(L, ws->n_rods, ws->rod_off.data());
    L.segsc = (ws->segsc_k == p->wave_k && ws->segsc_L == p->L) ? ws->d_segsc : nullptr;
    L.err = ws->ctx ? ws->ctx->d_err : nullptr;
    return L;
}

// (Re)builds the workspace's segment table for p's wave number and rod length when they changed.
static int rod_ws_prepare(RodWorkspace* ws, const mrs_rod_params* p, cudaStream_t s)
{
    if (ws->segsc_k == p->wave_k && ws->segsc_L == p->L) return MRS_OK;
    cudaError_t e = launch_segment_table(ws->N, ws->d_node_info, p->wave_k, p->L, ws->d_segsc, s);
    if (e != cudaSuccess) {
        set_error("segment table kernel failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    ws->segsc_k = p->wave_k;
    ws->segsc_L = p->L;
    return MRS_OK;
}

int rod_ws_set_times(RodWorkspace* ws, double t_first, double dT, cudaStream_t s)
{
    MRS_CHECK_CUDA(launch_set_times(ws->d_t0, ws->n_inst, t_first, dT, ws->d_step, s));
    return MRS_OK;
}

// Velocities of the current stage: forces -> (float32 pack) -> pair sum.  up (or NULL): the
// update that follows, which the pair sum applies itself when its plan runs the cluster kernel
// (*fused then true).
static int enqueue_velocity(RodWorkspace* ws, const RodLaunch& L, const double* X, const double* D,
                            double t_off, cudaStream_t s, const PlanUpdate* up = nullptr,
                            bool* fused = nullptr)
{
    if (fused) *fused = false;
    cudaError_t e;
    if (ws->precision == MRS_F64) {
        e = launch_rod_forces(L, X, D, t_off, ws->d_g64, ws->d_m64, nullptr, nullptr, nullptr, s);
        if (e != cudaSuccess) {
            set_error("rod force kernels failed: %s", cudaGetErrorString(e));
            return MRS_ECUDA;
        }
        return plan_run(ws->plan, X, ws->d_g64, ws->d_m64, nullptr, ws->d_u64, ws->d_w64, s);
    }
    e = launch_rod_forces(L, X, D, t_off, nullptr, nullptr, ws->d_Xf, ws->d_gf, ws->d_mf, s);
    if (e != cudaSuccess) {
        set_error("rod force kernels failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    return plan_run(ws->plan, ws->d_Xf, ws->d_gf, ws->d_mf, nullptr, ws->d_u, ws->d_w, s, up, fused);
}

static cudaError_t enqueue_update(RodWorkspace* ws, const RodLaunch& L, const double* X0,
                                  const double* D0, double h, double* X1, double* D1, bool bump,
                                  cudaStream_t s)
{
    if (ws->precision == MRS_F64)
        return launch_rod_update64(L, X0, D0, ws->d_u64, ws->d_w64, h, X1, D1, bump, s);
    return launch_rod_update(L, X0, D0, ws->d_u, ws->d_w, h, X1, D1, bump, s);
}

// One stage: velocities at (Xs, Ds, t_off), then (X1, D1) = update of (X0, D0) by h with them
// (in the pair-sum launch when its plan allows, else by the update kernel).
static int enqueue_stage(RodWorkspace* ws, const RodLaunch& L, const double* Xs, const double* Ds,
                         double t_off, const double* X0, const double* D0, double h, double* X1,
                         double* D1, bool bump, cudaStream_t s)
{
    // with the warp-cooperative kernels (small batches, mrs_ctx_set_rod_force_kernel) only: the
    // thread-per-segment setting keeps the separate update kernel
    const PlanUpdate up{X0, D0, X1, D1, h, bump ? L.step : nullptr};
    const bool offer = ws->precision != MRS_F64 && L.wchunks != nullptr;
    bool fused = false;
    int st = enqueue_velocity(ws, L, Xs, Ds, t_off, s, offer ? &up : nullptr, &fused);
    if (st || fused) return st;
    const cudaError_t e = enqueue_update(ws, L, X0, D0, h, X1, D1, bump, s);
    if (e != cudaSuccess) {
        set_error("rod update kernel failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    return MRS_OK;
}

// One time step (Euler or explicit-midpoint RK2) enqueued on s.
static int enqueue_step(RodWorkspace* ws, const RodLaunch& L, double* X, double* D, int scheme,
                        cudaStream_t s)
{
    if (scheme == MRS_EULER) return enqueue_stage(ws, L, X, D, 0.0, X, D, L.dt, X, D, true, s);
    const int st = enqueue_stage(ws, L, X, D, 0.0, X, D, 0.5 * L.dt, ws->d_Xh, ws->d_Dh, false, s);
    if (st) return st;
    return enqueue_stage(ws, L, ws->d_Xh, ws->d_Dh, 0.5 * L.dt, X, D, L.dt, X, D, true, s);
}

static int get_graph(RodWorkspace* ws, const mrs_rod_params* p, double* X, double* D, double dt,
                     int scheme, int steps, cudaGraphExec_t* out)
{
    for (auto& g : ws->graphs) {
        if (g.X == X && g.D == D && g.scheme == scheme && g.steps == steps && g.dt == dt &&
            g.force_kernel == ws->ctx->rod_force_kernel && std::memcmp(&g.p, p, sizeof(*p)) == 0) {
            *out = g.exec;
            return MRS_OK;
        }
    }
    const RodLaunch L = rod_launch(ws, p, dt);
    cudaGraph_t graph = nullptr;
    MRS_CHECK_CUDA(cudaStreamBeginCapture(ws->cap, cudaStreamCaptureModeThreadLocal));
    int st = MRS_OK;
    for (int i = 0; i < steps && st == MRS_OK; ++i) st = enqueue_step(ws, L, X, D, scheme, ws->cap);
    cudaError_t e = cudaStreamEndCapture(ws->cap, &graph);
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) {
        set_error("graph capture failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        set_error("graph instantiation failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    if (ws->graphs.size() >= 8) {
        cudaGraphExecDestroy(ws->graphs.front().exec);
        ws->graphs.erase(ws->graphs.begin());
    }
    RodWorkspace::Graph g;
    g.X = X;
    g.D = D;
    g.force_kernel = ws->ctx->rod_force_kernel;
    g.scheme = scheme;
    g.steps = steps;
    g.dt = dt;
    g.p = *p;
    g.exec = exec;
    ws->graphs.push_back(g);
    *out = exec;
    return MRS_OK;
}

constexpr int kStepsPerGraph = 16;

int rod_ws_steps(RodWorkspace* ws, const mrs_rod_params* p, double* X, double* D, double dt,
                 int nsteps, int scheme, cudaStream_t s)
{
    if (nsteps <= 0 || ws->N == 0) return MRS_OK;
    int pst = rod_ws_prepare(ws, p, s);
    if (pst) return pst;
    // small instances: every step of every instance in one launch, the state in shared memory
    // (one CTA per instance)
    // (by default only when the batch is too large for the warp-cooperative kernels of the
    // graph path, which are faster for a batch of up to kWarpForceMaxNodes nodes)
    const int fmode = ws->ctx->fused_steps;
    const int fk = ws->ctx->rod_force_kernel;
    const bool warp_kernels = fk == 2 || (fk == 0 && ws->N <= kWarpForceMaxNodes);
    if (fmode > 0 && ws->precision != MRS_F64 && fused_fits(ws->N1) &&
        (fmode == 2 || (ws->N1 <= kFusedAutoNodes && !warp_kernels))) {
        const RodLaunch L = rod_launch(ws, p, dt);
        cudaError_t e = launch_rod_fine_fused(L, X, D, nsteps, scheme, p->mu, p->eps, s);
        if (e != cudaSuccess) {
            set_error("fused rod step kernel failed: %s", cudaGetErrorString(e));
            return MRS_ECUDA;
        }
        return MRS_OK;
    }
    const int chunk = nsteps < kStepsPerGraph ? nsteps : kStepsPerGraph;
    cudaGraphExec_t gx = nullptr, gr = nullptr;
    int st = get_graph(ws, p, X, D, dt, scheme, chunk, &gx);
    if (st) return st;
    const int rem = nsteps % chunk;
    if (rem) {
        st = get_graph(ws, p, X, D, dt, scheme, rem, &gr);
        if (st) return st;
    }
    for (int i = 0; i < nsteps / chunk; ++i) MRS_CHECK_CUDA(cudaGraphLaunch(gx, s));
    if (rem) MRS_CHECK_CUDA(cudaGraphLaunch(gr, s));
    return MRS_OK;
}

}  // namespace mrs

using namespace mrs;

extern "C" {

int rod_forces(mrs_ctx* ctx, int n_rods, const int64_t* rod_off, const mrs_rod_params* p,
               const double* X, const double* D, double t, double* g, double* m, void* stream)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr, "ctx is NULL");
    int st = check_rods(n_rods, rod_off);
    if (st) return st;
    if ((st = check_params(p, false))) return st;
    MRS_REQUIRE(X && D && g && m, "NULL pointer");
    MRS_REQUIRE(std::isfinite(t), "t must be finite");
    MRS_CHECK_CUDA(cudaSetDevice(ctx->device));
    RodWorkspace* ws = nullptr;
    if ((st = rod_ws_get(ctx, n_rods, rod_off, 1, MRS_F64, 0.0, 0.0, &ws))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = rod_ws_prepare(ws, p, s))) return st;
    const RodLaunch L = rod_launch(ws, p, 0.0);
    if ((st = rod_ws_set_times(ws, 0.0, 0.0, s))) return st;
    cudaError_t e = launch_rod_forces(L, X, D, t, g, m, nullptr, nullptr, nullptr, s);
    if (e != cudaSuccess) {
        set_error("rod force kernels failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    return MRS_OK;
}

int rod_step(mrs_ctx* ctx, int n_rods, const int64_t* rod_off, const mrs_rod_params* p, double* X,
             double* D, double t0, double dt, int nsteps, int scheme, int mrs_precision,
             void* stream)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr, "ctx is NULL");
    int st = check_rods(n_rods, rod_off);
    if (st) return st;
    if ((st = check_params(p, true))) return st;
    MRS_REQUIRE(X && D, "NULL state pointer");
    MRS_REQUIRE(scheme == MRS_EULER || scheme == MRS_RK2, "unknown scheme %d", scheme);
    MRS_REQUIRE(mrs_precision == MRS_F64 || mrs_precision == MRS_F32 || mrs_precision == MRS_F32_COMP,
                "unknown precision %d", mrs_precision);
    MRS_REQUIRE(std::isfinite(t0) && std::isfinite(dt) && dt > 0.0, "t0 must be finite and dt > 0");
    MRS_REQUIRE(nsteps >= 0, "nsteps must be >= 0");
    if (nsteps == 0) return MRS_OK;
    MRS_CHECK_CUDA(cudaSetDevice(ctx->device));
    RodWorkspace* ws = nullptr;
    if ((st = rod_ws_get(ctx, n_rods, rod_off, 1, mrs_precision, p->mu, p->eps, &ws))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = rod_ws_set_times(ws, t0, 0.0, s))) return st;
    return rod_ws_steps(ws, p, X, D, dt, nsteps, scheme, s);
}

int rod_advance(mrs_ctx* ctx, int64_t N, double* X, double* D, const void* u, const void* w,
                double dt, int vel_f64, void* stream)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr, "ctx is NULL");
    MRS_REQUIRE(N >= 0 && N < (1LL << 30), "N out of range");
    MRS_REQUIRE(std::isfinite(dt), "dt must be finite");
    if (N == 0) return MRS_OK;
    MRS_REQUIRE(X && D && u && w, "NULL pointer");
    MRS_CHECK_CUDA(cudaSetDevice(ctx->device));
    RodLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.N = (int)N;
    L.nodes_per_inst = (int)N;
    cudaError_t e = vel_f64 ? launch_rod_update64(L, X, D, (const double*)u, (const double*)w, dt, X, D,
                                                  false, (cudaStream_t)stream)
                            : launch_rod_update(L, X, D, (const float*)u, (const float*)w, dt, X, D, false,
                                                (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error("rod update kernel failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    return MRS_OK;
}

int rot_sqrt_batch(mrs_ctx* ctx, int n, const double* R, double* S, void* stream)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr, "ctx is NULL");
    MRS_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return MRS_OK;
    MRS_REQUIRE(R && S, "NULL pointer");
    MRS_CHECK_CUDA(cudaSetDevice(ctx->device));
    cudaError_t e = launch_rot_sqrt_batch(n, R, S, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error("rotation square root kernel failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    return MRS_OK;
}

}  // extern "C"
