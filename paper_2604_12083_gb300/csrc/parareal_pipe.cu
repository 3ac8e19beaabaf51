// parareal_pipe.cu -- the pipelined Parareal schedule on one GPU (Section III-A).
//
// The regular schedule (parareal.cu) waits for a whole serial correction sweep before the next
// iteration's fine solves start.  Here the slices are cut into groups of consecutive slices;
// each group's fine solves run on their own stream and workspace and start as soon as the
// previous sweep has produced the group's last input state -- the coarse/correction sweep
// streams its results downstream and the fine solves overlap with it.  All ordering is by CUDA
// events between streams:
//   E[n]      the current sweep has produced U[n]               (sweep stream -> fine streams)
//   copied[j] group j has copied its inputs out of U             (fine stream -> sweep stream,
//             so the next sweep never overwrites a state a group still has to read)
//   done[j]   group j's fine results are in FX/FD                (fine stream -> sweep stream)
// The fine buffers alternate between iterations (FX[k % 2]) so that the speculative fine solves
// of iteration k+1 never overwrite rows that sweep k still reads.
// The host enqueues sweep k, then (speculatively) the fine solves of iteration k+1, and only
// then reads eta~^k; if iteration k converged, the speculative fine work is discarded (it only
// writes the fine buffers).  Discarded speculative work costs real time, so speculation is
// skipped when the increments so far predict that iteration k converges
// (eta~^{k-1} * (eta~^{k-1} / eta~^{k-2}) < tol, the geometric trend of the last two
// increments), or, at k = 2 where there is no trend yet, when eta~^1 is within kSpecFirst of
// tol (measured ratios eta~^2 / eta~^1 run from 0.004 to 0.2, so such an iteration 2 may well
// converge, and a wasted iteration costs far more than the overlap of one sweep): the host then
// reads eta~^k first and enqueues the fine solves of iteration k+1 only if they are needed.
// This holds for small systems too, whose fine stages leave most of the GPU idle: on one
// 128-node rod (64 slices) an unneeded fifth fine iteration made the pipelined schedule slower
// than the regular one (0.117 against 0.104 s); with the rule it runs no discarded steps
// (0.112 s).  No kernel waits on another kernel.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "rod_internal.h"

using namespace mrs;

namespace {

constexpr double kSpecFirst = 1e3;        // k = 2: speculate only if eta~^1 >= kSpecFirst tol

struct DBuf {
    double* p = nullptr;
    ~DBuf() { cudaFree(p); }
};

struct Streams {
    std::vector<cudaStream_t> s;
    std::vector<cudaEvent_t> e;
    ~Streams()
    {
        for (cudaStream_t x : s) {
            cudaStreamSynchronize(x);
            cudaStreamDestroy(x);
        }
        for (cudaEvent_t x : e) cudaEventDestroy(x);
    }
    cudaError_t stream(cudaStream_t* out)
    {
        cudaError_t r = cudaStreamCreateWithFlags(out, cudaStreamNonBlocking);
        if (!r) s.push_back(*out);
        return r;
    }
    cudaError_t event(cudaEvent_t* out)
    {
        cudaError_t r = cudaEventCreateWithFlags(out, cudaEventDisableTiming);
        if (!r) e.push_back(*out);
        return r;
    }
};

}  // namespace

extern "C" int parareal_run_pipelined(mrs_ctx* ctx, int n_rods, const int64_t* rod_off,
                                      const mrs_rod_params* p, double* X, double* D, double T0,
                                      double T1, int n_slices, double dt_fine, int coarse_ratio,
                                      int max_iter, double tol, int group_size,
                                      mrs_parareal_stats* out, void* stream)
{
    clear_error();
    const auto wall0 = std::chrono::steady_clock::now();
    MRS_REQUIRE(ctx != nullptr, "ctx is NULL");
    MRS_REQUIRE(n_rods >= 1 && rod_off != nullptr && rod_off[0] == 0, "bad rod offsets");
    for (int r = 0; r < n_rods; ++r)
        MRS_REQUIRE(rod_off[r + 1] - rod_off[r] >= 2 && rod_off[r + 1] - rod_off[r] <= 4096,
                    "rod %d must have 2..4096 nodes", r);
    MRS_REQUIRE(p != nullptr && p->mu > 0.0 && p->eps > 0.0 && p->L > 0.0, "bad rod parameters");
    MRS_REQUIRE(X && D, "NULL state pointer");
    MRS_REQUIRE(n_slices >= 1 && n_slices <= 64, "n_slices must be in 1..64");
    MRS_REQUIRE(group_size >= 1 && group_size <= n_slices, "group_size must be in 1..n_slices");
    MRS_REQUIRE(std::isfinite(T0) && std::isfinite(T1) && T1 > T0, "need T1 > T0");
    MRS_REQUIRE(dt_fine > 0.0 && coarse_ratio >= 1, "need dt_fine > 0 and coarse_ratio >= 1");
    MRS_REQUIRE(max_iter >= 1, "max_iter must be >= 1");
    const int Ns = n_slices;
    const double dT = (T1 - T0) / Ns;
    const long long n_fine = llround(dT / dt_fine);
    MRS_REQUIRE(n_fine >= 1 && std::fabs(n_fine * dt_fine - dT) <= 1e-9 * dT,
                "the slice length must be a whole number of fine steps");
    MRS_REQUIRE(n_fine % coarse_ratio == 0, "the slice length must be a whole number of coarse steps");
    MRS_REQUIRE(n_fine <= 0x7fffffff, "too many fine steps per slice");
    const int n_coarse = (int)(n_fine / coarse_ratio);
    const double dt_coarse = dt_fine * coarse_ratio;
    MRS_CHECK_CUDA(cudaSetDevice(ctx->device));
    const size_t N1 = (size_t)rod_off[n_rods];
    const size_t sx = 3 * N1, sd = 9 * N1;
    const int n_groups = (Ns + group_size - 1) / group_size;
    auto g_lo = [&](int j) { return j * group_size + 1; };                 // first slice of group j
    auto g_hi = [&](int j) { return std::min(Ns, (j + 1) * group_size); };  // last slice of group j
    auto group_of = [&](int n) { return (n - 1) / group_size; };

    // device buffers
    int st;
    DBuf UX, UD, GoX, GoD, FXb[2], FDb[2], WX, WD, INC;
    auto alloc = [&](DBuf& b, size_t n) -> int {
        if (cudaMalloc((void**)&b.p, n * sizeof(double)) != cudaSuccess) {
            b.p = nullptr;
            set_error("cudaMalloc of %zu bytes failed", n * sizeof(double));
            return MRS_ENOMEM;
        }
        return MRS_OK;
    };
    if ((st = alloc(UX, sx * (Ns + 1))) || (st = alloc(UD, sd * (Ns + 1))) ||
        (st = alloc(GoX, sx * (Ns + 1))) || (st = alloc(GoD, sd * (Ns + 1))) ||
        (st = alloc(FXb[0], sx * Ns)) || (st = alloc(FDb[0], sd * Ns)) ||
        (st = alloc(FXb[1], sx * Ns)) || (st = alloc(FDb[1], sd * Ns)) || (st = alloc(WX, sx)) ||
        (st = alloc(WD, sd)) || (st = alloc(INC, (size_t)max_iter)))
        return st;
    double* h_inc = nullptr;
    MRS_CHECK_CUDA(cudaHostAlloc((void**)&h_inc, sizeof(double) * max_iter, cudaHostAllocDefault));
    struct HostFree {
        double* p;
        ~HostFree() { cudaFreeHost(p); }
    } h_inc_guard{h_inc};

    // workspaces: the coarse one, and for every group every size its open part can take
    // (all created before any work is queued, so nothing below allocates or synchronizes)
    RodWorkspace* wsG = nullptr;
    if ((st = rod_ws_get(ctx, n_rods, rod_off, 1, MRS_F32_COMP, p->mu, p->eps, &wsG))) return st;
    std::vector<std::vector<RodWorkspace*>> wsF(n_groups);
    for (int j = 0; j < n_groups; ++j) {
        const int full = g_hi(j) - g_lo(j) + 1;
        wsF[j].assign(full + 1, nullptr);
        for (int m = 1; m <= full; ++m)
            if ((st = rod_ws_get(ctx, n_rods, rod_off, m, MRS_F32_COMP, p->mu, p->eps, &wsF[j][m], 1000 + j)))
                return st;
    }
    if ((int)ctx->rod_ws.size() > (int)ctx->rod_ws_max) {
        set_error("too many workspaces for this pipelined schedule");
        return MRS_EINVAL;
    }

    Streams S;
    cudaStream_t sC, caller = (cudaStream_t)stream;
    std::vector<cudaStream_t> sF(n_groups);
    std::vector<cudaEvent_t> E(Ns + 1), copied(n_groups), done(n_groups);
    cudaEvent_t start_ev, end_ev;
    MRS_CHECK_CUDA(S.stream(&sC));
    for (int j = 0; j < n_groups; ++j) {
        MRS_CHECK_CUDA(S.stream(&sF[j]));
        MRS_CHECK_CUDA(S.event(&copied[j]));
        MRS_CHECK_CUDA(S.event(&done[j]));
    }
    for (int n = 0; n <= Ns; ++n) MRS_CHECK_CUDA(S.event(&E[n]));
    MRS_CHECK_CUDA(S.event(&start_ev));
    MRS_CHECK_CUDA(S.event(&end_ev));
    MRS_CHECK_CUDA(cudaEventRecord(start_ev, caller));   // the caller's X, D are ready
    MRS_CHECK_CUDA(cudaStreamWaitEvent(sC, start_ev, 0));

    long long fine_steps = 0, coarse_steps = 0;
    auto cpy = [&](double* dst, const double* src, size_t n, cudaStream_t s) -> int {
        MRS_CHECK_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        return MRS_OK;
    };
    auto coarse = [&](int n) -> int {   // (WX, WD) over slice n on the sweep stream
        int r = rod_ws_set_times(wsG, T0 + (n - 1) * dT, 0.0, sC);
        if (r) return r;
        coarse_steps += n_coarse;
        return rod_ws_steps(wsG, p, WX.p, WD.p, dt_coarse, n_coarse, MRS_EULER, sC);
    };
    // fine solves of iteration k for every group with open slices
    auto enqueue_fine = [&](int k) -> int {
        double* FXp = FXb[k % 2].p;
        double* FDp = FDb[k % 2].p;
        for (int j = 0; j < n_groups; ++j) {
            const int lo = std::max(g_lo(j), k), hi = g_hi(j);
            if (lo > hi) continue;
            const int m = hi - lo + 1;
            cudaStream_t s = sF[j];
            MRS_CHECK_CUDA(cudaStreamWaitEvent(s, E[hi - 1], 0));   // U^{k-1}_{hi-1} produced
            int r;
            if ((r = cpy(FXp + (lo - 1) * sx, UX.p + (lo - 1) * sx, sx * m, s)) ||
                (r = cpy(FDp + (lo - 1) * sd, UD.p + (lo - 1) * sd, sd * m, s)))
                return r;
            MRS_CHECK_CUDA(cudaEventRecord(copied[j], s));
            RodWorkspace* ws = wsF[j][m];
            if ((r = rod_ws_set_times(ws, T0 + (lo - 1) * dT, dT, s))) return r;
            if ((r = rod_ws_steps(ws, p, FXp + (lo - 1) * sx, FDp + (lo - 1) * sd, dt_fine,
                                  (int)n_fine, MRS_RK2, s)))
                return r;
            MRS_CHECK_CUDA(cudaEventRecord(done[j], s));
            fine_steps += n_fine * m;
        }
        return MRS_OK;
    };

    // U[0] = x0 and the initial coarse sweep (Eq. initial), publishing every slice end
    if ((st = cpy(UX.p, X, sx, sC)) || (st = cpy(UD.p, D, sd, sC)) || (st = cpy(WX.p, X, sx, sC)) ||
        (st = cpy(WD.p, D, sd, sC)))
        return st;
    MRS_CHECK_CUDA(cudaEventRecord(E[0], sC));
    for (int n = 1; n <= Ns; ++n) {
        if ((st = coarse(n))) return st;
        if ((st = cpy(UX.p + n * sx, WX.p, sx, sC)) || (st = cpy(UD.p + n * sd, WD.p, sd, sC)) ||
            (st = cpy(GoX.p + n * sx, WX.p, sx, sC)) || (st = cpy(GoD.p + n * sd, WD.p, sd, sC)))
            return st;
        MRS_CHECK_CUDA(cudaEventRecord(E[n], sC));
    }
    if ((st = enqueue_fine(1))) return st;

    mrs_parareal_stats stats;
    std::memset(&stats, 0, sizeof(stats));
    double last = INFINITY;
    int status = MRS_OK;
    bool fine_queued = true;   // the fine solves of the next iteration are enqueued
    for (int k = 1; k <= max_iter && k <= Ns; ++k) {
        if (!fine_queued) {    // not speculated: enqueue them now (U^{k-1} is final)
            if ((st = enqueue_fine(k))) return st;
            for (int j = 0; j < n_groups; ++j)
                if (std::max(g_lo(j), k) <= g_hi(j)) MRS_CHECK_CUDA(cudaStreamWaitEvent(sC, copied[j], 0));
            fine_queued = true;
        }
        // the correction sweep of iteration k (Eq. serial_correct) on the sweep stream
        double* inc = INC.p + (k - 1);
        const double* FX = FXb[k % 2].p;
        const double* FD = FDb[k % 2].p;
        MRS_CHECK_CUDA(cudaMemsetAsync(inc, 0, sizeof(double), sC));
        MRS_CHECK_CUDA(cudaStreamWaitEvent(sC, done[group_of(k)], 0));
        MRS_CHECK_CUDA(launch_parareal_correct((int)N1, FX + (k - 1) * sx, FD + (k - 1) * sd,
                                               nullptr, nullptr, nullptr, nullptr, UX.p + k * sx,
                                               UD.p + k * sd, inc, sC));
        MRS_CHECK_CUDA(cudaEventRecord(E[k], sC));
        for (int n = k + 1; n <= Ns; ++n) {
            if ((st = cpy(WX.p, UX.p + (n - 1) * sx, sx, sC)) || (st = cpy(WD.p, UD.p + (n - 1) * sd, sd, sC)))
                return st;
            if ((st = coarse(n))) return st;
            MRS_CHECK_CUDA(cudaStreamWaitEvent(sC, done[group_of(n)], 0));
            MRS_CHECK_CUDA(launch_parareal_correct((int)N1, FX + (n - 1) * sx, FD + (n - 1) * sd,
                                                   WX.p, WD.p, GoX.p + n * sx, GoD.p + n * sd,
                                                   UX.p + n * sx, UD.p + n * sd, inc, sC));
            MRS_CHECK_CUDA(cudaEventRecord(E[n], sC));
        }
        MRS_CHECK_CUDA(cudaMemcpyAsync(h_inc + (k - 1), inc, sizeof(double), cudaMemcpyDeviceToHost, sC));
        MRS_CHECK_CUDA(cudaEventRecord(end_ev, sC));
        // speculative: the next iteration's fine solves start as the sweep publishes states.
        // The next sweep overwrites U[n] only after the group reading U[n] has copied it.
        fine_queued = false;
        bool speculate = k < max_iter && k < Ns;
        if (speculate && tol > 0.0 && k >= 2) {
            if (k == 2) {
                if (stats.incr[0] < kSpecFirst * tol) speculate = false;
            } else {
                const double a = stats.incr[k - 2], b = stats.incr[k - 3];   // eta~^{k-1}, eta~^{k-2}
                if (b > 0.0 && a < b && a * (a / b) < tol) speculate = false;
            }
        }
        if (speculate) {
            if ((st = enqueue_fine(k + 1))) return st;
            for (int j = 0; j < n_groups; ++j)
                if (std::max(g_lo(j), k + 1) <= g_hi(j)) MRS_CHECK_CUDA(cudaStreamWaitEvent(sC, copied[j], 0));
            fine_queued = true;
        }
        MRS_CHECK_CUDA(cudaEventSynchronize(end_ev));
        const double incr = h_inc[k - 1];
        stats.iterations = k;
        stats.incr[k - 1] = incr;
        last = incr;
        if (!std::isfinite(incr)) {
            status = MRS_ENOCONV;
            set_error("Parareal increment is not finite at iteration %d", k);
            break;
        }
        if (tol > 0.0 && incr < tol) break;
    }
    if (status == MRS_OK && tol > 0.0 && !(last < tol) && stats.iterations < Ns) {
        status = MRS_ENOCONV;
        set_error("Parareal did not reach tol %g in %d iterations (last increment %g)", tol,
                  stats.iterations, last);
    }
    if ((st = cpy(X, UX.p + Ns * sx, sx, sC)) || (st = cpy(D, UD.p + Ns * sd, sd, sC))) return st;
    MRS_CHECK_CUDA(cudaEventRecord(end_ev, sC));
    MRS_CHECK_CUDA(cudaStreamWaitEvent(caller, end_ev, 0));
    for (cudaStream_t s : sF) MRS_CHECK_CUDA(cudaStreamSynchronize(s));
    MRS_CHECK_CUDA(cudaStreamSynchronize(sC));
    stats.final_incr = last;
    stats.fine_steps = fine_steps;
    stats.coarse_steps = coarse_steps;
    stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - wall0).count();
    if (out) *out = stats;
    return status;
}
