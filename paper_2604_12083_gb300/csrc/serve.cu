// serve.cu -- continuous batching of pair-sum and rod-integration jobs on one GPU.
//
// A scheduler thread runs iterations on the server's stream.  Each iteration:
//   1. admits waiting jobs in submission order while a slot and pool memory for the job are
//      free (admission by device-memory footprint); an admitted job's inputs are copied into
//      the pool and, for rod jobs, its node table is set up by a kernel;
//   2. picks the jobs the iteration advances: every "small" admitted job (total pair work --
//      N^2 per stage times its stages -- below the server's big-job threshold) and the oldest
//      max_big "big" ones.  Big jobs therefore run one after another in admission order, as
//      they would one request per launch, while small jobs are batched along with them and
//      never wait behind a big one;
//   3. for every picked rod job, computes its rod forces for the current stage and packs
//      positions, forces and torques (float32) into the job's range of the point pool;
//   4. runs ONE persistent pair-sum launch over all picked jobs (each job one system of the
//      batch, its own eps and mu) -- the work of every job in flight overlaps on the GPU.  The
//      launch is the symmetric kernel (each unordered pair once, mrs_sym.cu) whenever the
//      iteration's row and column partials fit the server's scratch, else the ordered one;
//   5. velocity jobs copy their result out and finish; rod jobs apply the stage's update and
//      finish after their last step (state copied back to the caller).
// Why the split: when every admitted job advances in every iteration, a big rod job shares the
// GPU with everything that arrives during its hundreds of stages and finishes later than it
// would have alone (processor sharing), which raises the tail latency above that of one
// request per launch; serving big jobs in order and only small ones alongside keeps the tail
// at or below it while small jobs still finish in a few iterations.
// At most two iterations are in flight: the host builds iteration i+1 while the GPU runs i, and
// retires i (completion times from CUDA events, pool memory released) before building i+2.
// Pool memory of a finished job is released only after the GPU has passed its last use.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "rod_internal.h"

namespace mrs {
namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator of [0, capacity) in whole units, with coalescing on release.
class RangeAlloc {
  public:
    void init(size_t cap)
    {
        free_.clear();
        cap_ = cap;
        used_ = peak_ = 0;
        if (cap) free_[0] = cap;
    }
    bool alloc(size_t n, size_t* off)
    {
        if (n == 0) n = 1;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += n;
                if (used_ > peak_) peak_ = used_;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        if (n == 0) n = 1;
        used_ -= n;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + n == nx->first) {
            n += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += n;
                return;
            }
        }
        free_[off] = n;
    }
    size_t capacity() const { return cap_; }
    size_t peak() const { return peak_; }

  private:
    std::map<size_t, size_t> free_;
    size_t cap_ = 0, used_ = 0, peak_ = 0;
};

constexpr int kMaxRodsPerJob = 1024;
constexpr int kServeConfig = 8;             // 64 threads x 4 targets, packed f32x2 (TM = 256)
constexpr int kServeSymConfig = 25;         // symmetric, 64 threads x 6 points (TM = 384), 4 waves
constexpr int kMaxStagesPerIteration = 16;  // rod-only iterations: stages enqueued at once
constexpr double kIterPairBudget = 1.5e8;   // ... and pair interactions in all (~0.25 ms)
constexpr double kServeSymShare = 0.03;     // share of the budget for symmetric scratch ...
constexpr size_t kServeSymMax = (size_t)3 << 30;   // ... up to 3 GiB
constexpr int kMaxServeTiles = 1 << 20;     // tiles of one iteration's batched launch
constexpr size_t kByteAlign = 256;

struct RodTable {      // passed by value to the set-up kernel (kernel parameter space)
    int n_rods;
    int off[kMaxRodsPerJob + 1];
    int coff[kMaxRodsPerJob + 1];   // first chunk of kWNodes nodes of every rod
};

struct SJob {
    uint64_t ticket = 0;
    mrs_job spec;
    double work = 0.0;               // total pair interactions of the job (all its stages)
    bool big = false;                // work >= the server's big-job threshold (at admission)
    std::vector<int64_t> rod_off;
    double t_submit = 0.0, t_done = 0.0;
    int status = MRS_PENDING;
    bool finished = false;
    size_t pt_off = 0, pt_n = 0;     // point-pool range (points)
    size_t by_off = 0, by_n = 0;     // byte-pool range (bytes)
    int steps_done = 0, stage = 0;
    RodLaunch L;
    double *X = nullptr, *D = nullptr, *Xh = nullptr, *Dh = nullptr;
};

// Chunks of kWNodes nodes of a rod job (at most one partial chunk per rod).
size_t rod_chunks_bound(size_t N, int n_rods) { return N / kWNodes + (size_t)n_rods + 1; }

// Byte-pool layout of a rod job with N nodes in n_rods rods.
size_t rod_bytes(size_t N, int n_rods)
{
    auto al = [](size_t b) { return (b + kByteAlign - 1) / kByteAlign * kByteAlign; };
    return al(24 * N) + al(72 * N) + al(24 * N) + al(72 * N) + al(48 * N) + al(8 * N) +
           al(sizeof(int4) * rod_chunks_bound(N, n_rods)) + 2 * kByteAlign;
}

}  // namespace

__global__ void serve_rod_setup_kernel(int2* node_info, int4* wchunks, double* t0, long long* step,
                                       int N, double t_start, const RodTable tab)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        *t0 = t_start;
        *step = 0;
    }
    if (k >= N) return;
    int lo = 0, hi = tab.n_rods - 1;   // rod containing node k
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab.off[mid] <= k) lo = mid; else hi = mid - 1;
    }
    const int idx = k - tab.off[lo], M = tab.off[lo + 1] - tab.off[lo];
    node_info[k] = make_int2(idx, M);
    // the warp-cooperative force kernel's chunk table: (base node, rod nodes, index, instance)
    if (idx % kWNodes == 0) wchunks[tab.coff[lo] + idx / kWNodes] = make_int4(k, M, idx, 0);
}

}  // namespace mrs

using namespace mrs;

struct mrs_server {
    mrs_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    int max_slots = 0;
    // pools
    char* d_bytes = nullptr;
    RangeAlloc bytes;
    float *pX = nullptr, *pf = nullptr, *pn = nullptr, *pu = nullptr, *pw = nullptr;
    RangeAlloc pts;
    // batched pair-sum tables
    int config = 0, TM = 0, P = 0, tile_cap = 0, sys_cap = 0;
    long long tiles_in_use = 0;
    TileDesc* d_tiles = nullptr;
    SysConst* d_sc = nullptr;
    float* d_partial = nullptr;
    int* d_counters = nullptr;
    // symmetric launch: work table and row / column partials (capacities in floats)
    int sym_config = 0, sTM = 0, sP = 0;
    SymTile* d_stiles = nullptr;
    float* d_rowpart = nullptr;
    float* d_colpart = nullptr;
    size_t rowpart_cap = 0, colpart_cap = 0;
    int64_t sym_iterations = 0;
    // single-system iterations take the library's default configuration for that one system
    // (as mrs_velocity would): resident CTAs per SM of every ordered configuration, and clusters
    // of cl CTAs resident at once for the cluster configurations (0: none)
    int occ_cfg[64] = {};
    int cl_fit[64][17] = {};
    size_t partial_cap = 0;   // floats of d_partial
    struct Stage {
        TileDesc* tiles = nullptr;
        SymTile* stiles = nullptr;
        SysConst* sc = nullptr;
        cudaEvent_t used = nullptr;
    } stage[3];
    int stage_idx = 0;
    // jobs
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<SJob*> waiting;
    std::vector<SJob*> active;
    double big_pairs = 1.3e10;       // big-job threshold (pair interactions; <= 0: none big)
    int max_big = 1;                 // big jobs advanced per iteration
    uint64_t fail_ticket = 0;        // test hook: the admission of this ticket fails (ENOMEM)
    std::unordered_map<uint64_t, SJob*> jobs;
    uint64_t next_ticket = 1;
    int64_t submitted = 0, completed = 0, iterations = 0;
    double pairs = 0.0;
    int peak_active = 0;
    bool stop = false;
    int fatal = MRS_OK;
    char fatal_msg[512] = "";
    std::thread th;
    struct Iter {
        cudaEvent_t end;
        std::vector<SJob*> finishing;
    };
    std::deque<Iter> inflight;
    cudaEvent_t ref_ev = nullptr;
    double t_ref = 0.0;
};

namespace {

void fail_all(mrs_server* S, int status, const char* what, cudaError_t e)
{
    std::lock_guard<std::mutex> g(S->mu);
    S->fatal = status;
    snprintf(S->fatal_msg, sizeof(S->fatal_msg), "serving: %s failed: %s", what, cudaGetErrorString(e));
    set_error("%s", S->fatal_msg);
    for (auto& kv : S->jobs) {
        SJob* j = kv.second;
        if (!j->finished) {
            j->finished = true;
            j->status = status;
            j->t_done = now_s();
        }
    }
    S->waiting.clear();
    S->active.clear();
    S->cv_done.notify_all();
}

// Reserve pool memory for a job; false if it does not fit now.
bool reserve(mrs_server* S, SJob* j)
{
    const size_t N = (size_t)j->spec.n_points;
    const long long tiles = ((long long)N + S->TM - 1) / S->TM;
    if (S->tiles_in_use + tiles > S->tile_cap) return false;
    size_t po = 0, bo = 0;
    if (!S->pts.alloc(N, &po)) return false;
    if (j->spec.kind == MRS_JOB_ROD) {
        const size_t nb = rod_bytes(N, j->spec.n_rods) / kByteAlign;
        if (!S->bytes.alloc(nb, &bo)) {
            S->pts.release(po, N);
            return false;
        }
        j->by_off = bo * kByteAlign;
        j->by_n = nb;
    }
    j->pt_off = po;
    j->pt_n = N;
    S->tiles_in_use += tiles;
    return true;
}

void release(mrs_server* S, SJob* j)
{
    S->tiles_in_use -= ((long long)j->pt_n + S->TM - 1) / S->TM;
    S->pts.release(j->pt_off, j->pt_n);
    if (j->by_n) S->bytes.release(j->by_off / kByteAlign, j->by_n);
}

// Enqueue the copy-in / set-up of a newly admitted job on the server stream.
cudaError_t admit_enqueue(mrs_server* S, SJob* j)
{
    const size_t N = (size_t)j->spec.n_points;
    const mrs_job& J = j->spec;
    cudaStream_t s = S->stream;
    cudaError_t e;
    if (J.kind == MRS_JOB_VELOCITY) {
        if ((e = cudaMemcpyAsync(S->pX + 3 * j->pt_off, J.X, 12 * N, cudaMemcpyDeviceToDevice, s))) return e;
        if ((e = cudaMemcpyAsync(S->pf + 3 * j->pt_off, J.f, 12 * N, cudaMemcpyDeviceToDevice, s))) return e;
        return cudaMemcpyAsync(S->pn + 3 * j->pt_off, J.n, 12 * N, cudaMemcpyDeviceToDevice, s);
    }
    auto al = [](size_t b) { return (b + kByteAlign - 1) / kByteAlign * kByteAlign; };
    char* base = S->d_bytes + j->by_off;
    j->X = (double*)base;
    base += al(24 * N);
    j->D = (double*)base;
    base += al(72 * N);
    j->Xh = (double*)base;
    base += al(24 * N);
    j->Dh = (double*)base;
    base += al(72 * N);
    double* FN = (double*)base;
    base += al(48 * N);
    int2* info = (int2*)base;
    base += al(8 * N);
    int4* wch = (int4*)base;
    base += al(sizeof(int4) * rod_chunks_bound(N, J.n_rods));
    double* t0 = (double*)base;
    long long* step = (long long*)(base + kByteAlign);
    if ((e = cudaMemcpyAsync(j->X, J.Xr, 24 * N, cudaMemcpyDeviceToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(j->D, J.Dr, 72 * N, cudaMemcpyDeviceToDevice, s))) return e;
    RodTable tab;
    tab.n_rods = J.n_rods;
    tab.coff[0] = 0;
    for (int r = 0; r <= J.n_rods; ++r) tab.off[r] = (int)j->rod_off[r];
    for (int r = 0; r < J.n_rods; ++r) tab.coff[r + 1] = tab.coff[r] + (tab.off[r + 1] - tab.off[r] + kWNodes - 1) / kWNodes;
    serve_rod_setup_kernel<<<(int)((N + 127) / 128), 128, 0, s>>>(info, wch, t0, step, (int)N, J.t0, tab);
    if ((e = cudaGetLastError())) return e;
    RodLaunch& L = j->L;
    L.N = (int)N;
    L.nodes_per_inst = (int)N;
    L.node_info = info;
    L.t0 = t0;
    L.step = step;
    L.dt = J.dt;
    L.p = J.params;
    L.p.lj_sigma = lj_sigma_of(J.params);
    L.FN = FN;
    L.chunks = nullptr;   // no thread-per-segment chunk table in the pool: two-kernel force path
    L.n_chunks = 0;
    // small jobs: the warp-cooperative force and update kernels (the context's setting)
    const int fk = S->ctx->rod_force_kernel;
    const bool warp = fk == 2 || (fk == 0 && N <= (size_t)kWarpForceMaxNodes);
    L.wchunks = warp ? wch : nullptr;
    L.n_wchunks = tab.coff[J.n_rods];
    L.inv_L = 1.0 / J.params.L;
    set_pack_reference(L, J.n_rods, j->rod_off.data());
    L.segsc = nullptr;    // two-kernel force path: sin(k_w s_mid + f t) per segment
    L.err = S->ctx->d_err;
    return cudaSuccess;
}

// Build and enqueue one iteration over the admitted jobs; returns the jobs that finish in it.
cudaError_t run_iteration(mrs_server* S, std::vector<SJob*>& finishing)
{
    cudaStream_t s = S->stream;
    cudaError_t e;
    // the jobs this iteration advances: every small job and the oldest max_big big ones
    std::vector<SJob*> run;
    run.reserve(S->active.size());
    {
        int nbig = 0;
        for (SJob* j : S->active) {
            if (!j->big) {
                run.push_back(j);
            } else if (nbig < S->max_big) {
                run.push_back(j);
                ++nbig;
            }
        }
    }
    // stages this iteration: several when every job it advances is a rod job and none is
    // waiting for admission, so that small rod jobs do not pay one iteration's host work per
    // stage; bounded by the jobs' remaining stages (none finishes before the last) and by
    // kIterPairBudget pair interactions in all (a later arrival waits at most that long)
    int stages = 1;
    {
        bool rods_only = !run.empty();
        long long rem = kMaxStagesPerIteration;
        double stage_pairs = 0.0;
        for (SJob* j : run) {
            if (j->spec.kind != MRS_JOB_ROD) {
                rods_only = false;
                break;
            }
            const int per = j->spec.scheme == MRS_RK2 ? 2 : 1;
            rem = std::min<long long>(rem, (long long)j->spec.nsteps * per - ((long long)j->steps_done * per + j->stage));
            stage_pairs += (double)j->spec.n_points * (double)j->spec.n_points;
        }
        bool queue_empty;
        {
            std::lock_guard<std::mutex> g(S->mu);
            queue_empty = S->waiting.empty();
        }
        if (rods_only && queue_empty && stage_pairs > 0.0) {
            const double fit = std::floor(kIterPairBudget / stage_pairs);
            stages = (int)std::max<double>(1.0, std::min<double>((double)rem, fit));
        }
    }
    // rod forces of the current stage, packed into each job's point range
    auto enqueue_forces = [&]() -> cudaError_t {
        for (SJob* j : run) {
            if (j->spec.kind != MRS_JOB_ROD) continue;
            const bool half = j->spec.scheme == MRS_RK2 && j->stage == 1;
            const size_t o = 3 * j->pt_off;
            e = launch_rod_forces(j->L, half ? j->Xh : j->X, half ? j->Dh : j->D,
                                  half ? 0.5 * j->spec.dt : 0.0, nullptr, nullptr, S->pX + o, S->pf + o,
                                  S->pn + o, s);
            if (e) return e;
        }
        return cudaSuccess;
    };
    if ((e = enqueue_forces())) return e;
    // work table of the batched pair sum
    mrs_server::Stage& st = S->stage[S->stage_idx];
    S->stage_idx = (S->stage_idx + 1) % 3;
    if ((e = cudaEventSynchronize(st.used))) return e;   // the staging buffer is free again
    const int n_sys = (int)run.size();
    double pairs = 0.0;
    for (int q = 0; q < n_sys; ++q) {
        SJob* j = run[q];
        const double e2 = j->spec.eps * j->spec.eps;
        SysConst& c = st.sc[q];
        c.e2 = (float)e2;
        c.c1 = (float)(1.5 * e2);
        c.c2 = (float)(3.75 * e2 * e2);
        c.c3 = (float)(-0.75 * e2);
        c.c5 = (float)(3.75 * e2);
        c.scale = (float)(1.0 / (8.0 * M_PI * j->spec.mu));
        pairs += (double)j->spec.n_points * (double)j->spec.n_points;
    }
    // symmetric work table (see SymTile), used when its partials fit the scratch
    int snt = 0;
    long long sW = 0;
    for (int q = 0; q < n_sys; ++q) {
        SJob* j = run[q];
        const long long N = j->spec.n_points;
        const int tfirst = snt;
        for (long long t = 0, k = 0; t < N; t += S->sTM, ++k) {
            SymTile& T = st.stiles[snt++];
            T = SymTile{};
            T.sys = q;
            T.t0 = (int)(j->pt_off + t);
            T.tn = (int)std::min<long long>(S->sTM, N - t);
            T.send = (int)(j->pt_off + N);
            T.nu = (int)((N - t + kUnitSources - 1) / kUnitSources);
            T.nd = (T.tn + kUnitSources - 1) / kUnitSources;
            T.kt = (int)k;
            T.tfirst = tfirst;
            T.u0 = sW;
            sW += T.nu;
        }
    }
    const int sP = (int)std::min<long long>(S->sP, sW);
    long long nseg = 0;
    for (int i = 0; i < snt; ++i) {
        SymTile& T = st.stiles[i];
        T.qlo = cta_of_unit_host(sW, sP, T.u0);
        T.nseg = cta_of_unit_host(sW, sP, T.u0 + T.nu - 1) - T.qlo + 1;
        T.seg0 = (int)nseg;
        nseg += T.nseg;
    }
    // one system: the configuration a plan for it would choose (cluster kernel, ordered
    // persistent kernel or symmetric kernel), when the server's buffers hold its tables
    int ocfg = S->config, oTM = S->TM, ocl = 0;
    long long oP = -1;
    if (n_sys == 1) {
        const long long N = run[0]->spec.n_points;
        const int64_t off[2] = {0, N};
        const int c = default_config(S->ctx, 1, off, MRS_F32_COMP);
        const KernelConfig kc = kConfigs[c];
        if (!kc.sym && c < 64 && S->occ_cfg[c] > 0) {
            const int TMc = tile_targets(kc);
            const long long ntc = (N + TMc - 1) / TMc, nu = (N + kUnitSources - 1) / kUnitSources;
            if (kc.cluster) {
                int cl = (int)std::min<long long>(kc.cluster, nu);
                while (cl > 1 && S->cl_fit[c][cl] < ntc) --cl;
                if (ntc <= S->tile_cap && S->cl_fit[c][cl] > 0) {
                    ocfg = c;
                    oTM = TMc;
                    ocl = cl;
                    oP = ntc * cl;
                }
            } else {
                const long long full = (long long)S->ctx->num_sms * S->occ_cfg[c] * std::max(1, kc.over);
                const long long Wc = ntc * nu;
                const long long P = balanced_ctas(ordered_ctas(full, Wc, nu), full, Wc, S->ctx->num_sms,
                                                  kc.threads);
                if (ntc <= S->tile_cap && (size_t)2 * P * 6 * TMc <= S->partial_cap) {
                    ocfg = c;
                    oTM = TMc;
                    oP = P;
                }
            }
        }
    }
    const bool sym = oP < 0 && (size_t)sW * kUnitSources * 6 <= S->colpart_cap &&
                     (size_t)nseg * S->sTM * 6 <= S->rowpart_cap;
    int nt = 0;
    long long W = 0, max_nu = 0;
    if (!sym) {
        for (int q = 0; q < n_sys; ++q) {
            SJob* j = run[q];
            const long long N = j->spec.n_points;
            const int nu = (int)((N + kUnitSources - 1) / kUnitSources);
            for (long long t = 0; t < N; t += oTM) {
                TileDesc& T = st.tiles[nt++];
                T.sys = q;
                T.t0 = (int)(j->pt_off + t);
                T.tn = (int)std::min<long long>(oTM, N - t);
                T.s0 = (int)j->pt_off;
                T.sn = (int)N;
                T.nu = nu;
                T.u0 = W;
                W += nu;
                max_nu = std::max<long long>(max_nu, nu);
            }
        }
        if ((e = cudaMemcpyAsync(S->d_tiles, st.tiles, nt * sizeof(TileDesc), cudaMemcpyHostToDevice, s))) return e;
    } else {
        if ((e = cudaMemcpyAsync(S->d_stiles, st.stiles, snt * sizeof(SymTile), cudaMemcpyHostToDevice, s))) return e;
    }
    if ((e = cudaMemcpyAsync(S->d_sc, st.sc, n_sys * sizeof(SysConst), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaEventRecord(st.used, s))) return e;
    // the batched pair sum of the iteration's tables
    auto enqueue_pair = [&]() -> cudaError_t {
        if (sym) {
            SymLaunch L;
            L.tiles = S->d_stiles;
            L.n_tiles = snt;
            L.TM = S->sTM;
            L.W = sW;
            L.P = sP;
            L.U0 = 0;                 // one pass over every tile of the iteration
            L.ta = 0;
            L.tb = snt;
            L.tc = snt;
            L.acc = nullptr;
            L.n_points = (long long)S->pts.capacity();
            L.col_units = (long long)(S->colpart_cap / (kUnitSources * 6));
            L.row_segs = (long long)(S->rowpart_cap / ((size_t)S->sTM * 6));
            L.sc = S->d_sc;
            L.X = S->pX;
            L.f = S->pf;
            L.n = S->pn;
            L.u = S->pu;
            L.w = S->pw;
            L.rowpart = S->d_rowpart;
            L.colpart = S->d_colpart;
            L.err = S->ctx->d_err;
            if ((e = launch_mrs_sym(S->sym_config, true, L, s))) return e;
        } else {
            MrsLaunch L;
            L.tiles = S->d_tiles;
            L.n_tiles = nt;
            L.W = W;
            L.P = (int)ordered_ctas(S->P, W, max_nu);
            L.sc = S->d_sc;
            L.X = S->pX;
            L.f = S->pf;
            L.n = S->pn;
            L.Xt = S->pX;
            L.u = S->pu;
            L.w = S->pw;
            L.partial = S->d_partial;
            L.counters = S->d_counters;
            L.err = S->ctx->d_err;
            L.n_points = (long long)S->pts.capacity();
            if (oP >= 0) {   // the one system's own configuration
                L.P = (int)oP;
                L.cl = ocl;
            }
            if ((e = launch_mrs_f32(ocfg, true, L, s))) return e;
        }
        return cudaSuccess;
    };
    // stage updates and copy-out
    auto enqueue_updates = [&]() -> cudaError_t {
        for (SJob* j : run) {
            const size_t N = (size_t)j->spec.n_points, o = 3 * j->pt_off;
            bool done = false;
            if (j->spec.kind == MRS_JOB_VELOCITY) {
                if ((e = cudaMemcpyAsync(j->spec.u, S->pu + o, 12 * N, cudaMemcpyDeviceToDevice, s))) return e;
                if ((e = cudaMemcpyAsync(j->spec.w, S->pw + o, 12 * N, cudaMemcpyDeviceToDevice, s))) return e;
                done = true;
            } else {
                const double dt = j->spec.dt;
                if (j->spec.scheme == MRS_RK2 && j->stage == 0) {
                    e = launch_rod_update(j->L, j->X, j->D, S->pu + o, S->pw + o, 0.5 * dt, j->Xh, j->Dh, false, s);
                    j->stage = 1;
                } else {
                    e = launch_rod_update(j->L, j->X, j->D, S->pu + o, S->pw + o, dt, j->X, j->D, true, s);
                    j->stage = 0;
                    j->steps_done += 1;
                }
                if (e) return e;
                if (j->steps_done == j->spec.nsteps) {
                    if ((e = cudaMemcpyAsync(j->spec.Xr, j->X, 24 * N, cudaMemcpyDeviceToDevice, s))) return e;
                    if ((e = cudaMemcpyAsync(j->spec.Dr, j->D, 72 * N, cudaMemcpyDeviceToDevice, s))) return e;
                    done = true;
                }
            }
            if (done) finishing.push_back(j);
        }
        return cudaSuccess;
    };
    for (int k = 0; k < stages; ++k) {
        if (k > 0 && (e = enqueue_forces())) return e;
        if ((e = enqueue_pair())) return e;
        if ((e = enqueue_updates())) return e;
    }
    if (!finishing.empty()) {
        std::vector<SJob*> keep;
        keep.reserve(S->active.size());
        for (SJob* j : S->active)
            if (std::find(finishing.begin(), finishing.end(), j) == finishing.end()) keep.push_back(j);
        S->active.swap(keep);
    }
    std::lock_guard<std::mutex> g(S->mu);
    S->iterations += 1;
    S->sym_iterations += sym ? 1 : 0;
    S->pairs += pairs * stages;
    return cudaSuccess;
}

cudaError_t retire_oldest(mrs_server* S)
{
    mrs_server::Iter it = S->inflight.front();
    S->inflight.pop_front();
    cudaError_t e = cudaEventSynchronize(it.end);
    if (e) return e;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, S->ref_ev, it.end);
    const double t_done = S->t_ref + 1e-3 * ms;
    cudaEventDestroy(it.end);
    std::lock_guard<std::mutex> g(S->mu);
    for (SJob* j : it.finishing) {
        release(S, j);
        j->t_done = t_done;
        j->status = MRS_OK;
        j->finished = true;
        S->completed += 1;
    }
    S->cv_done.notify_all();
    S->cv.notify_all();
    return cudaSuccess;
}

void scheduler(mrs_server* S)
{
    cudaSetDevice(S->ctx->device);
    for (;;) {
        std::vector<SJob*> admitted;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            while (!S->stop && S->waiting.empty() && S->active.empty() && S->inflight.empty())
                S->cv.wait_for(lk, std::chrono::milliseconds(50));
            if (S->fatal) return;
            if (S->stop && S->waiting.empty() && S->active.empty() && S->inflight.empty()) return;
            // admission: submission order, while a slot and the job's footprint are free
            while (!S->waiting.empty() && (int)S->active.size() < S->max_slots) {
                SJob* j = S->waiting.front();
                if (j->ticket == S->fail_ticket) {
                    // injected allocation failure: the job ends with MRS_ENOMEM, untouched
                    S->fail_ticket = 0;
                    S->waiting.pop_front();
                    j->finished = true;
                    j->status = MRS_ENOMEM;
                    j->t_done = now_s();
                    S->completed += 1;
                    S->cv_done.notify_all();
                    continue;
                }
                if (!reserve(S, j)) break;
                S->waiting.pop_front();
                j->big = S->big_pairs > 0.0 && j->work >= S->big_pairs;
                S->active.push_back(j);
                admitted.push_back(j);
            }
            if ((int)S->active.size() > S->peak_active) S->peak_active = (int)S->active.size();
        }
        cudaError_t e = cudaSuccess;
        for (SJob* j : admitted)
            if (!e) e = admit_enqueue(S, j);
        if (e) return fail_all(S, MRS_ECUDA, "job admission", e);
        if (!S->active.empty()) {
            std::vector<SJob*> fin;
            e = run_iteration(S, fin);
            if (e) return fail_all(S, MRS_ECUDA, "iteration", e);
            mrs_server::Iter it;
            e = cudaEventCreate(&it.end);
            if (!e) e = cudaEventRecord(it.end, S->stream);
            if (e) return fail_all(S, MRS_ECUDA, "event record", e);
            it.finishing = fin;
            S->inflight.push_back(it);
        }
        // keep at most one iteration queued behind the running one
        while (S->inflight.size() > (S->active.empty() ? 0u : 1u)) {
            e = retire_oldest(S);
            if (e) return fail_all(S, MRS_ECUDA, "iteration completion", e);
        }
    }
}

template <typename T>
int dalloc(T** p, size_t n)
{
    cudaError_t e = cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("serving pool allocation of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
        return MRS_ENOMEM;
    }
    return MRS_OK;
}

void server_free(mrs_server* S)
{
    cudaFree(S->d_bytes);
    cudaFree(S->pX);
    cudaFree(S->pf);
    cudaFree(S->pn);
    cudaFree(S->pu);
    cudaFree(S->pw);
    cudaFree(S->d_tiles);
    cudaFree(S->d_sc);
    cudaFree(S->d_partial);
    cudaFree(S->d_counters);
    cudaFree(S->d_stiles);
    cudaFree(S->d_rowpart);
    cudaFree(S->d_colpart);
    for (auto& st : S->stage) {
        cudaFreeHost(st.tiles);
        cudaFreeHost(st.stiles);
        cudaFreeHost(st.sc);
        if (st.used) cudaEventDestroy(st.used);
    }
    if (S->ref_ev) cudaEventDestroy(S->ref_ev);
    if (S->stream) cudaStreamDestroy(S->stream);
    for (auto& kv : S->jobs) delete kv.second;
    delete S;
}

}  // namespace

extern "C" {

int serve_create(mrs_server** srv, mrs_ctx* ctx, size_t hbm_budget_bytes, int max_slots)
{
    clear_error();
    MRS_REQUIRE(srv != nullptr && ctx != nullptr, "NULL argument");
    MRS_REQUIRE(max_slots >= 1 && max_slots <= 4096, "max_slots must be in 1..4096");
    MRS_REQUIRE(hbm_budget_bytes >= ((size_t)1 << 20), "hbm_budget_bytes must be at least 1 MiB");
    *srv = nullptr;
    MRS_CHECK_CUDA(cudaSetDevice(ctx->device));
    // point indices of the batched launch are 32-bit: the point pool (27 % of the budget at 60 B
    // per point) must stay below 2^31 points
    MRS_REQUIRE((double)hbm_budget_bytes * 0.27 / 60.0 < (double)((1u << 31) - (1u << 24)),
                "hbm_budget_bytes too large (%zu)", hbm_budget_bytes);
    mrs_server* S = new mrs_server();
    S->ctx = ctx;
    S->max_slots = max_slots;
    // pools: 27 % of the budget as point slots (5 float32 [.][3] arrays, 60 B per point),
    // 70 % as bytes for rod state (~248 B per node), 3 % (at most 3 GiB) as scratch of the
    // symmetric launch (two thirds column partials, one third row partials)
    const size_t pt_cap = (size_t)(0.27 * (double)hbm_budget_bytes) / 60;
    const size_t by_cap = (size_t)(0.70 * (double)hbm_budget_bytes) / kByteAlign;
    const size_t sym_bytes = std::min<size_t>((size_t)(kServeSymShare * (double)hbm_budget_bytes), kServeSymMax);
    S->config = kServeConfig;
    S->TM = kConfigs[S->config].threads * kConfigs[S->config].tpt;
    int occ = 0, st;
    if (occupancy_f32(S->config, true, &occ) != MRS_OK || occ < 1) {
        delete S;
        set_error("occupancy query failed");
        return MRS_ECUDA;
    }
    S->P = ctx->num_sms * occ;
    S->sym_config = kServeSymConfig;
    S->sTM = kConfigs[S->sym_config].threads * kConfigs[S->sym_config].tpt;
    if (occupancy_sym(S->sym_config, true, &occ) != MRS_OK || occ < 1) {
        delete S;
        set_error("occupancy query failed");
        return MRS_ECUDA;
    }
    S->sP = ctx->num_sms * occ * std::max(1, kConfigs[S->sym_config].over);
    for (int c = 0; c < kNumConfigs && c < 64; ++c) {
        if (kConfigs[c].sym) continue;
        int oc = 0;
        if (occupancy_f32(c, true, &oc) != MRS_OK) {
            cudaGetLastError();
            oc = 0;
        }
        S->occ_cfg[c] = oc;
        if (kConfigs[c].cluster && oc > 0)
            for (int cl = 1; cl <= 16 && cl <= kConfigs[c].cluster; ++cl) {
                int mc = 0;
                if (cluster_setup_f32(c, true, cl, &mc) != MRS_OK) {
                    cudaGetLastError();   // a refused cluster shape: that size is not used
                    mc = 0;
                }
                S->cl_fit[c][cl] = mc;
            }
    }
    S->colpart_cap = sym_bytes / 3 * 2 / sizeof(float);
    S->rowpart_cap = sym_bytes / 3 / sizeof(float);
    // tiles of the symmetric table (TM = sTM >= TM) never outnumber the ordered ones
    S->tile_cap = (int)std::min<size_t>(pt_cap / S->TM + max_slots + 1, (size_t)kMaxServeTiles);
    S->sys_cap = max_slots;
    if ((st = dalloc(&S->pX, 3 * pt_cap)) || (st = dalloc(&S->pf, 3 * pt_cap)) ||
        (st = dalloc(&S->pn, 3 * pt_cap)) || (st = dalloc(&S->pu, 3 * pt_cap)) ||
        (st = dalloc(&S->pw, 3 * pt_cap)) || (st = dalloc(&S->d_bytes, by_cap * kByteAlign)) ||
        (st = dalloc(&S->d_tiles, (size_t)S->tile_cap)) || (st = dalloc(&S->d_sc, (size_t)S->sys_cap)) ||
        (st = dalloc(&S->d_partial, S->partial_cap = (size_t)2 * S->P * 6 * S->TM)) ||
        (st = dalloc(&S->d_counters, (size_t)S->tile_cap)) ||
        (st = dalloc(&S->d_stiles, (size_t)S->tile_cap)) ||
        (st = dalloc(&S->d_rowpart, S->rowpart_cap)) || (st = dalloc(&S->d_colpart, S->colpart_cap))) {
        server_free(S);
        return st;
    }
    S->pts.init(pt_cap);
    S->bytes.init(by_cap);
    cudaError_t e = cudaMemset(S->d_counters, 0, sizeof(int) * (size_t)S->tile_cap);
    for (auto& sg : S->stage) {
        if (!e) e = cudaHostAlloc((void**)&sg.tiles, sizeof(TileDesc) * (size_t)S->tile_cap, cudaHostAllocDefault);
        if (!e) e = cudaHostAlloc((void**)&sg.stiles, sizeof(SymTile) * (size_t)S->tile_cap, cudaHostAllocDefault);
        if (!e) e = cudaHostAlloc((void**)&sg.sc, sizeof(SysConst) * (size_t)S->sys_cap, cudaHostAllocDefault);
        if (!e) e = cudaEventCreateWithFlags(&sg.used, cudaEventDisableTiming);
        if (!e) e = cudaEventRecord(sg.used, 0);
    }
    if (!e) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreate(&S->ref_ev);
    if (!e) e = cudaEventRecord(S->ref_ev, S->stream);
    if (!e) e = cudaEventSynchronize(S->ref_ev);
    if (!e) e = cudaDeviceSynchronize();
    if (e) {
        server_free(S);
        set_error("serving set-up failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    S->t_ref = now_s();
    S->th = std::thread(scheduler, S);
    *srv = S;
    return MRS_OK;
}

int serve_submit(mrs_server* S, const mrs_job* job, uint64_t* ticket)
{
    clear_error();
    MRS_REQUIRE(S != nullptr && job != nullptr && ticket != nullptr, "NULL argument");
    const mrs_job& J = *job;
    MRS_REQUIRE(J.kind == MRS_JOB_VELOCITY || J.kind == MRS_JOB_ROD, "unknown job kind %d", J.kind);
    MRS_REQUIRE(J.n_points >= 1 && J.n_points < (1LL << 28), "n_points out of range");
    MRS_REQUIRE(std::isfinite(J.mu) && J.mu > 0.0 && std::isfinite(J.eps) && J.eps > 0.0,
                "mu and eps must be > 0");
    SJob* j = new SJob();
    j->spec = J;
    if (J.kind == MRS_JOB_VELOCITY) {
        if (!(J.X && J.f && J.n && J.u && J.w)) {
            delete j;
            MRS_REQUIRE(false, "NULL buffer in velocity job");
        }
    } else {
        const bool ok = J.Xr && J.Dr && J.rod_off && J.n_rods >= 1 && J.n_rods <= kMaxRodsPerJob &&
                        J.rod_off[0] == 0 && J.rod_off[J.n_rods] == J.n_points && J.nsteps >= 1 &&
                        std::isfinite(J.dt) && J.dt > 0.0 && std::isfinite(J.t0) &&
                        (J.scheme == MRS_EULER || J.scheme == MRS_RK2);
        bool rods_ok = ok;
        for (int r = 0; rods_ok && r < J.n_rods; ++r) {
            const int64_t M = J.rod_off[r + 1] - J.rod_off[r];
            rods_ok = M >= 2 && M <= 4096;
        }
        if (!rods_ok) {
            delete j;
            MRS_REQUIRE(false, "invalid rod job (buffers, 1..%d rods of 2..4096 nodes, rod_off[n_rods] == "
                        "n_points, nsteps >= 1, dt > 0, scheme)", kMaxRodsPerJob);
        }
        j->rod_off.assign(J.rod_off, J.rod_off + J.n_rods + 1);
        j->spec.rod_off = nullptr;
    }
    const size_t N = (size_t)J.n_points;
    if (N > S->pts.capacity() || (long long)((N + S->TM - 1) / S->TM) > S->tile_cap ||
        (J.kind == MRS_JOB_ROD && rod_bytes(N, J.n_rods) / kByteAlign > S->bytes.capacity())) {
        delete j;
        set_error("job of %zu points does not fit the serving pool", N);
        return MRS_EBUSY;
    }
    std::lock_guard<std::mutex> g(S->mu);
    if (S->fatal) {
        delete j;
        set_error("server stopped after an error");
        return S->fatal;
    }
    j->work = (double)N * (double)N *
              (J.kind == MRS_JOB_ROD ? (double)J.nsteps * (J.scheme == MRS_RK2 ? 2.0 : 1.0) : 1.0);
    j->ticket = S->next_ticket++;
    j->t_submit = now_s();
    S->jobs[j->ticket] = j;
    S->waiting.push_back(j);
    S->submitted += 1;
    *ticket = j->ticket;
    S->cv.notify_all();
    return MRS_OK;
}

int serve_poll(mrs_server* S, uint64_t ticket, int* done, double* latency_s)
{
    clear_error();
    MRS_REQUIRE(S != nullptr, "NULL server");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->jobs.find(ticket);
    MRS_REQUIRE(it != S->jobs.end(), "unknown ticket %llu", (unsigned long long)ticket);
    SJob* j = it->second;
    if (done) *done = j->finished ? 1 : 0;
    if (!j->finished) return MRS_PENDING;
    if (latency_s) *latency_s = j->t_done - j->t_submit;
    if (j->status == MRS_ECANCELED) set_error("job %llu was cancelled", (unsigned long long)ticket);
    else if (j->status == MRS_ENOMEM && !S->fatal)
        set_error("job %llu: pool allocation failed at admission", (unsigned long long)ticket);
    else if (j->status != MRS_OK) set_error("%s", S->fatal_msg);
    return j->status;
}

int serve_cancel(mrs_server* S, uint64_t ticket)
{
    clear_error();
    MRS_REQUIRE(S != nullptr, "NULL server");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->jobs.find(ticket);
    MRS_REQUIRE(it != S->jobs.end(), "unknown ticket %llu", (unsigned long long)ticket);
    SJob* j = it->second;
    for (auto w = S->waiting.begin(); w != S->waiting.end(); ++w) {
        if (*w == j) {
            S->waiting.erase(w);
            j->finished = true;
            j->status = MRS_ECANCELED;
            j->t_done = now_s();
            S->completed += 1;
            S->cv_done.notify_all();
            return MRS_OK;
        }
    }
    if (j->finished) {
        set_error("job %llu has already finished", (unsigned long long)ticket);
        return MRS_EINVAL;
    }
    set_error("job %llu is already running and cannot be cancelled", (unsigned long long)ticket);
    return MRS_EBUSY;
}

int serve_drain(mrs_server* S, double timeout_s)
{
    clear_error();
    MRS_REQUIRE(S != nullptr, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (S->completed < S->submitted && !S->fatal) {
        if (S->cv_done.wait_until(lk, until) == std::cv_status::timeout && S->completed < S->submitted) {
            set_error("serve_drain timed out with %lld of %lld jobs done", (long long)S->completed,
                      (long long)S->submitted);
            return MRS_ETIMEOUT;
        }
    }
    return S->fatal ? S->fatal : MRS_OK;
}

int serve_stats(mrs_server* S, int64_t* iterations, int64_t* completed, double* pairs,
                int* peak_active, size_t* peak_pool_bytes, int64_t* symmetric_iterations)
{
    clear_error();
    MRS_REQUIRE(S != nullptr, "NULL server");
    std::lock_guard<std::mutex> g(S->mu);
    if (iterations) *iterations = S->iterations;
    if (completed) *completed = S->completed;
    if (pairs) *pairs = S->pairs;
    if (peak_active) *peak_active = S->peak_active;
    if (peak_pool_bytes) *peak_pool_bytes = S->pts.peak() * 60 + S->bytes.peak() * kByteAlign;
    if (symmetric_iterations) *symmetric_iterations = S->sym_iterations;
    return MRS_OK;
}

int serve_set_policy(mrs_server* S, double big_job_pairs, int max_big_jobs)
{
    clear_error();
    MRS_REQUIRE(S != nullptr, "NULL server");
    MRS_REQUIRE(std::isfinite(big_job_pairs), "big_job_pairs must be finite");
    MRS_REQUIRE(max_big_jobs >= 1 && max_big_jobs <= 4096, "max_big_jobs must be in 1..4096");
    std::lock_guard<std::mutex> g(S->mu);
    S->big_pairs = big_job_pairs;
    S->max_big = max_big_jobs;
    return MRS_OK;
}

int serve_inject_alloc_failure(mrs_server* S, uint64_t ticket)
{
    clear_error();
    MRS_REQUIRE(S != nullptr, "NULL server");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->jobs.find(ticket);
    MRS_REQUIRE(it != S->jobs.end(), "unknown ticket %llu", (unsigned long long)ticket);
    bool waiting = false;
    for (SJob* w : S->waiting) waiting = waiting || w == it->second;
    if (!waiting) {
        set_error("job %llu is not waiting for admission", (unsigned long long)ticket);
        return MRS_EBUSY;
    }
    S->fail_ticket = ticket;
    return MRS_OK;
}

int serve_destroy(mrs_server* S)
{
    clear_error();
    if (!S) return MRS_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    cudaSetDevice(S->ctx->device);
    cudaStreamSynchronize(S->stream);
    server_free(S);
    return MRS_OK;
}

}  // extern "C"
