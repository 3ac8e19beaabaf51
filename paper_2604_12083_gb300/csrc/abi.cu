// abi.cu -- host side of the C ABI: errors, contexts, pair-sum plans and mrs_velocity.
#include <cstdarg>
#include <cmath>
#include <cstring>

#include "mrs_internal.h"

namespace mrs {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

template <typename T>
static int dev_alloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        return MRS_ENOMEM;
    }
    return MRS_OK;
}

static int check_offsets(int n_sys, const int64_t* off)
{
    MRS_REQUIRE(n_sys >= 1, "n_sys must be >= 1 (got %d)", n_sys);
    MRS_REQUIRE(off != nullptr, "offsets is NULL");
    MRS_REQUIRE(off[0] == 0, "offsets[0] must be 0 (got %lld)", (long long)off[0]);
    for (int s = 0; s < n_sys; ++s)
        MRS_REQUIRE(off[s + 1] >= off[s], "offsets must be non-decreasing (offsets[%d] > offsets[%d])",
                    s, s + 1);
    MRS_REQUIRE(off[n_sys] < (int64_t)0x7fffffff, "total points %lld exceed 2^31-1",
                (long long)off[n_sys]);
    return MRS_OK;
}

int default_ordered_config(int n_sys, const int64_t* offsets)
{
    // Measured on GB300: the packed f32x2 variants are fastest.  256 threads x 2 targets
    // (512-target tiles) for systems of tens of thousands of points; when most points sit in
    // systems of at most 8192 points, for a few systems 256 threads x 1 target with the source
    // loop unrolled twice (a single 4096-point system: 41 us against 50 us with 512-target
    // tiles), or the cluster kernel when no system exceeds 2560 points: 32-target tiles with 8
    // source groups up to 1536 points (per call from a CUDA graph, 51 / 204 / 612 / 1275
    // points: 3.0 / 3.0 / 4.2 / 7.2 us against 5.3 / 5.9 / 8.0 / 12.4 with the persistent
    // kernel's 128-target tiles), 64-target tiles with 4 groups above (2048 points: 12.3
    // against 14.3 us); 64 threads x 4 targets (256-target tiles, 8 CTAs per SM) for many
    // systems (64 systems of 4096 points: 1.69 ms against 1.77 ms).  mrs_autotune overrides
    // all of them.
    int64_t small = 0, total = offsets[n_sys], largest = 0;
    for (int s = 0; s < n_sys; ++s) {
        const int64_t ns = offsets[s + 1] - offsets[s];
        if (ns <= 8192) small += ns;
        largest = std::max(largest, ns);
    }
    if (total > 0 && small * 2 > total)
        return n_sys >= 16 ? 8 : largest <= 1536 ? 27 : largest <= 2560 ? 28 : 14;
    return 9;
}

// Symmetric configurations used by default: 64 threads x 6 points launched as 4 waves of CTAs,
// and the same as one wave for systems with fewer work units.
constexpr int kDefaultSymConfig = 25;
constexpr int kOneWaveSymConfig = 23;

// Work units and column-partial bytes of a symmetric plan with tiles of TM points.
static double sym_units(int n_sys, const int64_t* offsets, int TM)
{
    double units = 0;
    for (int s = 0; s < n_sys; ++s) {
        const int64_t ns = offsets[s + 1] - offsets[s];
        for (int64_t t = 0; t < ns; t += TM) units += (double)((ns - t + kUnitSources - 1) / kUnitSources);
    }
    return units;
}

int default_config(mrs_ctx* ctx, int n_sys, const int64_t* offsets, int precision)
{
    (void)precision;
    // Measured on GB300: the symmetric kernel (each unordered pair once) beats the ordered
    // ones when most pairs lie in systems of 8192 points or more and there are enough work
    // units to keep every CTA of the persistent grid busy (a 4096-point system has ~600 units
    // for ~450 CTAs and runs slower than the ordered kernel).  Its column partials, which grow
    // as N^2 / TM, are bounded by splitting the plan into passes (sym_plan_build).
    double big = 0, all = 0;
    for (int s = 0; s < n_sys; ++s) {
        const double ns = (double)(offsets[s + 1] - offsets[s]);
        all += ns * ns;
        if (ns >= 8192) big += ns * ns;
    }
    const KernelConfig kc = kConfigs[kDefaultSymConfig];
    const double units = sym_units(n_sys, offsets, kc.threads * kc.tpt);
    const double ctas = 3.0 * (ctx ? ctx->num_sms : 152);
    if (all > 0 && big >= 0.5 * all && units >= 32.0 * ctas) return kDefaultSymConfig;
    // fewer units: the same tiles launched as one wave of CTAs still beat the ordered kernel
    // from ~12 units per resident CTA (one system, µs per call, this / default ordered:
    // 12288 points 248.6 / 260.8, 16384 points 422.3 / 444.2; at 8192 points, ~6 units per
    // CTA, 117.0 / 118.2 -- kept ordered)
    if (all > 0 && big >= 0.5 * all && units >= 12.0 * ctas) return kOneWaveSymConfig;
    return default_ordered_config(n_sys, offsets);
}

// Work table of the symmetric path (see SymTile): one row per tile of TM points, from the
// tile's first point to the end of its system; the tiles are cut into passes (SymPass) of
// about equal work whose column partials fit ctx->sym_pass_bytes; within a pass, row segments
// are numbered tile by tile, one per CTA whose unit range meets the row.
static int sym_plan_build(mrs_plan* p, mrs_ctx* ctx, int cfg, const int64_t* offsets)
{
    const KernelConfig kc = kConfigs[cfg];
    const int TM = kc.threads * kc.tpt;
    std::vector<SymTile> tiles;
    long long W = 0;
    for (int s = 0; s < p->n_sys; ++s) {
        const int64_t ns = offsets[s + 1] - offsets[s];
        const int tfirst = (int)tiles.size();
        for (int64_t t = 0, k = 0; t < ns; t += TM, ++k) {
            SymTile T{};
            T.sys = s;
            T.t0 = (int)(offsets[s] + t);
            T.tn = (int)std::min<int64_t>(TM, ns - t);
            T.send = (int)offsets[s + 1];
            T.nu = (int)((ns - t + kUnitSources - 1) / kUnitSources);
            T.nd = (T.tn + kUnitSources - 1) / kUnitSources;
            T.kt = (int)k;
            T.tfirst = tfirst;
            T.u0 = W;
            tiles.push_back(T);
            W += T.nu;
        }
    }
    int occ = 0;
    int st = occupancy_sym(cfg, p->precision == MRS_F32_COMP, &occ);
    if (st != MRS_OK || occ < 1) {
        set_error("occupancy query failed for config %d", cfg);
        return MRS_ECUDA;
    }
    const long long Pmax = (long long)ctx->num_sms * occ * std::max(1, kc.over);
    // passes: n_pass = ceil(column-partial bytes / sym_pass_bytes); cut at the tile where the
    // running unit count first reaches g W / n_pass
    const double unit_bytes = (double)kUnitSources * 6 * sizeof(float);
    const double cap = std::max<double>((double)ctx->sym_pass_bytes, unit_bytes);
    const long long n_pass =
        std::max<long long>(1, (long long)std::ceil((double)W * unit_bytes / cap));
    p->passes.clear();
    {
        const int nt = (int)tiles.size();
        int ta = 0;
        for (long long g = 1; g <= n_pass && ta < nt; ++g) {
            const long long target = (W * g) / n_pass;
            int tb = ta + 1;
            while (tb < nt && tiles[tb].u0 < target) ++tb;
            if (g == n_pass) tb = nt;
            SymPass ps{};
            ps.ta = ta;
            ps.tb = tb;
            ps.U0 = tiles[ta].u0;
            ps.W = (tb < nt ? tiles[tb].u0 : W) - ps.U0;
            const int last_sys = tiles[tb - 1].sys;
            int tc = tb;
            while (tc < nt && tiles[tc].sys == last_sys) ++tc;
            ps.tc = tc;
            ps.P = (int)std::min<long long>(Pmax, ps.W);
            p->passes.push_back(ps);
            ta = tb;
        }
    }
    long long max_seg = 0, max_units = 0, max_P = 0;
    for (SymPass& ps : p->passes) {
        long long nseg = 0;
        for (int t = ps.ta; t < ps.tb; ++t) {
            SymTile& T = tiles[t];
            T.qlo = cta_of_unit_host(ps.W, ps.P, T.u0 - ps.U0);
            const int qhi = cta_of_unit_host(ps.W, ps.P, T.u0 - ps.U0 + T.nu - 1);
            T.nseg = qhi - T.qlo + 1;
            T.seg0 = (int)nseg;
            nseg += T.nseg;
        }
        ps.nseg = nseg;
        max_seg = std::max(max_seg, nseg);
        max_units = std::max(max_units, ps.W);
        max_P = std::max<long long>(max_P, ps.P);
    }
    p->sym_config = cfg;
    p->sP = (int)max_P;
    p->sW = W;
    p->s_tiles = (int)tiles.size();
    p->sTM = TM;
    if ((st = dev_alloc(&p->d_stiles, tiles.size())) ||
        (st = dev_alloc(&p->d_rowpart, (size_t)max_seg * TM * 6)) ||
        (st = dev_alloc(&p->d_colpart, (size_t)max_units * kUnitSources * 6)))
        return st;
    if (p->passes.size() > 1 && (st = dev_alloc(&p->d_acc, (size_t)p->n_points * 6))) return st;
    cudaMemcpy(p->d_stiles, tiles.data(), tiles.size() * sizeof(SymTile), cudaMemcpyHostToDevice);
    return MRS_OK;
}

void plan_free(mrs_plan* p)
{
    if (!p) return;
    cudaFree(p->d_tiles);
    cudaFree(p->d_sc);
    cudaFree(p->d_partial);
    cudaFree(p->d_counters);
    cudaFree(p->d_off64);
    cudaFree(p->d_eps64);
    cudaFree(p->d_tile_sys);
    cudaFree(p->d_tile_t0);
    cudaFree(p->d_stiles);
    cudaFree(p->d_rowpart);
    cudaFree(p->d_colpart);
    cudaFree(p->d_acc);
    delete p;
}

int plan_build(mrs_ctx* ctx, int n_sys, const int64_t* offsets, double mu, double eps,
               const double* eps_per_sys, int precision, int config, mrs_plan** out)
{
    *out = nullptr;
    MRS_REQUIRE(ctx != nullptr, "ctx is NULL");
    int st = check_offsets(n_sys, offsets);
    if (st) return st;
    MRS_REQUIRE(precision == MRS_F64 || precision == MRS_F32 || precision == MRS_F32_COMP,
                "unknown precision %d", precision);
    MRS_REQUIRE(std::isfinite(mu) && mu > 0.0, "mu must be > 0 (got %g)", mu);
    MRS_REQUIRE(config >= -1 && config < kNumConfigs, "config %d out of range", config);
    std::vector<double> epsv(n_sys);
    for (int s = 0; s < n_sys; ++s) {
        epsv[s] = eps_per_sys ? eps_per_sys[s] : eps;
        MRS_REQUIRE(std::isfinite(epsv[s]) && epsv[s] > 0.0, "eps of system %d must be > 0 (got %g)",
                    s, epsv[s]);
    }
    MRS_CHECK_CUDA(cudaSetDevice(ctx->device));

    mrs_plan* p = new mrs_plan();
    p->ctx = ctx;
    p->precision = precision;
    p->n_sys = n_sys;
    p->n_points = offsets[n_sys];
    p->mu = mu;
    p->offsets.assign(offsets, offsets + n_sys + 1);
    p->eps = epsv;

    if (precision == MRS_F64) {
        std::vector<int> bs, bt;
        for (int s = 0; s < n_sys; ++s)
            for (int64_t t = offsets[s]; t < offsets[s + 1]; t += kF64Block) {
                bs.push_back(s);
                bt.push_back((int)t);
            }
        p->n_blocks64 = (int)bs.size();
        std::vector<long long> off64(offsets, offsets + n_sys + 1);
        if ((st = dev_alloc(&p->d_off64, off64.size())) || (st = dev_alloc(&p->d_eps64, epsv.size())) ||
            (st = dev_alloc(&p->d_tile_sys, bs.size())) || (st = dev_alloc(&p->d_tile_t0, bt.size()))) {
            plan_free(p);
            return st;
        }
        cudaMemcpy(p->d_off64, off64.data(), off64.size() * sizeof(long long), cudaMemcpyHostToDevice);
        cudaMemcpy(p->d_eps64, epsv.data(), epsv.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (!bs.empty()) {
            cudaMemcpy(p->d_tile_sys, bs.data(), bs.size() * sizeof(int), cudaMemcpyHostToDevice);
            cudaMemcpy(p->d_tile_t0, bt.data(), bt.size() * sizeof(int), cudaMemcpyHostToDevice);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            plan_free(p);
            set_error("plan upload failed: %s", cudaGetErrorString(e));
            return MRS_ECUDA;
        }
        *out = p;
        return MRS_OK;
    }

    int cfg = config;
    if (cfg < 0) cfg = tuned_config(ctx, tune_key(n_sys, offsets, precision));
    if (cfg < 0) cfg = default_config(ctx, n_sys, offsets, precision);
    p->config = cfg;
    p->ocfg = kConfigs[cfg].sym ? default_ordered_config(n_sys, offsets) : cfg;
    const KernelConfig kc = kConfigs[p->ocfg];
    p->TM = tile_targets(kc);
    std::vector<TileDesc> tiles;
    long long W = 0;
    for (int s = 0; s < n_sys; ++s) {
        const int64_t ns = offsets[s + 1] - offsets[s];
        if (ns == 0) continue;
        const int nu = (int)((ns + kUnitSources - 1) / kUnitSources);
        for (int64_t t = 0; t < ns; t += p->TM) {
            TileDesc T;
            T.sys = s;
            T.t0 = (int)(offsets[s] + t);
            T.tn = (int)std::min<int64_t>(p->TM, ns - t);
            T.s0 = (int)offsets[s];
            T.sn = (int)ns;
            T.nu = nu;
            T.u0 = W;
            tiles.push_back(T);
            W += nu;
        }
    }
    p->W = W;
    p->n_tiles = (int)tiles.size();
    std::vector<SysConst> sc(n_sys);
    for (int s = 0; s < n_sys; ++s) {
        const double e2 = epsv[s] * epsv[s];
        sc[s].e2 = (float)e2;
        sc[s].c1 = (float)(1.5 * e2);
        sc[s].c2 = (float)(3.75 * e2 * e2);
        sc[s].c3 = (float)(-0.75 * e2);
        sc[s].c5 = (float)(3.75 * e2);
        sc[s].scale = (float)(1.0 / (8.0 * M_PI * mu));
    }
    if (p->n_tiles == 0) {
        *out = p;
        return MRS_OK;
    }
    int occ = 0;
    if ((st = occupancy_f32(p->ocfg, precision == MRS_F32_COMP, &occ)) != MRS_OK || occ < 1) {
        plan_free(p);
        set_error("occupancy query failed for config %d", p->ocfg);
        return MRS_ECUDA;
    }
    long long max_nu = 0;
    for (const TileDesc& T : tiles) max_nu = std::max<long long>(max_nu, T.nu);
    long long P = 0;
    if (kc.cluster) {
        // one cluster per tile: the largest size (at most the configuration's cap and the
        // largest tile's units) for which the clusters of all tiles are resident at once, so
        // that no cluster waits for a second wave; size 1 if none
        const bool comp = precision == MRS_F32_COMP;
        int cl = (int)std::max<long long>(1, std::min<long long>(kc.cluster, max_nu));
        for (;; --cl) {
            int mc = 0;
            const int cst = cluster_setup_f32(p->ocfg, comp, cl, &mc);
            if (cst != MRS_OK) cudaGetLastError();   // a refused cluster shape is not an error of the plan
            if (cst == MRS_OK && mc >= 1 && (mc >= p->n_tiles || cl == 1)) break;
            if (cl == 1) {
                plan_free(p);
                set_error("no cluster of config %d fits on the device", p->ocfg);
                return MRS_ECUDA;
            }
        }
        p->cl = cl;
        P = (long long)p->n_tiles * cl;
    } else {
        const long long full = (long long)ctx->num_sms * occ * std::max(1, kc.over);
        P = balanced_ctas(ordered_ctas(full, W, max_nu), full, W, ctx->num_sms, kc.threads);
    }
    p->P = (int)P;
    const size_t part_floats = kc.cluster ? 1 : (size_t)2 * P * 6 * p->TM;
    if ((st = dev_alloc(&p->d_tiles, tiles.size())) || (st = dev_alloc(&p->d_sc, sc.size())) ||
        (st = dev_alloc(&p->d_partial, part_floats)) || (st = dev_alloc(&p->d_counters, tiles.size()))) {
        plan_free(p);
        return st;
    }
    cudaMemcpy(p->d_tiles, tiles.data(), tiles.size() * sizeof(TileDesc), cudaMemcpyHostToDevice);
    cudaMemcpy(p->d_sc, sc.data(), sc.size() * sizeof(SysConst), cudaMemcpyHostToDevice);
    cudaMemset(p->d_counters, 0, tiles.size() * sizeof(int));
    if (kConfigs[cfg].sym && (st = sym_plan_build(p, ctx, cfg, offsets)) != MRS_OK) {
        plan_free(p);
        return st;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        plan_free(p);
        set_error("plan upload failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    *out = p;
    return MRS_OK;
}

static bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb)
{
    const char* pa = (const char*)a;
    const char* pb = (const char*)b;
    return pa < pb + nb && pb < pa + na;
}

int plan_run(mrs_plan* p, const void* X, const void* f, const void* n, const void* Xt, void* u,
             void* w, cudaStream_t s, const PlanUpdate* up, bool* fused)
{
    if (fused) *fused = false;
    MRS_REQUIRE(p != nullptr, "plan is NULL");
    if (p->n_points == 0) return MRS_OK;
    MRS_REQUIRE(X && f && n && u && w, "NULL input or output pointer");
    const size_t es = p->precision == MRS_F64 ? 8 : 4;
    const size_t bytes = (size_t)p->n_points * 3 * es;
    const void* ins[4] = {X, f, n, Xt ? Xt : X};
    for (int i = 0; i < 4; ++i)
        MRS_REQUIRE(!ranges_overlap(ins[i], bytes, u, bytes) && !ranges_overlap(ins[i], bytes, w, bytes),
                    "outputs must not overlap the inputs");
    MRS_REQUIRE(!ranges_overlap(u, bytes, w, bytes), "u and w must not overlap");
    MRS_REQUIRE(((uintptr_t)X | (uintptr_t)f | (uintptr_t)n | (uintptr_t)ins[3] | (uintptr_t)u |
                 (uintptr_t)w) % es == 0, "pointers must be aligned to the element size");
    cudaError_t e;
    if (p->precision == MRS_F64) {
        MrsLaunch64 L;
        L.n_sys = p->n_sys;
        L.offsets = p->d_off64;
        L.eps = p->d_eps64;
        L.tile_sys = p->d_tile_sys;
        L.tile_t0 = p->d_tile_t0;
        L.n_blocks = p->n_blocks64;
        L.inv_mu = 1.0 / p->mu;
        L.X = (const double*)X;
        L.f = (const double*)f;
        L.n = (const double*)n;
        L.Xt = (const double*)ins[3];
        L.u = (double*)u;
        L.w = (double*)w;
        L.err = p->ctx->d_err;
        e = launch_mrs_f64(L, s);
    } else {
        if (p->n_tiles == 0) return MRS_OK;
        MrsLaunch L;
        L.tiles = p->d_tiles;
        L.n_tiles = p->n_tiles;
        L.W = p->W;
        L.P = p->P;
        L.sc = p->d_sc;
        L.X = (const float*)X;
        L.f = (const float*)f;
        L.n = (const float*)n;
        L.Xt = (const float*)ins[3];
        L.u = (float*)u;
        L.w = (float*)w;
        L.partial = p->d_partial;
        L.counters = p->d_counters;
        L.err = p->ctx->d_err;
        L.n_points = p->n_points;
        L.cl = p->cl;
        if (p->sym_config >= 0 && (Xt == nullptr || Xt == X)) {
            SymLaunch S;
            S.tiles = p->d_stiles;
            S.n_tiles = p->s_tiles;
            S.TM = p->sTM;
            S.sc = p->d_sc;
            S.X = L.X;
            S.f = L.f;
            S.n = L.n;
            S.u = L.u;
            S.w = L.w;
            S.rowpart = p->d_rowpart;
            S.colpart = p->d_colpart;
            S.acc = p->d_acc;
            S.err = L.err;
            S.n_points = p->n_points;
            {
                long long cu = 0, rs = 0;
                for (const SymPass& ps : p->passes) {
                    cu = std::max(cu, ps.W);
                    rs = std::max(rs, ps.nseg);
                }
                S.col_units = cu;
                S.row_segs = rs;
            }
            e = cudaSuccess;
            for (const SymPass& ps : p->passes) {   // in order: each pass reuses the buffers
                S.W = ps.W;
                S.P = ps.P;
                S.U0 = ps.U0;
                S.ta = ps.ta;
                S.tb = ps.tb;
                S.tc = ps.tc;
                e = launch_mrs_sym(p->sym_config, p->precision == MRS_F32_COMP, S, s);
                if (e != cudaSuccess) break;
            }
        } else {
            if (up && p->cl > 0) {   // the cluster kernel applies the rod-step update itself
                L.upX0 = up->X0;
                L.upD0 = up->D0;
                L.upX1 = up->X1;
                L.upD1 = up->D1;
                L.up_h = up->h;
                L.up_step = up->step;
                if (fused) *fused = true;
            }
            e = launch_mrs_f32(p->ocfg, p->precision == MRS_F32_COMP, L, s);
        }
    }
    if (e != cudaSuccess) {
        set_error("pair-sum launch failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    return MRS_OK;
}

}  // namespace mrs

using namespace mrs;

extern "C" {

const char* mrs_last_error(void) { return g_err; }

const char* mrs_version(void) { return "mrs_gb300 0.1 (sm_103a)"; }

int mrs_ctx_create(mrs_ctx** ctx, int device)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr, "ctx is NULL");
    *ctx = nullptr;
    int ndev = 0;
    MRS_CHECK_CUDA(cudaGetDeviceCount(&ndev));
    MRS_REQUIRE(device >= 0 && device < ndev, "device %d out of range (%d devices)", device, ndev);
    MRS_CHECK_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    MRS_CHECK_CUDA(cudaGetDeviceProperties(&prop, device));
    MRS_REQUIRE(prop.major == 10 && prop.minor == 3,
                "this library is built for sm_103a (GB300); device %d is sm_%d%d", device,
                prop.major, prop.minor);
    mrs_ctx* c = new mrs_ctx();
    c->device = device;
    if (cudaMalloc((void**)&c->d_err, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(c->d_err, 0, sizeof(unsigned int)) != cudaSuccess) {
        cudaFree(c->d_err);
        delete c;
        set_error("device error word allocation failed");
        return MRS_ENOMEM;
    }
    c->num_sms = prop.multiProcessorCount;
    c->cc_major = prop.major;
    c->cc_minor = prop.minor;
    c->smem_per_block_optin = prop.sharedMemPerBlockOptin;
    *ctx = c;
    return MRS_OK;
}

int mrs_ctx_destroy(mrs_ctx* ctx)
{
    clear_error();
    if (!ctx) return MRS_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (mrs_plan* p : ctx->plan_cache) plan_free(p);
    ctx->plan_cache.clear();
    for (RodWorkspace* w : ctx->rod_ws) rod_ws_free(w);
    ctx->rod_ws.clear();
    cudaFree(ctx->d_err);
    delete ctx;
    return MRS_OK;
}

int mrs_ctx_num_sms(const mrs_ctx* ctx) { return ctx ? ctx->num_sms : 0; }

int mrs_ctx_set_fused_steps(mrs_ctx* ctx, int enable)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr, "ctx is NULL");
    MRS_REQUIRE(enable >= 0 && enable <= 2, "mode must be 0, 1 or 2 (got %d)", enable);
    ctx->fused_steps = enable;
    return MRS_OK;
}

int mrs_ctx_set_rod_force_kernel(mrs_ctx* ctx, int mode)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr, "ctx is NULL");
    MRS_REQUIRE(mode >= 0 && mode <= 2, "mode must be 0, 1 or 2 (got %d)", mode);
    ctx->rod_force_kernel = mode;
    return MRS_OK;
}

int mrs_ctx_set_sym_pass_bytes(mrs_ctx* ctx, size_t bytes)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr, "ctx is NULL");
    MRS_REQUIRE(bytes >= (size_t)kUnitSources * 6 * sizeof(float),
                "bytes must hold at least one work unit's column partials (%zu)",
                (size_t)kUnitSources * 6 * sizeof(float));
    ctx->sym_pass_bytes = bytes;
    return MRS_OK;
}

int mrs_device_status(mrs_ctx* ctx, unsigned int* flags)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr && flags != nullptr, "NULL argument");
    MRS_CHECK_CUDA(cudaSetDevice(ctx->device));
    MRS_CHECK_CUDA(cudaDeviceSynchronize());
    MRS_CHECK_CUDA(cudaMemcpy(flags, ctx->d_err, sizeof(unsigned int), cudaMemcpyDeviceToHost));
    MRS_CHECK_CUDA(cudaMemset(ctx->d_err, 0, sizeof(unsigned int)));
    return MRS_OK;
}

int mrs_plan_create(mrs_ctx* ctx, int n_sys, const int64_t* offsets, double mu, double eps,
                    const double* eps_per_sys, int precision, int config, mrs_plan** plan)
{
    clear_error();
    MRS_REQUIRE(plan != nullptr, "plan is NULL");
    return plan_build(ctx, n_sys, offsets, mu, eps, eps_per_sys, precision, config, plan);
}

int mrs_plan_execute(mrs_plan* plan, const void* X, const void* f, const void* n, const void* Xt,
                     void* u, void* w, void* stream)
{
    clear_error();
    MRS_REQUIRE(plan != nullptr, "plan is NULL");
    MRS_CHECK_CUDA(cudaSetDevice(plan->ctx->device));
    return plan_run(plan, X, f, n, Xt, u, w, (cudaStream_t)stream);
}

int mrs_plan_destroy(mrs_plan* plan)
{
    clear_error();
    if (!plan) return MRS_OK;
    MRS_REQUIRE(!plan->owned_by_ctx, "plan is owned by its context's cache");
    cudaSetDevice(plan->ctx->device);
    plan_free(plan);
    return MRS_OK;
}

int mrs_plan_config_count(void) { return kNumConfigs; }

int mrs_plan_config_symmetric(int config)
{
    return (config >= 0 && config < kNumConfigs) ? kConfigs[config].sym : -1;
}

int mrs_plan_config_info(mrs_ctx* ctx, int config, int* threads, int* tpt, int* ctas_per_sm)
{
    clear_error();
    MRS_REQUIRE(config >= 0 && config < kNumConfigs, "config %d out of range", config);
    if (threads) *threads = kConfigs[config].threads;
    if (tpt) *tpt = kConfigs[config].tpt;
    if (ctas_per_sm) {
        MRS_REQUIRE(ctx != nullptr, "ctx is NULL");
        MRS_CHECK_CUDA(cudaSetDevice(ctx->device));
        int st = kConfigs[config].sym ? occupancy_sym(config, true, ctas_per_sm)
                                      : occupancy_f32(config, true, ctas_per_sm);
        if (st) return st;
    }
    return MRS_OK;
}

int mrs_plan_info(const mrs_plan* plan, int* grid, int64_t* work_units, int* config)
{
    clear_error();
    MRS_REQUIRE(plan != nullptr, "plan is NULL");
    const bool sym = plan->precision != MRS_F64 && plan->sym_config >= 0;
    if (grid) *grid = plan->precision == MRS_F64 ? plan->n_blocks64 : (sym ? plan->sP : plan->P);
    if (work_units) *work_units = sym ? plan->sW : plan->W;
    if (config) *config = plan->config;
    return MRS_OK;
}

int mrs_plan_scratch(const mrs_plan* plan, int* passes, size_t* scratch_bytes)
{
    clear_error();
    MRS_REQUIRE(plan != nullptr, "plan is NULL");
    const bool sym = plan->precision != MRS_F64 && plan->sym_config >= 0;
    if (passes) *passes = sym ? (int)plan->passes.size() : 1;
    if (scratch_bytes) {
        // ordered slots (none for a cluster configuration: its partials stay on chip)
        size_t b = plan->cl ? 0 : (size_t)2 * plan->P * 6 * plan->TM * sizeof(float);
        if (sym) {
            long long seg = 0, units = 0;
            for (const SymPass& ps : plan->passes) {
                seg = std::max(seg, ps.nseg);
                units = std::max(units, ps.W);
            }
            b += (size_t)seg * plan->sTM * 6 * sizeof(float) +
                 (size_t)units * kUnitSources * 6 * sizeof(float) +
                 (plan->passes.size() > 1 ? (size_t)plan->n_points * 6 * sizeof(float2) : 0);
        }
        *scratch_bytes = b;
    }
    return MRS_OK;
}

}  // extern "C"

namespace mrs {

// The context's cached plan for (offsets, eps, precision, mu), built and cached on a miss (the
// least recently used plan is evicted beyond plan_cache_max).
static int cached_plan(mrs_ctx* ctx, int n_sys, const int64_t* offsets, double mu, double eps,
                       const double* eps_per_sys, int precision, mrs_plan** out)
{
    for (auto it = ctx->plan_cache.begin(); it != ctx->plan_cache.end(); ++it) {
        mrs_plan* p = *it;
        if (p->precision != precision || p->n_sys != n_sys || p->mu != mu) continue;
        if (std::memcmp(p->offsets.data(), offsets, sizeof(int64_t) * (n_sys + 1)) != 0) continue;
        bool same = true;
        for (int s = 0; s < n_sys && same; ++s)
            same = p->eps[s] == (eps_per_sys ? eps_per_sys[s] : eps);
        if (!same) continue;
        ctx->plan_cache.erase(it);
        ctx->plan_cache.push_front(p);
        *out = p;
        return MRS_OK;
    }
    mrs_plan* hit = nullptr;
    const int st = plan_build(ctx, n_sys, offsets, mu, eps, eps_per_sys, precision, -1, &hit);
    if (st) return st;
    hit->owned_by_ctx = true;
    ctx->plan_cache.push_front(hit);
    while (ctx->plan_cache.size() > ctx->plan_cache_max) {  // evict the least recent
        mrs_plan* old = ctx->plan_cache.back();
        ctx->plan_cache.pop_back();
        cudaDeviceSynchronize();   // the evicted plan's scratch may still be in use
        plan_free(old);
    }
    *out = hit;
    return MRS_OK;
}

}  // namespace mrs

extern "C" {

int mrs_reserve(mrs_ctx* ctx, int n_sys, const int64_t* offsets, double mu, double eps,
                const double* eps_per_sys, int precision)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr, "ctx is NULL");
    int st = check_offsets(n_sys, offsets);
    if (st) return st;
    mrs_plan* p = nullptr;
    return cached_plan(ctx, n_sys, offsets, mu, eps, eps_per_sys, precision, &p);
}

int mrs_velocity(mrs_ctx* ctx, int n_sys, const int64_t* offsets, const void* X, const void* f,
                 const void* n, const void* Xt, void* u, void* w, double mu, double eps,
                 const double* eps_per_sys, int precision, void* stream)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr, "ctx is NULL");
    int st = check_offsets(n_sys, offsets);
    if (st) return st;
    mrs_plan* hit = nullptr;
    if ((st = cached_plan(ctx, n_sys, offsets, mu, eps, eps_per_sys, precision, &hit))) return st;
    MRS_CHECK_CUDA(cudaSetDevice(ctx->device));
    return plan_run(hit, X, f, n, Xt, u, w, (cudaStream_t)stream);
}

}  // extern "C"
