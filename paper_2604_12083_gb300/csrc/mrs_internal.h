// mrs_internal.h -- internal declarations shared by the library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <list>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mrs_gb300.h"

namespace mrs {

// ---------------------------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of a time step (forces -> pair sum -> update) and
// of a symmetric pair sum (pair kernel -> reduction) are launched with programmatic stream
// serialization: a kernel may be scheduled while its predecessor's last CTAs are still running,
// and waits (pdl_wait, griddepcontrol.wait) before its first access to memory, until the
// predecessor has completed and its writes are visible.  This hides the launch gap between
// dependent kernels (inside captured graphs too).  For a kernel launched without the attribute
// the wait returns at once.  Every kernel launched through launch_pdl calls pdl_wait first, so
// a kernel also never overwrites what its predecessor still reads.
// ---------------------------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
#endif

// cluster > 0: the grid is also cut into thread-block clusters of `cluster` CTAs along x.
template <typename... Params, typename... Args>
inline cudaError_t launch_pdl_cl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem,
                                 cudaStream_t s, int cluster, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.numAttrs = 1;
    if (cluster > 0) {
        attr[1].id = cudaLaunchAttributeClusterDimension;
        attr[1].val.clusterDim.x = (unsigned)cluster;
        attr[1].val.clusterDim.y = 1;
        attr[1].val.clusterDim.z = 1;
        cfg.numAttrs = 2;
    }
    cfg.attrs = attr;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... Params, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args)
{
    return launch_pdl_cl(kernel, grid, block, smem, s, 0, args...);
}

// ---------------------------------------------------------------------------------------------
// Errors: a per-thread message plus the int status of the C ABI.
// ---------------------------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

#define MRS_CHECK_CUDA(call)                                                                  \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            ::mrs::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                             __LINE__);                                                       \
            return MRS_ECUDA;                                                                 \
        }                                                                                     \
    } while (0)

#define MRS_REQUIRE(cond, ...)                  \
    do {                                        \
        if (!(cond)) {                          \
            ::mrs::set_error(__VA_ARGS__);      \
            return MRS_EINVAL;                  \
        }                                       \
    } while (0)

// ---------------------------------------------------------------------------------------------
// Pair-sum work description (float32 persistent kernel).
//
// A system's targets are cut into tiles of TM = threads * targets_per_thread targets.  Each
// tile sweeps all sources of its system; that sweep is cut into work units of kUnitSources
// sources.  The units of all tiles are numbered consecutively (tile by tile) and CTA p of the
// persistent grid of P CTAs processes units [W p / P, W (p+1) / P): every CTA gets the same
// number of pairs up to one unit, whatever the mix of system sizes.  A tile processed by more
// than one CTA is completed by whichever of them finishes last (an atomic unit counter per
// tile), which sums the partial results in a fixed order.
// ---------------------------------------------------------------------------------------------
constexpr int kUnitSources = 32;   // sources per work unit (granularity of the CTA ranges)
constexpr int kChunk = 256;        // sources staged in shared memory at a time

// Persistent CTAs of an ordered launch over W units whose largest tile has max_nu units.  The
// CTA that completes a tile reads the partial slot of every CTA that worked on it, one L2 round
// trip per eight slots, while the other SMs idle at the end of the launch; for small systems
// (few tiles, each cut over tens of CTAs with a unit or two each) that read dominated the call.
// When the full grid would give a CTA fewer than kFewUnits units, the cut is capped at
// kMaxSlotsPerTile CTAs per tile (measured on GB300: a single 2048-point system 26 -> 16.5 us,
// 4096 points with 512-target tiles 50 -> 41 us).  With more work per CTA the full grid is
// kept: a cap there leaves SMs with unequal numbers of resident CTAs (16384 points with
// 512-target tiles: 486 -> 562 us when capped).
constexpr int kMaxSlotsPerTile = 16;
constexpr int kFewUnits = 4;
inline long long ordered_ctas(long long P, long long W, long long max_nu)
{
    if (P > W) P = W;
    if (max_nu > 0 && W < (long long)kFewUnits * P) {
        const long long cap = (long long)kMaxSlotsPerTile * W / max_nu;
        if (P > cap) P = cap;
    }
    return P < 1 ? 1 : P;
}

// CTAs of 256 threads or more (two warps per scheduler each): when the full grid of `full`
// CTAs would give each fewer than kBalancedUnits of the W units, one CTA per SM (at most P).
// A second such CTA on an SM shares its schedulers, so with a grid that is not a whole number
// of CTAs per SM the SMs that hold two set the call's length, and with little work per CTA
// the finishing CTAs' slot reads weigh more.  Measured on GB300, one system with 256-target
// tiles (µs per call, capped or full grid -> one CTA per SM): 2560 points 27.5 -> 20.6 (160
// -> 152 CTAs), 3072 points 31.9 -> 24.9 (192 -> 152), 4096 points 38.9 -> 35.5 (456 -> 152),
// 6144 points 76.9 -> 72.5; at 8192 points (18 units per CTA) the full grid stays best.
// Smaller CTAs keep the grid (64-thread CTAs lost 20 % when cut to one per SM).
constexpr int kBalancedUnits = 12;
inline long long balanced_ctas(long long P, long long full, long long W, int sms, int threads)
{
    if (threads >= 256 && W < (long long)kBalancedUnits * full && P > sms) P = sms;
    return P;
}

struct TileDesc {
    int sys;     // system index
    int t0;      // first target (global point index)
    int tn;      // number of targets in the tile (1..TM)
    int s0;      // first source of the system (global point index)
    int sn;      // number of sources of the system
    int nu;      // number of work units = ceil(sn / kUnitSources)
    long long u0;  // global index of the tile's first unit
};

struct SysConst {  // per-system constants of the scaled kernels (see mrs_kernels.cu)
    float e2, c1, c2, c3, c5, scale;
};

struct KernelConfig {
    int threads;   // threads per CTA
    int tpt;       // targets per thread
    int paired;    // 1: packed f32x2 inner loop (two sources per instruction)
    int unroll;    // source-loop unroll of the packed loop (independent pair chains in flight)
    int sq;        // 1: s^2 = s*s by a packed multiply instead of an SFU reciprocal
    int sym;       // 1: each unordered pair once (targets = sources only; mrs_sym.cu)
    int over;      // CTAs launched per resident CTA slot (0 or 1: one wave; > 1: the hardware
                   // block scheduler hands the later CTAs to SMs as earlier ones finish)
    int cluster;   // > 0: the cluster kernel (mrs_f32_cluster, ordered, TPT = 1): one
                   // thread-block cluster of up to `cluster` CTAs per target tile, each CTA over
                   // a share of the tile's sources, partials summed through distributed shared
                   // memory (small systems: no scratch, no counters, no finishing CTA)
    int groups;    // cluster kernel: source groups per CTA (threads = targets per tile x groups;
                   // each group sweeps every groups-th 4-source block of the CTA's sources)
};

// Targets per tile of a configuration.
inline int tile_targets(const KernelConfig& k)
{
    return k.threads * k.tpt / (k.groups > 1 ? k.groups : 1);
}

// Configurations compiled into the library (index = plan config id).
extern const KernelConfig kConfigs[];
extern const int kNumConfigs;

struct MrsLaunch {
    const TileDesc* tiles;
    int n_tiles;
    long long W;          // total work units
    int P;                // persistent CTAs
    const SysConst* sc;
    const float* X;
    const float* f;
    const float* n;
    const float* Xt;      // targets (== X when none given)
    float* u;
    float* w;
    float* partial;       // [2P][6][TM] floats
    int* counters;        // [n_tiles], zero between launches
    long long n_points;   // points of the arrays (index checks of the debug build)
    unsigned int* err;    // device error word: bit 0 = a non-finite output was written
    int cl = 0;           // cluster kernel: CTAs per cluster (P = n_tiles * cl); else unused
    // Rod stepping (cluster kernel only): when upX0 is set, the CTA that completes a target
    // also applies the update of Eqs. (newx, newD) to it with the velocities just summed:
    // X1 = X0 + u h, D1 = the frame D0 rotated by |w| h about w (float64; X1/D1 may alias
    // X0/D0, which the pair sum itself never reads); up_step (or NULL) advances by one.
    const double* upX0 = nullptr;
    const double* upD0 = nullptr;
    double* upX1 = nullptr;
    double* upD1 = nullptr;
    double up_h = 0.0;
    long long* up_step = nullptr;
};

cudaError_t launch_mrs_f32(int config, bool comp, const MrsLaunch& L, cudaStream_t s);
int occupancy_f32(int config, bool comp, int* ctas_per_sm);
// Cluster configurations: allow clusters of more than 8 CTAs for the kernel and return in
// *max_clusters how many clusters of `cl` CTAs can be resident at once (0: none fits).
int cluster_setup_f32(int config, bool comp, int cl, int* max_clusters);

// ---------------------------------------------------------------------------------------------
// Symmetric pair sum (targets = sources): every unordered pair {i, j} of a system is evaluated
// once and contributes to both points.
//
// A system's points are cut into tiles of TM points.  The row of a tile holds the sources
// from the tile's first point to the end of the system, cut into work units of kUnitSources
// sources: the first nd units are the tile itself (the diagonal block, evaluated as ordered
// pairs, each point as target only), the rest are later tiles (each unordered pair once: the
// tile's points collect their share in registers, the source points' share is reduced over
// the tile and written to a column partial).  As in the ordered kernel, CTA p of P processes
// the contiguous unit range [W p / P, W (p+1) / P).  Every segment of a row processed by one
// CTA writes a row partial; a second kernel sums, for every point, its row partials and the
// column partials of all earlier tiles of its system in a fixed order (deterministic).
//
// Passes: the column partials (one 6-vector per source slot of every unit, ~N^2 / (2 TM) of
// them) are bounded by cutting the tile list into consecutive passes of about equal work, each
// one launch of the pair kernel over its own units and one of the reduction kernel, which
// reuse one column-partial buffer of the largest pass's size.  A point's sum is final after
// the pass holding its tile (later passes only hold later tiles, whose column partials go to
// later points); the reduction of a pass writes the final values of its own tiles and carries
// the Kahan pair of every later point of the systems it touches to the next pass in `acc`.
// ---------------------------------------------------------------------------------------------
constexpr int kSymChunk = 128;     // sources staged in shared memory at a time

struct SymTile {
    int sys;       // system index
    int t0;        // first point of the tile (global point index)
    int tn;        // points in the tile (1..TM)
    int send;      // one past the system's last point (global point index)
    int nu;        // work units of the row: ceil((send - t0) / kUnitSources)
    int nd;        // diagonal units: ceil(tn / kUnitSources)
    int kt;        // index of the tile within its system
    int tfirst;    // global index of the system's first tile
    int seg0;      // first row-partial slot of this tile
    int nseg;      // number of CTAs (row segments) that process this row
    int qlo;       // first CTA (of the tile's pass) whose unit range meets the row
    int pad_;
    long long u0;  // global index of the row's first unit
};

// One pass of a symmetric plan: tiles [ta, tb) and their units [U0, U0 + W), run by P CTAs;
// the reduction covers tiles [ta, tc), tc = the end of the system of tile tb - 1.  seg0 and
// qlo of its tiles count from the pass's first row segment and first CTA.
struct SymPass {
    int ta, tb, tc, P;
    long long U0, W;
    long long nseg;       // row segments of the pass
};

struct SymLaunch {
    const SymTile* tiles;
    int n_tiles;
    int TM;
    long long W;          // work units of this pass
    int P;                // persistent CTAs
    long long U0;         // first work unit of this pass (global unit index; 0: one pass)
    int ta, tb, tc;       // tiles of this pass [ta, tb); the reduction covers tiles [ta, tc)
    float2* acc;          // [points][6] Kahan pairs carried between passes (NULL: one pass)
    long long n_points;   // points of the arrays (index checks of the debug build)
    long long col_units;  // work units the column-partial buffer holds
    long long row_segs;   // row segments the row-partial buffer holds
    const SysConst* sc;
    const float* X;
    const float* f;
    const float* n;
    float* u;
    float* w;
    float* rowpart;       // [segments][TM][6]
    float* colpart;       // [W * kUnitSources][6]: unit-major from U0, one 6-vector per source slot
    unsigned int* err;
};

cudaError_t launch_mrs_sym(int config, bool comp, const SymLaunch& L, cudaStream_t s);
int occupancy_sym(int config, bool comp, int* ctas_per_sm);
// The CTA (of P over W units) whose range contains unit x: host twin of the device search.
int cta_of_unit_host(long long W, int P, long long x);

struct MrsLaunch64 {
    int n_sys;
    const long long* offsets;   // device [n_sys+1]
    const double* eps;          // device [n_sys]
    const int* tile_sys;        // device [n_blocks]: system of each 128-target block
    const int* tile_t0;         // device [n_blocks]: first target of each block
    int n_blocks;
    double inv_mu;
    const double* X;
    const double* f;
    const double* n;
    const double* Xt;
    double* u;
    double* w;
    unsigned int* err;
};
cudaError_t launch_mrs_f64(const MrsLaunch64& L, cudaStream_t s);
constexpr int kF64Block = 128;

// Autotuning: best configuration per batch-shape bucket (precision, log2 of the number of
// systems, of the total points and of the largest system).
struct TuneKey {
    int precision, sys_log2, n_log2, max_log2;
    bool operator==(const TuneKey& o) const
    {
        return precision == o.precision && sys_log2 == o.sys_log2 && n_log2 == o.n_log2 &&
               max_log2 == o.max_log2;
    }
};
struct TuneEntry {
    TuneKey key;
    int config;
    float ms;
};
TuneKey tune_key(int n_sys, const int64_t* offsets, int precision);

struct RodWorkspace;
void rod_ws_free(RodWorkspace* ws);

}  // namespace mrs

// ---------------------------------------------------------------------------------------------
// Opaque ABI objects.
// ---------------------------------------------------------------------------------------------
struct mrs_plan {
    mrs_ctx* ctx = nullptr;
    int precision = MRS_F32_COMP;
    int config = 0;               // the plan's configuration (symmetric or ordered)
    int ocfg = 0;                 // ordered configuration (targets given apart from the sources)
    int n_sys = 0;
    int64_t n_points = 0;
    double mu = 1.0;
    std::vector<int64_t> offsets;
    std::vector<double> eps;
    // float32 persistent path
    int P = 0;
    int TM = 0;
    int cl = 0;                   // cluster configuration: CTAs per cluster (P = n_tiles * cl)
    long long W = 0;
    int n_tiles = 0;
    mrs::TileDesc* d_tiles = nullptr;
    mrs::SysConst* d_sc = nullptr;
    float* d_partial = nullptr;
    int* d_counters = nullptr;
    // symmetric path (config with sym = 1; used when the targets are the sources)
    int sym_config = -1;          // -1: no symmetric path; config then is the ordered one
    int sP = 0;
    int sTM = 0;
    long long sW = 0;
    int s_tiles = 0;
    std::vector<mrs::SymPass> passes;
    mrs::SymTile* d_stiles = nullptr;
    float* d_rowpart = nullptr;
    float* d_colpart = nullptr;
    float2* d_acc = nullptr;      // Kahan pairs carried between passes (more than one pass)
    // float64 path
    long long* d_off64 = nullptr;
    double* d_eps64 = nullptr;
    int* d_tile_sys = nullptr;
    int* d_tile_t0 = nullptr;
    int n_blocks64 = 0;
    bool owned_by_ctx = false;
};

struct mrs_ctx {
    int device = 0;
    unsigned int* d_err = nullptr;   // device error word (see mrs_device_status)
    int num_sms = 0;
    int cc_major = 0, cc_minor = 0;
    size_t smem_per_block_optin = 0;
    // plan cache used by mrs_velocity (LRU, most recent first)
    std::list<mrs_plan*> plan_cache;
    size_t plan_cache_max = 16;
    // rod workspaces used by rod_forces / rod_step / parareal_run (LRU, most recent first)
    std::list<mrs::RodWorkspace*> rod_ws;
    size_t rod_ws_max = 256;
    // measured best kernel configurations (mrs_autotune)
    std::vector<mrs::TuneEntry> tuned;
    // rod stepping in one fused launch per call (mrs_ctx_set_fused_steps): 0 never, 1 for
    // instances of at most kFusedAutoNodes nodes in batches too large for the warp-cooperative
    // kernels, 2 whenever the instance fits shared memory
    int fused_steps = 1;
    // rod force kernel (mrs_ctx_set_rod_force_kernel): 0 warp-cooperative for batches of at
    // most kWarpForceMaxNodes nodes, else one thread per segment; 1 always one thread per
    // segment; 2 always warp-cooperative
    int rod_force_kernel = 0;
    // largest column-partial buffer (bytes) of one pass of a symmetric plan; a plan with more
    // column partials is split into passes (mrs_ctx_set_sym_pass_bytes)
    size_t sym_pass_bytes = (size_t)192 << 20;
};

namespace mrs {
int plan_build(mrs_ctx* ctx, int n_sys, const int64_t* offsets, double mu, double eps,
               const double* eps_per_sys, int precision, int config, mrs_plan** out);
// Rod-step update applied by the pair sum itself (MrsLaunch::upX0 ...), when the plan runs the
// cluster kernel.
struct PlanUpdate {
    const double* X0;
    const double* D0;
    double* X1;
    double* D1;
    double h;
    long long* step;   // advanced by one, or NULL
};
// up != NULL: apply *up in the pair-sum launch when the plan allows it; *fused (when given)
// tells whether it did (otherwise the caller runs the update itself).
int plan_run(mrs_plan* p, const void* X, const void* f, const void* n, const void* Xt, void* u,
             void* w, cudaStream_t s, const PlanUpdate* up = nullptr, bool* fused = nullptr);
void plan_free(mrs_plan* p);
int default_config(mrs_ctx* ctx, int n_sys, const int64_t* offsets, int precision);
int default_ordered_config(int n_sys, const int64_t* offsets);
int tuned_config(const mrs_ctx* ctx, const TuneKey& k);
}  // namespace mrs
