// rod_internal.h -- rod kernels, rod workspaces (device buffers + captured step graphs).
#pragma once

#include "mrs_internal.h"

namespace mrs {

struct RodLaunch {
    int N;                     // nodes in the batch (all instances)
    int nodes_per_inst;        // nodes of one instance
    const int2* node_info;     // [N]: (index within rod, nodes of the rod)
    const double* t0;          // [n_inst]: start time of every instance
    long long* step;           // step counter of the current run (time = t0 + step * dt)
    double dt;
    mrs_rod_params p;
    double* FN;                // [N][6] segment force / moment scratch (two-kernel path)
    const int* chunks;         // [n_chunks] base node of every fused-kernel chunk, or NULL
    int n_chunks;
    // [n_wchunks] every chunk of kWNodes nodes of the warp-cooperative force kernel (batches of
    // at most kWarpForceMaxNodes nodes by default): (base node, nodes of its rod, index of the
    // base node in the rod, instance), or NULL
    const int4* wchunks = nullptr;
    int n_wchunks = 0;
    double inv_L;              // 1 / p.L
    // Reference point of the float32 position packs (see rod_kernels.cu): the mean of the
    // nodes ref[0..n_ref) of the instance (indices within it), weight ref_w = 1 / n_ref;
    // n_ref = 0 packs X itself.
    int n_ref;
    int ref[8];
    double ref_w;
    // [N] (sin, cos) of k_w s_mid for the segment k+1/2 of every node (Omega_2 by angle
    // addition, one sincos(f t) per CTA), or NULL: sin(k_w s_mid + f t) per segment
    const double2* segsc;
    unsigned int* err;         // device error word (MRS_FLAG_BOUNDS of the debug build), or NULL
};

// The reference nodes of an instance with rods rod_off[0..n_rods]: the middle node of up to 8
// rods spread over it (a function of the rod layout only).
inline void set_pack_reference(RodLaunch& L, int n_rods, const int64_t* rod_off)
{
    const int R = n_rods < 8 ? n_rods : 8;
    L.n_ref = R;
    for (int i = 0; i < R; ++i) {
        const int r = (int)((long long)i * n_rods / R);
        L.ref[i] = (int)(rod_off[r] + (rod_off[r + 1] - rod_off[r] - 1) / 2);
    }
    L.ref_w = R > 0 ? 1.0 / R : 0.0;
}
constexpr int kRodChunk = 128;   // threads per fused rod-force CTA (kRodChunk - 1 nodes each)
constexpr int kWNodes = 8;       // nodes per CTA of the warp-cooperative force kernel
// Largest batch (nodes) given the warp-cooperative force kernel: below it the kernel's many
// short float64 paths beat one long path per thread; above it every scheduler already has a
// thread-per-segment warp and the duplicated per-lane work costs more than it saves.
constexpr int kWarpForceMaxNodes = 4096;

cudaError_t launch_rod_forces(const RodLaunch& L, const double* X, const double* D, double t_off,
                              double* g64, double* m64, float* Xf, float* gf, float* mf,
                              cudaStream_t s);
cudaError_t launch_rod_update(const RodLaunch& L, const double* X0, const double* D0,
                              const float* u, const float* w, double h, double* X1, double* D1,
                              bool bump_step, cudaStream_t s);
cudaError_t launch_rod_update64(const RodLaunch& L, const double* X0, const double* D0,
                                const double* u, const double* w, double h, double* X1,
                                double* D1, bool bump_step, cudaStream_t s);
cudaError_t launch_rot_sqrt_batch(int n, const double* R, double* S, cudaStream_t s);
// segsc table of RodLaunch for wave number wave_k and rod length Lrod.
cudaError_t launch_segment_table(int N, const int2* node_info, double wave_k, double Lrod,
                                 double2* out, cudaStream_t s);
// Fused fine propagator (one CTA per instance, state in shared memory): nsteps steps of size
// L.dt of every instance of the batch in one launch, then the step counter advances by nsteps.
// Usable when the instance fits shared memory (fused_fits) -- float32 pair sum.
constexpr size_t kFusedMaxSmem = 200 * 1024;
// Largest instance the fused path takes by default, for batches of more than
// kWarpForceMaxNodes nodes.  Measured on GB300 (us per Euler step of a single instance, fused /
// graphs with the thread-per-segment kernels): 51 nodes 16.2 / 21.4, 128 nodes 22.6 / 22.7,
// 192 nodes 39.0 / 22.6, 512 nodes 163 / 26.5; 64-slice Parareal batches tie at 128 nodes and
// favour the graphs from 192 on (3.6x at 512): one SM per instance stops paying beyond ~128
// nodes.  With the warp-cooperative kernels (batches of up to kWarpForceMaxNodes nodes) the
// graphs win outright: 51 nodes 15.6 / 11.6 us.
constexpr int kFusedAutoNodes = 128;
size_t fused_smem_bytes(int N1);
bool fused_fits(int N1);
cudaError_t launch_rod_fine_fused(const RodLaunch& L, double* X, double* D, int nsteps, int scheme,
                                  double mu, double eps, cudaStream_t s);
cudaError_t launch_set_times(double* t0, int n_inst, double t_first, double dT, long long* step,
                             cudaStream_t s);


// One batch of n_inst identical rod sets (instance i = the rods of rod_off shifted by i*N1
// nodes); every instance is its own hydrodynamic system.
struct RodWorkspace {
    mrs_ctx* ctx = nullptr;
    int n_inst = 0;
    int tag = 0;               // distinguishes workspaces used concurrently for the same shape
    int n_rods = 0;            // rods per instance
    int N1 = 0;                // nodes per instance
    int N = 0;                 // total nodes
    int precision = MRS_F32_COMP;
    std::vector<int64_t> rod_off;   // per instance, n_rods+1
    int2* d_node_info = nullptr;
    int* d_chunks = nullptr;
    int n_chunks = 0;
    int4* d_wchunks = nullptr;
    int n_wchunks = 0;
    double* d_t0 = nullptr;
    long long* d_step = nullptr;
    double* d_FN = nullptr;
    float* d_Xf = nullptr;
    float* d_gf = nullptr;
    float* d_mf = nullptr;
    float* d_u = nullptr;
    float* d_w = nullptr;
    double* d_g64 = nullptr;
    double* d_m64 = nullptr;
    double* d_u64 = nullptr;
    double* d_w64 = nullptr;
    double* d_Xh = nullptr;
    double* d_Dh = nullptr;
    double2* d_segsc = nullptr;      // RodLaunch::segsc, valid for (segsc_k, segsc_L)
    double segsc_k = 0.0, segsc_L = -1.0;
    mrs_plan* plan = nullptr;
    cudaStream_t cap = nullptr;   // private stream used only for graph capture
    struct Graph {
        const double* X;
        const double* D;
        int scheme;
        int steps;
        double dt;
        mrs_rod_params p;
        int force_kernel;   // the context's rod force kernel setting at capture
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
};

int rod_ws_get(mrs_ctx* ctx, int n_rods, const int64_t* rod_off, int n_inst, int precision,
               double mu, double eps, RodWorkspace** out, int tag = 0);
// Parareal correction of one slice (see parareal.cu); GnX == NULL accepts the fine value.
cudaError_t launch_parareal_correct(int N1, const double* FpX, const double* FpD, const double* GnX,
                                    const double* GnD, double* GoX, double* GoD, double* UX,
                                    double* UD, double* incr, cudaStream_t s);
void rod_ws_free(RodWorkspace* ws);
RodLaunch rod_launch(const RodWorkspace* ws, const mrs_rod_params* p, double dt);

// Lennard-Jones length used by the kernels: lj_sigma when > 0, else 3 eps (Section IV-A).
inline double lj_sigma_of(const mrs_rod_params& p)
{
    return p.lj_sigma > 0.0 ? p.lj_sigma : 3.0 * p.eps;
}
// Enqueue `nsteps` steps of size dt on the workspace's state buffers X, D (device), with the
// instance start times already set; replays captured graphs.
int rod_ws_steps(RodWorkspace* ws, const mrs_rod_params* p, double* X, double* D, double dt,
                 int nsteps, int scheme, cudaStream_t s);
// Instance i of the batch starts at t_first + i * dT; resets the step counter (stream-ordered).
int rod_ws_set_times(RodWorkspace* ws, double t_first, double dT, cudaStream_t s);

}  // namespace mrs
