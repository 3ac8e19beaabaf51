/*
 * mrs_gb300.h -- C ABI of the GB300 (sm_103a) regularized-Stokeslet filament library.
 *
 * Method: "Accelerating Microswimmer Simulations via a Heterogeneous Pipelined
 * Parallel-in-Time Framework" -- Kirchhoff-rod filaments coupled through the Method of
 * Regularized Stokeslets (MRS), advanced in time by explicit Euler / RK2 and by Parareal.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns an int status: MRS_OK (0) or one of the MRS_E* codes below.  On an
 *    error, mrs_last_error() returns a message for the calling thread.  No call aborts the
 *    process; invalid arguments are rejected before anything is launched.
 *  - Pointers named "device" must point to device memory of the context's GPU; "host"
 *    pointers to host memory.  The CALLER owns every buffer passed in: the library never frees
 *    or retains caller memory beyond the call (plans keep only their own tables).
 *  - Point arrays are AoS, row-major: p[k*3 + c] is component c of point k.  Frames are
 *    D[k*9 + i*3 + c]: component c of director D^{i+1} of node k (rows are directors).
 *  - Independent systems (or rods) are concatenated along the point axis and delimited by
 *    CSR offsets: offsets[0] = 0 <= offsets[1] <= ... <= offsets[n] = total points.
 *  - A context (and everything created from it) is used by one host thread at a time; its plan
 *    and workspace caches are not locked.  A server (serve_*) may be driven from any thread:
 *    its scheduler runs on a thread and stream of its own.
 *  - Work is enqueued on the caller's CUDA stream (`stream`, a cudaStream_t passed as void*;
 *    NULL = the legacy default stream) and the call returns without synchronizing, except
 *    where an entry point says otherwise.
 *  - The library allocates device memory only in the plan
 *    constructors, mrs_reserve, the first call of mrs_velocity for a given problem shape (which
 *    builds and caches a plan) and the rod/Parareal/serving set-up calls -- never on a repeated
 *    call of the same shape.  Reserve or warm a shape up before capturing its calls in a CUDA
 *    graph.
 */
#ifndef MRS_GB300_H
#define MRS_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MRS_API __attribute__((visibility("default")))
#else
#define MRS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------ */
#define MRS_OK        0   /* success */
#define MRS_EINVAL    1   /* invalid argument (sizes, offsets, eps <= 0, mu <= 0, NULL, ...) */
#define MRS_ENOMEM    2   /* device or host allocation failed */
#define MRS_ECUDA     3   /* a CUDA runtime call or kernel launch failed */
#define MRS_ETIMEOUT  4   /* a bounded device-side wait ran out (the kernel returned early) */
#define MRS_ENOCONV   5   /* Parareal did not reach the tolerance, or its increment diverged */
#define MRS_EBUSY     6   /* serving: no free slot / budget for the job right now */
#define MRS_PENDING   7   /* serving: the job has not finished yet */
#define MRS_ECANCELED 8   /* serving: the job was cancelled before it was admitted */

/* ---- arithmetic of the pair sum ---------------------------------------------------------- */
#define MRS_F64       0   /* float64 inputs/outputs, float64 arithmetic */
#define MRS_F32       1   /* float32 inputs/outputs, float32 arithmetic and accumulation */
#define MRS_F32_COMP  2   /* float32 inputs/outputs, float32 arithmetic, compensated
                             (Kahan-folded per-chunk partials) per-target accumulation */

/* ---- time-stepping schemes (Section III-B) ----------------------------------------------- */
#define MRS_EULER     0   /* explicit Euler, Eqs. newx / newD (the coarse propagator G) */
#define MRS_RK2       1   /* second-order Runge-Kutta, explicit midpoint (the fine propagator F) */

typedef struct mrs_ctx mrs_ctx;
typedef struct mrs_plan mrs_plan;

/* Message of the last failed call made by this thread ("" if none).  Valid until the next call. */
MRS_API const char* mrs_last_error(void);

/* Library version string. */
MRS_API const char* mrs_version(void);

/* Create a context on CUDA device `device` (the calling thread's current device is set to it).
 * Queries the device (must be compute capability 10.3) and records SM count and limits.
 * Errors: MRS_EINVAL (no such device or wrong architecture), MRS_ECUDA. */
MRS_API int mrs_ctx_create(mrs_ctx** ctx, int device);

/* Destroy a context and every plan it still owns.  Synchronizes the device first. */
MRS_API int mrs_ctx_destroy(mrs_ctx* ctx);

/* Number of SMs of the context's device (host-side query; no GPU work). */
MRS_API int mrs_ctx_num_sms(const mrs_ctx* ctx);

/* Rod stepping path of the context (rod_step, parareal_run, parareal_run_pipelined).  The fused
 * path advances a batch of instances through all its steps in ONE launch: one CTA per instance
 * keeps the instance's state in shared memory and runs forces (with the Lennard-Jones repulsion
 * when enabled), float32 pair sum and update of every stage back to back.  The other path runs
 * every step as forces -> pair-sum plan -> update kernels replayed from captured CUDA graphs,
 * over all SMs.  mode = 1 (the default): fused for instances of at most 128 nodes in a batch of
 * more than 4096 nodes (e.g. the slices of a Parareal solve), where one SM per instance is the
 * faster choice; smaller batches take the graphs, whose warp-cooperative force and update
 * kernels (mrs_ctx_set_rod_force_kernel) are faster there; mode = 2: fused whenever the
 * instance fits shared memory
 * (at most ~600 nodes); mode = 0: never.  MRS_F64 stepping always takes the graphs.  Both paths
 * compute the same steps; results agree to float32 rounding of the pair sum.  Host only.
 * Errors: MRS_EINVAL (mode outside 0..2). */
MRS_API int mrs_ctx_set_fused_steps(mrs_ctx* ctx, int enable);

/* Rod force kernel of the context (rod_forces; rod_step, parareal_run and
 * parareal_run_pipelined on the graph path): the internal force and moment of every segment
 * and the node force and torque (Eqs. mid_triad, F_comp_discrete, N_comp_discrete,
 * discrete_f, discrete_n).  GB300 executes a float64 warp instruction in about 64 cycles per
 * scheduler whatever the number of active lanes, so a segment computed by one thread costs its
 * whole float64 path on one scheduler.  The warp-cooperative kernel spreads each segment over
 * ten lanes (three segments per warp, a fourth warp per CTA for the preferred curvature and the
 * node phase), which shortens the path per scheduler and uses more schedulers; the
 * thread-per-segment kernel does the least float64 work in all.  mode = 0 (the default):
 * warp-cooperative for batches of at most 4096 nodes, thread per segment above; 1: always one
 * thread per segment; 2: always warp-cooperative.  With the warp-cooperative kernels the frame
 * update is warp-cooperative too (nine lanes per node), and in rod stepping the small-system
 * pair sum applies it to the nodes it completes; with 1 it runs as its own thread-per-node
 * kernel.  Both compute the same expressions; results agree to float64 rounding.  Takes effect for calls made afterwards (captured step graphs are
 * kept per setting).  Host only.  Errors: MRS_EINVAL (mode outside 0..2). */
MRS_API int mrs_ctx_set_rod_force_kernel(mrs_ctx* ctx, int mode);

/* Largest column-partial buffer of one pass of a symmetric pair-sum plan (configurations
 * 17..26; see mrs_plan_create), in bytes, for plans created from then on.  A plan whose column
 * partials -- 24 bytes per source slot of every work unit, about N^2 / (2 TM) * 24 bytes for one
 * system of N points -- exceed it runs as several passes of about equal work over consecutive
 * tiles, each one launch of the pair kernel and one of the reduction kernel, reusing one buffer
 * (plus 48 bytes per point to carry sums between passes).  Default 192 MiB: the 32768-point
 * system (34 MB) runs in one pass, a 2^18-point one (2.1 GB) in 11 with under 256 MB of
 * scratch in all, the 512-system batch of 256..16384-point systems (515 MB) in 3.  Each further pass costs about 60 us on a GB300 (the
 * tail of one more persistent launch and one more reduction).  A pass holds at least one tile
 * row, so its buffer may exceed the setting by up to one row (N / 32 units).  Host only.
 * Errors: MRS_EINVAL (fewer bytes than one work unit's partials, 768). */
MRS_API int mrs_ctx_set_sym_pass_bytes(mrs_ctx* ctx, size_t bytes);

/* Measurement aid (the paper has no counterpart): FP32 FMA-pipe throughput of the device, in
 * TFLOP/s (2 flops per lane FMA), for kind 0: scalar FFMA, 1: packed FFMA2 (fma.rn.f32x2, the
 * form the pair-sum kernels use), 2: the two interleaved, 3: float64 DFMA (the pipe the rod
 * kernels are bound by), 4: float64 DFMA on lane 0 of each warp only (the flops of that one lane
 * are counted; kind 3 / kind 4 near 32 means a DFMA costs the same whatever the active mask).
 * One launch in which every (active) thread runs 8 independent chains of `iters`
 * steps (two FP32 lane FMAs, or one DFMA, per chain and step): warps_per_scheduler = 0 fills
 * every thread slot of the device; w >= 1 runs w warps on each scheduler of each SM (the
 * pair-sum kernel runs 2).  Timed with CUDA events after a warm-up launch; *ms (may be NULL)
 * gets the launch's time.  Allocates and frees a small buffer and synchronizes the device.
 * Errors: MRS_EINVAL, MRS_ENOMEM, MRS_ECUDA. */
MRS_API int mrs_fma_probe(int device, int kind, int iters, int warps_per_scheduler,
                          double* tflops, float* ms);

/* Device-side anomaly flags raised by the pair-sum kernels of this context since the last call
 * (MRS_FLAG_NONFINITE: a non-finite u or omega was written, e.g. from non-finite inputs).
 * Synchronizes the device, returns the flags in *flags and clears them. */
#define MRS_FLAG_NONFINITE 1u
#define MRS_FLAG_BOUNDS    2u   /* debug build only: a work-table or node-table index was out of
                                   range; the access was skipped (results are then invalid) */
MRS_API int mrs_device_status(mrs_ctx* ctx, unsigned int* flags);

/* ==========================================================================================
 * MRS pair sum -- Section II-C, Eqs. (velocity_field), (angular_velocity_field),
 * (superposition); Section III-C-2.
 *
 * For every target i of system s and every source j of the same system (the self pair
 * included; every kernel is finite at r = 0):
 *     u_i     = (1/mu) sum_j [ f_j H1 + (f_j.r) r H2 + (n_j x r) H3 ]
 *     omega_i = (1/mu) sum_j [ (f_j x r) H3 + n_j H4 + (n_j.r) r H5 ],    r = x_i - X_j,
 * with the regularized kernels of the blob phi_eps(r) = 15 eps^4 / (8 pi (r^2+eps^2)^{7/2}):
 *     H1 = (r^2+2e^2)/(8 pi d^{3/2}),  H2 = 1/(8 pi d^{3/2}),  H3 = (2r^2+5e^2)/(16 pi d^{5/2}),
 *     H4 = (10e^4-7e^2r^2-2r^4)/(32 pi d^{7/2}),  H5 = (6r^2+21e^2)/(32 pi d^{7/2}),
 * d = r^2 + eps^2 (H1, H2 as in the paper's cited source; H3..H5 from omega = curl(u)/2).
 * ========================================================================================== */

/* One call of the pair sum over n_sys independent systems.
 *   offsets      host int64[n_sys+1], CSR point offsets (system s = points offsets[s]..offsets[s+1])
 *   X, f, n      device [N][3] source positions, forces, torques (N = offsets[n_sys]);
 *                float32 for MRS_F32 / MRS_F32_COMP, float64 for MRS_F64
 *   Xt           device [N][3] target positions, or NULL: targets = sources (same offsets)
 *   u, w         device [N][3] outputs (overwritten), same type as the inputs; must not
 *                overlap any input
 *   mu, eps      viscosity (> 0) and regularisation (> 0) for every system ...
 *   eps_per_sys  ... unless non-NULL: host double[n_sys], one eps (> 0) per system
 *   precision    MRS_F64 | MRS_F32 | MRS_F32_COMP
 * The first call for a given (offsets, eps, precision, mu) builds a plan (device tables and
 * scratch) and caches it in the context; later calls with the same shape allocate nothing.
 * Calls that share a cached plan must not overlap on the GPU (issue them on one stream).
 * Empty systems are allowed; N = 0 is a no-op.
 * Errors: MRS_EINVAL (offsets not monotone, eps/mu <= 0, NULL pointers, bad precision),
 *         MRS_ENOMEM, MRS_ECUDA. */
MRS_API int mrs_velocity(mrs_ctx* ctx, int n_sys, const int64_t* offsets,
                 const void* X, const void* f, const void* n, const void* Xt,
                 void* u, void* w, double mu, double eps, const double* eps_per_sys,
                 int precision, void* stream);

/* Builds and caches, without launching anything, the plan mrs_velocity uses for the shape
 * (offsets, mu, eps or eps_per_sys, precision) -- its work table and scratch -- so that later
 * mrs_velocity calls with that shape allocate nothing and may be captured in a CUDA graph.
 * Call it off the hot path, once per shape; a shape already cached is only marked as the most
 * recently used.  The context caches up to 16 shapes (the least recently used is evicted,
 * after a device synchronisation, when a 17th is reserved or used).
 * Arguments as for mrs_velocity.  Errors: MRS_EINVAL, MRS_ENOMEM, MRS_ECUDA. */
MRS_API int mrs_reserve(mrs_ctx* ctx, int n_sys, const int64_t* offsets, double mu, double eps,
                        const double* eps_per_sys, int precision);

/* Pair sum that allocates nothing (the paper has no counterpart: this is a library service).
 * For callers that cannot call cudaMalloc -- code whose device memory belongs to another
 * allocator or a fixed budget, latency-critical loops that cannot pay for cudaMalloc's implicit
 * device synchronisation, or code running while another component captures the stream.
 * Computes the same sum as mrs_velocity for ONE system (targets = sources), float32 with
 * compensated accumulation (MRS_F32_COMP), on the calling thread's current device:
 *   n_points     number of points, 0 <= n_points <= 1048576 (larger: MRS_EINVAL with a message)
 *   X, f, n      device float32 [n_points][3] positions, forces, torques (caller-owned)
 *   u, w         device float32 [n_points][3] outputs (caller-owned, overwritten)
 *   mu, eps      viscosity (> 0) and regularisation (> 0)
 * Scratch (work table, partial results, tile counters) lives in a fixed ~9.1 MiB __device__
 * array that every GPU loading the library holds until the process exits.  The FIRST call on a
 * device looks up that array's device address (cudaGetSymbolAddress) and the device's SM count;
 * make that first call before any stream capture.  No call allocates or frees memory.  Every
 * call shares the one array and each call re-initialises what must start at zero, so calls
 * whose GPU work overlaps (other streams, other host threads) race and give wrong results:
 * issue them on one stream.  The array's address is remembered per device ordinal for the life
 * of the process: do not call this entry point again on a device after cudaDeviceReset (or any
 * other teardown of its primary context), which reloads the module at a new address.
 * Non-finite inputs are NOT reported: unlike mrs_velocity, no flag reaches mrs_device_status
 * (there is no context); the NaN/Inf shows up in u and w instead.
 * Errors: MRS_EINVAL (size, mu, eps, NULL, outputs overlapping inputs or each other, pointers
 *         not 4-byte aligned -- all checked before any launch), MRS_ECUDA. */
MRS_API int mrs_velocity_noalloc(int64_t n_points, const float* X, const float* f, const float* n,
                                 float* u, float* w, double mu, double eps, void* stream);

/* Explicit plans: build once, then execute many times (e.g. inside a CUDA graph).
 *   config  -1: the library's choice (tuned table or heuristic); otherwise an index into
 *           mrs_plan_config_count() kernel configurations (tile shape / targets per thread).
 *           Configurations 17..26 are symmetric: when the targets are the sources (Xt NULL
 *           or equal to X) each unordered pair {i, j} is evaluated once and serves both points
 *           (the kernel values depend on |r| only and the reversed pair has separation -r),
 *           and execution launches the persistent pair kernel plus a small deterministic
 *           reduction kernel; with other targets such a plan runs an ordered configuration.
 *           Their column partials hold one 6-vector per source slot of every work unit (about
 *           N^2 / (2 TM) * 24 bytes for one system of N points, TM = threads x points per
 *           thread of the configuration: 384 for the default symmetric one, up to 1536); beyond
 *           the context's pass size (mrs_ctx_set_sym_pass_bytes) the plan runs in passes.
 *           Configurations 27 and 28 are the small-system cluster kernel (ordered): one
 *           thread-block cluster of up to 16 CTAs per tile of 32 (27) or 64 (28) targets, each
 *           CTA over a share of the tile's sources split among 8 (4) thread groups, the CTAs'
 *           partials summed through distributed shared memory in rank order (deterministic, no
 *           scratch).  The cluster size is the largest for which all tiles' clusters are
 *           resident at once.  The library's choice for a few systems of up to 2560 points.
 * A plan owns device tables and scratch; mrs_plan_execute allocates nothing and launches one
 * kernel (the persistent or cluster pair kernel, plus the reduction kernel for a symmetric
 * configuration; for MRS_F64 one plain kernel).  Executions of the same plan must not overlap on the GPU.  Arguments as for
 * mrs_velocity. */
MRS_API int mrs_plan_create(mrs_ctx* ctx, int n_sys, const int64_t* offsets, double mu, double eps,
                    const double* eps_per_sys, int precision, int config, mrs_plan** plan);
MRS_API int mrs_plan_execute(mrs_plan* plan, const void* X, const void* f, const void* n,
                     const void* Xt, void* u, void* w, void* stream);
MRS_API int mrs_plan_destroy(mrs_plan* plan);
/* Passes a plan's execution runs (1 unless a symmetric plan's column partials exceed the
 * context's pass size) and the bytes of partial-sum scratch it holds.  Either output may be
 * NULL.  Host only.  Errors: MRS_EINVAL. */
MRS_API int mrs_plan_scratch(const mrs_plan* plan, int* passes, size_t* scratch_bytes);

/* Autotuner: time every kernel configuration on this batch shape (synthetic inputs generated
 * on the device; temporary buffers allocated and freed here), `reps` timed runs each, and
 * remember the fastest for the shape's bucket (precision, log2 of #systems, of total points and
 * of the largest system) in the context; plans created with config = -1 then use it.
 * Float32 precisions only.  Synchronizes the device.  Outputs (host) may be NULL.
 * Errors: MRS_EINVAL, MRS_ENOMEM, MRS_ECUDA. */
MRS_API int mrs_autotune(mrs_ctx* ctx, int n_sys, const int64_t* offsets, double mu, double eps,
                         const double* eps_per_sys, int precision, int reps, int* best_config,
                         float* best_ms);
/* Write / read the context's tuning table as JSON (tied to the device architecture). */
MRS_API int mrs_autotune_save(const mrs_ctx* ctx, const char* path);
MRS_API int mrs_autotune_load(mrs_ctx* ctx, const char* path);

/* Kernel configurations available to plans: count, and a description of entry `config`
 * (threads per CTA, targets per thread, CTAs resident per SM on this device). */
MRS_API int mrs_plan_config_count(void);
/* 1 if configuration `config` is symmetric (each unordered pair once; see mrs_plan_create),
 * 0 if it is ordered, -1 if it is out of range.  Host only; no device call. */
MRS_API int mrs_plan_config_symmetric(int config);
MRS_API int mrs_plan_config_info(mrs_ctx* ctx, int config, int* threads, int* targets_per_thread,
                         int* ctas_per_sm);
/* Grid size (persistent CTAs) and total work units of a plan, for reporting. */
MRS_API int mrs_plan_info(const mrs_plan* plan, int* grid, int64_t* work_units, int* config);

/* ==========================================================================================
 * Kirchhoff rods -- Sections II-A, II-B (Eqs. discrete_f, discrete_n, F_comp_discrete,
 * N_comp_discrete, mid_triad), Section III-C-1 (rotation square root), Section IV-A
 * (preferred strain-twist wave).
 * ========================================================================================== */
typedef struct {
    double L;          /* rod length; ds = L/(M-1) for a rod of M nodes */
    double a[3];       /* bending moduli a1, a2 and torsional rigidity a3 */
    double b[3];       /* shear moduli b1, b2 and stretching stiffness b3 */
    double wave_A;     /* amplitude A of Omega_2 = -k^2 A sin(k s + f t) */
    double wave_k;     /* wavenumber k = 2 pi / lambda */
    double wave_f;     /* frequency f */
    double mu;         /* viscosity used by rod_step / parareal_run */
    double eps;        /* MRS regularisation used by rod_step / parareal_run */
    double lj_eps;     /* Lennard-Jones well depth between rods (Section IV-A); 0 = no repulsion */
    double lj_sigma;   /* Lennard-Jones length sigma, cut at 2^{1/6} sigma; <= 0 selects the
                          paper's 3 eps (then eps must be > 0 when lj_eps > 0) */
} mrs_rod_params;

/* Point force g_k and torque m_k that every node applies to the fluid at time t (plus, when
 * p->lj_eps > 0, the Lennard-Jones repulsion 24 e [2 (s/r)^12 - (s/r)^6] r_vec / r^2 from every
 * node of another rod closer than 2^{1/6} s, added to g_k -- reading of Section IV-A):
 * g_k = F_{k+1/2} - F_{k-1/2},  m_k = N_{k+1/2} - N_{k-1/2}
 *        + (1/2)[(X_{k+1}-X_k) x F_{k+1/2} + (X_k-X_{k-1}) x F_{k-1/2}]
 * (the negatives of the fluid-on-rod densities of Eqs. discrete_f / discrete_n times ds),
 * with the mid-segment frame D_{k+1/2} = A_k^{1/2} D_k computed in float64 on the GPU.
 * Free ends: no internal force or moment beyond the first and last node.
 *   rod_off  host int64[n_rods+1] node offsets; every rod has 2..4096 nodes
 *   X, D     device float64 [N][3], [N][3][3];  g, m  device float64 [N][3] (outputs)
 * Errors: MRS_EINVAL, MRS_ECUDA. */
MRS_API int rod_forces(mrs_ctx* ctx, int n_rods, const int64_t* rod_off, const mrs_rod_params* p,
               const double* X, const double* D, double t, double* g, double* m, void* stream);

/* One explicit update (Eqs. newx, newD) with given velocities: X_k += u_k dt and every director
 * of node k rotated by |w_k| dt about w_k (unchanged where w_k = 0), in place.
 *   X, D   device float64 [N][3], [N][3][3];  u, w  device [N][3], float32 (vel_f64 = 0) or
 *   float64 (vel_f64 = 1).  Errors: MRS_EINVAL, MRS_ECUDA. */
MRS_API int rod_advance(mrs_ctx* ctx, int64_t N, double* X, double* D, const void* u, const void* w,
                        double dt, int vel_f64, void* stream);

/* nsteps explicit time steps of all rods as ONE hydrodynamic system (every node is a source
 * for every node), in place on device float64 X[N][3], D[N][3][3], from time t0 with step dt.
 * Each stage: rod_forces -> float32 pack -> MRS pair sum (mrs_precision) -> float64 update
 * (Eq. newx; Eq. newD Rodrigues rotation of the frame by |omega| dt about omega).  The float32
 * packs hold positions relative to a reference point of the current state (the mean of the
 * middle nodes of up to 8 rods), so the pair sum's accuracy does not depend on where the
 * system sits; results do not depend on how a run is split into calls.
 * scheme MRS_EULER or MRS_RK2 (explicit midpoint on positions and frames).  The steps replay
 * from CUDA graphs captured once per (rods, scheme).  For systems of up to 4096 nodes they use
 * the warp-cooperative force kernel, and the small-system pair sum applies the update itself:
 * two launches per stage (mrs_ctx_set_rod_force_kernel).  A system takes the fused one-launch
 * path (mrs_ctx_set_fused_steps) only when the fused-steps mode is 2, or when it has at most
 * 128 nodes and the force-kernel setting is 1.  Synchronizes `stream`
 * only at set-up.  Errors: MRS_EINVAL, MRS_ENOMEM, MRS_ECUDA. */
MRS_API int rod_step(mrs_ctx* ctx, int n_rods, const int64_t* rod_off, const mrs_rod_params* p,
             double* X, double* D, double t0, double dt, int nsteps, int scheme,
             int mrs_precision, void* stream);

/* Principal square root S (S^2 = R, rotation angle halved about the same axis) of n rotation
 * matrices (Section III-C-1, Eqs. rodrigues / halfangle), float64, device R[n][3][3] ->
 * S[n][3][3] (row-major).  Computed through the quaternion q of R and the half-angle
 * quaternion (1+q)/|1+q|, normalised once by its full norm; at an angle of exactly pi either
 * quarter turn is returned.
 * Errors: MRS_EINVAL, MRS_ECUDA. */
MRS_API int rot_sqrt_batch(mrs_ctx* ctx, int n, const double* R, double* S, void* stream);

/* Checkpoint / resume of a rod system (no counterpart in the paper; Parareal slice states and
 * long runs restart from one).  Saves t, the rod offsets, X [N][3] and D [N][3][3] (float64,
 * device or host pointers) with a hash; load checks magic, version, sizes, offsets and hash
 * before writing X, D (device or host) and *t.  Both synchronize `stream`.
 * Errors: MRS_EINVAL (I/O, mismatch, corruption), MRS_ECUDA. */
MRS_API int rod_checkpoint_save(const char* path, int n_rods, const int64_t* rod_off,
                                const double* X, const double* D, double t, void* stream);
MRS_API int rod_checkpoint_load(const char* path, int n_rods, const int64_t* rod_off, double* X,
                                double* D, double* t, void* stream);

/* ==========================================================================================
 * Parareal -- Section II-D, Eqs. (initial), (intermediate), (serial_correct); Eq. (true_err).
 * ========================================================================================== */
typedef struct {
    int iterations;          /* Parareal iterations k performed */
    double incr[64];         /* relative increment eta~^k (Eq. true_err) for k = 1..iterations */
    double final_incr;       /* eta~ of the last iteration */
    double seconds;          /* wall time of the call */
    int64_t fine_steps;      /* fine RK2 steps executed (all slices, all iterations) */
    int64_t coarse_steps;    /* coarse Euler steps executed */
} mrs_parareal_stats;

/* Parareal over [T0, T1] split into n_slices equal slices on ONE GPU: coarse G = Euler with
 * step coarse_ratio*dt_fine, fine F = RK2 with step dt_fine; every iteration runs the fine
 * solves of all open slices together as independent systems of one batched launch per stage,
 * then the serial correction X^k_n = F' + G(X^k_{n-1}) - G(X^{k-1}_{n-1}) in float64 with
 * polar re-orthonormalisation of the frames.  Stops when eta~^k < tol or after max_iter
 * iterations.  On return X, D (device float64) hold the state at T1.  Synchronizes `stream`.
 *   out  host, may be NULL.
 * Errors: MRS_EINVAL, MRS_ENOMEM, MRS_ECUDA, MRS_ENOCONV (tolerance not reached within
 * max_iter, or a non-finite increment; X, D then hold the last iterate). */
MRS_API int parareal_run(mrs_ctx* ctx, int n_rods, const int64_t* rod_off, const mrs_rod_params* p,
                 double* X, double* D, double T0, double T1, int n_slices, double dt_fine,
                 int coarse_ratio, int max_iter, double tol, mrs_parareal_stats* out,
                 void* stream);

/* The pipelined schedule of Section III-A on one GPU: same iteration and same result as
 * parareal_run, but the slices are cut into groups of group_size consecutive slices whose fine
 * solves run on their own streams and start as soon as the previous correction sweep has
 * produced their input states (the sweep streams its results downstream), overlapping the
 * serial coarse/correction sweep with fine work.  The next iteration's fine solves are queued
 * before the current increment is known; if the current iteration converges, that work is
 * discarded.  When either (second iteration) the first increment is below 1000 tol or (from
 * the third iteration on) the last two increments extrapolate geometrically below tol, the
 * current increment is read first and the next fine solves are queued only if needed.  All ordering
 * is by CUDA events between streams (no device-side waiting).
 * Arguments, outputs and errors as for parareal_run; group_size in 1..n_slices. */
MRS_API int parareal_run_pipelined(mrs_ctx* ctx, int n_rods, const int64_t* rod_off,
                                   const mrs_rod_params* p, double* X, double* D, double T0,
                                   double T1, int n_slices, double dt_fine, int coarse_ratio,
                                   int max_iter, double tol, int group_size,
                                   mrs_parareal_stats* out, void* stream);

/* ==========================================================================================
 * Serving -- continuous batching of pair-sum and rod-integration jobs on one GPU.
 * (The paper has no serving layer; this is the library's request loop around the method.)
 *
 * A server owns one CUDA stream, a device memory pool of hbm_budget_bytes and a scheduler
 * thread.  Jobs are admitted, in submission order, as soon as a slot (max_slots) and pool
 * memory for their footprint are free.  Every scheduler iteration advances admitted jobs by
 * one stage -- a velocity job is one stage, a rod job one stage per Euler step (two per RK2
 * step) -- and the pair sums of all of them run as ONE persistent kernel launch, so jobs
 * that arrive while others are on the GPU join the next iteration and their work overlaps.
 * Which admitted jobs an iteration advances (serve_set_policy): every "small" job, and the
 * oldest "big" one(s), a job being big when its total pair work (n_points^2 per stage times
 * its stages) reaches a threshold.  Big jobs thus run one after another in admission order,
 * as they would one request per launch, and small jobs never wait behind them.
 * Inputs are copied into the pool when the job is admitted and results are copied out when
 * it finishes; the caller's buffers must stay valid and unmodified until serve_poll reports
 * the job done.
 * ========================================================================================== */
typedef struct mrs_server mrs_server;

#define MRS_JOB_VELOCITY 0   /* one mrs_velocity (float32, compensated) of one system */
#define MRS_JOB_ROD      1   /* nsteps rod_step steps of one system of rods */

typedef struct {
    int kind;                 /* MRS_JOB_VELOCITY | MRS_JOB_ROD */
    int64_t n_points;         /* points (velocity job) or nodes of all rods (rod job), >= 1 */
    double mu, eps;           /* viscosity and regularisation of the job's system (> 0) */
    /* velocity job: device float32 [n_points][3] inputs and outputs */
    const float* X;
    const float* f;
    const float* n;
    float* u;
    float* w;
    /* rod job: host rod offsets (n_rods+1, copied at submit), device float64 state advanced in
     * place (X [n_points][3], D [n_points][3][3]); params.mu/eps are ignored (mu, eps above) */
    int n_rods;
    const int64_t* rod_off;
    double* Xr;
    double* Dr;
    mrs_rod_params params;
    double t0, dt;
    int nsteps;
    int scheme;               /* MRS_EULER | MRS_RK2 */
} mrs_job;

/* Create a server on the context's device: pool of hbm_budget_bytes (allocated here, once),
 * at most max_slots jobs admitted at a time.  Errors: MRS_EINVAL, MRS_ENOMEM, MRS_ECUDA. */
MRS_API int serve_create(mrs_server** srv, mrs_ctx* ctx, size_t hbm_budget_bytes, int max_slots);

/* Queue a job (host call, never blocks on the GPU).  *ticket identifies it for serve_poll.
 * Errors: MRS_EINVAL (bad sizes/pointers), MRS_EBUSY (the job alone exceeds the pool). */
MRS_API int serve_submit(mrs_server* srv, const mrs_job* job, uint64_t* ticket);

/* Non-blocking status: *done = 1 and *latency_s = completion time - submit time once the job
 * has finished and its results are in the caller's buffers; returns MRS_PENDING (done = 0)
 * while it is queued or running, MRS_OK when done, or the job's error status. */
MRS_API int serve_poll(mrs_server* srv, uint64_t ticket, int* done, double* latency_s);

/* Cancel a job that has not been admitted yet: it finishes with status MRS_ECANCELED and its
 * buffers are never touched.  Errors: MRS_EBUSY (already admitted, it will run to completion),
 * MRS_EINVAL (unknown or finished ticket). */
MRS_API int serve_cancel(mrs_server* srv, uint64_t ticket);

/* Block until every submitted job has finished (or timeout_s seconds pass: MRS_ETIMEOUT). */
MRS_API int serve_drain(mrs_server* srv, double timeout_s);

/* Counters: iterations run, jobs completed, pair interactions computed, peak jobs admitted at
 * once, peak pool bytes in use, and the iterations whose batched pair sum ran the symmetric
 * kernel (each unordered pair once; the others ran the ordered kernel because the iteration's
 * partial sums did not fit the server's scratch: 3 % of hbm_budget_bytes, at most 3 GiB, carved
 * from the budget).  Any output pointer may be NULL. */
MRS_API int serve_stats(mrs_server* srv, int64_t* iterations, int64_t* completed, double* pairs,
                        int* peak_active, size_t* peak_pool_bytes, int64_t* symmetric_iterations);

/* Scheduling policy (host call; applies to jobs admitted from then on).  A job whose total pair
 * work n_points^2 x stages is at least big_job_pairs is "big": each iteration advances all
 * small jobs and only the max_big_jobs oldest big ones.  Default: 1.3e10 pair interactions
 * (about 20 ms of the pair-sum kernel on a GB300) and 1 big job.  big_job_pairs <= 0 makes
 * every job small (every admitted job advances in every iteration).
 * Errors: MRS_EINVAL (non-finite threshold, max_big_jobs outside 1..4096). */
MRS_API int serve_set_policy(mrs_server* srv, double big_job_pairs, int max_big_jobs);

/* Fault injection for tests (no GPU involvement): the admission of the waiting job `ticket`
 * fails as a pool allocation failure would -- the job finishes with MRS_ENOMEM without
 * touching its buffers or the GPU, and the other jobs are unaffected.
 * Errors: MRS_EINVAL (unknown ticket), MRS_EBUSY (the job is no longer waiting). */
MRS_API int serve_inject_alloc_failure(mrs_server* srv, uint64_t ticket);

/* Stop the scheduler (after the queued work finishes) and free the pool. */
MRS_API int serve_destroy(mrs_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* MRS_GB300_H */
