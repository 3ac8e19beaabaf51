// rod_kernels.cu -- float64 Kirchhoff-rod kernels on sm_103a.
//
// Sections II-A, II-B: Eqs. (discrete_f), (discrete_n), (F_comp_discrete), (N_comp_discrete),
// (mid_triad); Section III-C-1 (rotation square root); Section III-C-3: Eqs. (newx), (newD);
// Section IV-A (preferred strain-twist wave).
//
// Layout: node k of the whole batch (all instances, all rods) is one row; X[k*3+c],
// D[k*9 + i*3 + c] (row i = director D^{i+1}).  node_info[k] = (index of k within its rod,
// number of nodes of its rod); segment k+1/2 exists when the index is below M-1 and is
// stored at row k of the segment buffer FN (F_{k+1/2} then N_{k+1/2}, 6 doubles).
//
// Mid-segment frame: A_k = D_{k+1}^T D_k (= sum_j D^j_{k+1} (D^j_k)^T) is turned into its unit
// quaternion q (Shepperd's pivoted formula), the principal square root is the quaternion
// (1 + q)/|1 + q| (q taken with a non-negative scalar part), and each director of D_k is
// rotated by it.  This is the same principal root as the half-angle Rodrigues form of the
// paper, reached without trigonometric calls or endpoint branches.
#include <cmath>

#include "mrs_checks.h"
#include "rod_internal.h"
#include "rod_update.cuh"

namespace mrs {

// Debug build: a node table entry outside its rod raises MRS_FLAG_BOUNDS and the node is
// skipped (returns false).
__device__ __forceinline__ bool node_checked(const RodLaunch& L, int2 ni, long long k, long long N)
{
#if MRS_DEBUG_BOUNDS
    if (!rod_node_ok(ni, k, N)) {
        if (L.err) atomicOr(L.err, MRS_FLAG_BOUNDS);
        return false;
    }
#endif
    return true;
}

__device__ __forceinline__ double dot3(const double* a, const double* b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Quaternion (w, x, y, z) of a rotation matrix A (row-major), w >= 0, of unit length up to the
// rounding of A (not normalised: its one user normalises the half-angle quaternion instead).
__device__ __forceinline__ void rot_to_quat(const double* A, double* q)
{
    // each branch: r = sqrt(x) and 1/(2r) from one reciprocal square root (x >= 1 on the
    // branch taken, so no zero division)
    const double tr = A[0] + A[4] + A[8];
    if (tr >= A[0] && tr >= A[4] && tr >= A[8]) {
        const double x = fmax(1.0 + tr, 0.0), ir = rsqrt(x);
        const double s = 0.5 * ir;
        q[0] = 0.5 * x * ir;
        q[1] = (A[7] - A[5]) * s;
        q[2] = (A[2] - A[6]) * s;
        q[3] = (A[3] - A[1]) * s;
    } else if (A[0] >= A[4] && A[0] >= A[8]) {
        const double x = fmax(1.0 + A[0] - A[4] - A[8], 0.0), ir = rsqrt(x);
        const double s = 0.5 * ir;
        q[1] = 0.5 * x * ir;
        q[0] = (A[7] - A[5]) * s;
        q[2] = (A[1] + A[3]) * s;
        q[3] = (A[2] + A[6]) * s;
    } else if (A[4] >= A[8]) {
        const double x = fmax(1.0 - A[0] + A[4] - A[8], 0.0), ir = rsqrt(x);
        const double s = 0.5 * ir;
        q[2] = 0.5 * x * ir;
        q[0] = (A[2] - A[6]) * s;
        q[1] = (A[1] + A[3]) * s;
        q[3] = (A[5] + A[7]) * s;
    } else {
        const double x = fmax(1.0 - A[0] - A[4] + A[8], 0.0), ir = rsqrt(x);
        const double s = 0.5 * ir;
        q[3] = 0.5 * x * ir;
        q[0] = (A[3] - A[1]) * s;
        q[1] = (A[2] + A[6]) * s;
        q[2] = (A[5] + A[7]) * s;
    }
    if (q[0] < 0.0) {
        q[0] = -q[0];
        q[1] = -q[1];
        q[2] = -q[2];
        q[3] = -q[3];
    }
}

// Rotation matrix (row-major) of the principal square root of the rotation A.
__device__ void rot_sqrt_dev(const double* A, double* S)
{
    double q[4];
    rot_to_quat(A, q);
    // half-angle quaternion (1 + q) / |1 + q|, the norm taken in full so that S is a rotation to
    // rounding whether or not |q| = 1 exactly (one reciprocal square root for both
    // normalisations; for a unit q, |1 + q|^2 = 2 (1 + w))
    const double w1 = 1.0 + q[0];
    const double inv = rsqrt(w1 * w1 + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const double a = w1 * inv, b = q[1] * inv, c = q[2] * inv, d = q[3] * inv;
    S[0] = 1.0 - 2.0 * (c * c + d * d);
    S[1] = 2.0 * (b * c - a * d);
    S[2] = 2.0 * (b * d + a * c);
    S[3] = 2.0 * (b * c + a * d);
    S[4] = 1.0 - 2.0 * (b * b + d * d);
    S[5] = 2.0 * (c * d - a * b);
    S[6] = 2.0 * (b * d - a * c);
    S[7] = 2.0 * (c * d + a * b);
    S[8] = 1.0 - 2.0 * (b * b + c * c);
}

__global__ void rot_sqrt_batch_kernel(int n, const double* R, double* S)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rot_sqrt_dev(R + 9 * (size_t)i, S + 9 * (size_t)i);
}

// Segment k+1/2 (Xk, Dk point at node k, node k+1 follows; ids = 1/ds of its rod; om2 = the
// preferred curvature Omega_2 of Section IV-A at the segment midpoint and the current time):
// internal force F and moment N in lab coordinates (Eqs. mid_triad, F_comp_discrete,
// N_comp_discrete), written to o[0..5].
__device__ __forceinline__ void segment_core(const mrs_rod_params& P, const double* Xk,
                                             const double* Dk, double ids, double om2, double* o)
{
    const double* Dk1 = Dk + 9;
    double A[9], S[9], Dh[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            A[3 * r + c] = Dk1[r] * Dk[c] + Dk1[3 + r] * Dk[3 + c] + Dk1[6 + r] * Dk[6 + c];
    rot_sqrt_dev(A, S);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int r = 0; r < 3; ++r)
            Dh[3 * i + r] = S[3 * r] * Dk[3 * i] + S[3 * r + 1] * Dk[3 * i + 1] + S[3 * r + 2] * Dk[3 * i + 2];
    const double e[3] = {(Xk[3] - Xk[0]) * ids, (Xk[4] - Xk[1]) * ids, (Xk[5] - Xk[2]) * ids};
    double F[3] = {0, 0, 0}, Nm[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double Fi = P.b[i] * (dot3(e, Dh + 3 * i) - (i == 2 ? 1.0 : 0.0));
        const int j = (i + 1) % 3, l = (i + 2) % 3;
        const double dD[3] = {Dk1[3 * j] - Dk[3 * j], Dk1[3 * j + 1] - Dk[3 * j + 1],
                              Dk1[3 * j + 2] - Dk[3 * j + 2]};
        const double Ni = P.a[i] * (dot3(dD, Dh + 3 * l) * ids - (i == 1 ? om2 : 0.0));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            F[c] += Fi * Dh[3 * i + c];
            Nm[c] += Ni * Dh[3 * i + c];
        }
    }
    o[0] = F[0];
    o[1] = F[1];
    o[2] = F[2];
    o[3] = Nm[0];
    o[4] = Nm[1];
    o[5] = Nm[2];
}

// Segment k+1/2 of the batch (index idx within a rod of M nodes) at the current step's time
// (+ t_off).
// sc: (sin, cos) of f t for this segment's instance when L.segsc is given (the caller's CTA
// computed them once), else NULL.
__device__ void segment_fn(const RodLaunch& L, const double* __restrict__ X,
                           const double* __restrict__ D, double t_off, long long k, int idx, int M,
                           double* o, const double* sc = nullptr)
{
    const double ids = (double)(M - 1) * L.inv_L;   // one division fewer per segment
    const double amp = -L.p.wave_k * L.p.wave_k * L.p.wave_A;
    double om2;
    if (sc) {   // Omega_2 = amp sin(k_w s_mid + f t) by angle addition (as the fused propagator)
        const double2 v = L.segsc[k];
        om2 = amp * (v.x * sc[1] + v.y * sc[0]);
    } else {
        const int inst = (int)(k / L.nodes_per_inst);
        const double t = L.t0[inst] + (double)(*L.step) * L.dt + t_off;
        const double s_mid = ((double)idx + 0.5) * (L.p.L / (double)(M - 1));
        om2 = amp * sin(L.p.wave_k * s_mid + L.p.wave_f * t);
    }
    segment_core(L.p, X + 3 * (size_t)k, D + 9 * (size_t)k, ids, om2, o);
}

__global__ void rod_segsc_kernel(int N, const int2* __restrict__ node_info, double wave_k, double Lrod,
                                 double2* out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int2 ni = node_info[k];
    if (ni.y < 2) return;
    const double ds = Lrod / (double)(ni.y - 1);
    double sk, ck;
    sincos(wave_k * ((double)ni.x + 0.5) * ds, &sk, &ck);   // the fused propagator's expression
    out[k] = make_double2(sk, ck);
}

__global__ void rod_segment_kernel(const RodLaunch L, const double* __restrict__ X,
                                   const double* __restrict__ D, double t_off)
{
    pdl_wait();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.N) return;
    const int2 ni = L.node_info[k];
    if (!node_checked(L, ni, k, L.N)) return;
    if (ni.x >= ni.y - 1) return;  // last node of its rod: no segment
    segment_fn(L, X, D, t_off, k, ni.x, ni.y, L.FN + 6 * (size_t)k);
}

// Node k: g_k = F_{k+1/2} - F_{k-1/2}, m_k = N_{k+1/2} - N_{k-1/2} + (1/2)(dX_{k+1/2} x F_{k+1/2}
// + dX_{k-1/2} x F_{k-1/2}) (free ends: missing segments contribute nothing; fp / fm point to the
// segments k+1/2 / k-1/2 or are NULL).  Writes the float64 outputs g64/m64 when given, and the
// float32 copies (X, g, m) the pair sum reads when Xf is given.
__device__ __forceinline__ void node_fn(const double* __restrict__ X, long long k, const double* fp,
                                        const double* fm, double* g64, double* m64, float* Xf,
                                        float* gf, float* mf, const double* ref = nullptr)
{
    const double* Xk = X + 3 * (size_t)k;
    double g[3] = {0, 0, 0}, m[3] = {0, 0, 0};
    if (fp) {  // segment k+1/2
        const double dX[3] = {Xk[3] - Xk[0], Xk[4] - Xk[1], Xk[5] - Xk[2]};
        g[0] += fp[0];
        g[1] += fp[1];
        g[2] += fp[2];
        m[0] += fp[3] + 0.5 * (dX[1] * fp[2] - dX[2] * fp[1]);
        m[1] += fp[4] + 0.5 * (dX[2] * fp[0] - dX[0] * fp[2]);
        m[2] += fp[5] + 0.5 * (dX[0] * fp[1] - dX[1] * fp[0]);
    }
    if (fm) {  // segment k-1/2
        const double dX[3] = {Xk[0] - Xk[-3], Xk[1] - Xk[-2], Xk[2] - Xk[-1]};
        g[0] -= fm[0];
        g[1] -= fm[1];
        g[2] -= fm[2];
        m[0] += -fm[3] + 0.5 * (dX[1] * fm[2] - dX[2] * fm[1]);
        m[1] += -fm[4] + 0.5 * (dX[2] * fm[0] - dX[0] * fm[2]);
        m[2] += -fm[5] + 0.5 * (dX[0] * fm[1] - dX[1] * fm[0]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (g64) {
            g64[3 * (size_t)k + c] = g[c];
            m64[3 * (size_t)k + c] = m[c];
        }
        if (Xf) {
            Xf[3 * (size_t)k + c] = (float)(ref ? Xk[c] - ref[c] : Xk[c]);
            gf[3 * (size_t)k + c] = (float)g[c];
            mf[3 * (size_t)k + c] = (float)m[c];
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Reference point of the float32 position packs.  The pair sum depends on differences of
// positions only, but rounding X to float32 moves every separation by up to |X| 2^-24, which
// against a node spacing ds is a relative error |X| 2^-24 / ds in the near-field kernels.  So the
// packs hold X - c, c the mean of a few fixed nodes of the instance (the middle node of up to 8
// rods spread over it, RodLaunch::ref) in the state being packed: a function of that state
// alone, summed in a fixed order, so every path packs the same values and how a run is split
// into calls does not change its rounding.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void pack_reference(const RodLaunch& L, const double* Xinst, double* c)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = 0; i < L.n_ref; ++i) {
        const double* x = Xinst + 3 * L.ref[i];
        s0 += x[0];
        s1 += x[1];
        s2 += x[2];
    }
    c[0] = s0 * L.ref_w;
    c[1] = s1 * L.ref_w;
    c[2] = s2 * L.ref_w;
}

__global__ void rod_node_kernel(const RodLaunch L, const double* __restrict__ X, double* g64,
                                double* m64, float* Xf, float* gf, float* mf)
{
    pdl_wait();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.N) return;
    const int2 ni = L.node_info[k];
    if (!node_checked(L, ni, k, L.N)) return;
    double ref[3];
    const bool centred = Xf && L.n_ref > 0;
    if (centred) pack_reference(L, X + 3 * (size_t)(k / L.nodes_per_inst) * L.nodes_per_inst, ref);
    node_fn(X, k, ni.x < ni.y - 1 ? L.FN + 6 * (size_t)k : nullptr,
            ni.x > 0 ? L.FN + 6 * (size_t)(k - 1) : nullptr, g64, m64, Xf, gf, mf,
            centred ? ref : nullptr);
}

// Both steps in one launch.  A CTA covers kRodChunk - 1 consecutive nodes of one rod: thread t
// computes segment base - 1 + t into shared memory, then threads 1.. emit node base + t - 1,
// whose two segments are slots t - 1 and t (chunks overlap by one segment, so every thread
// computes exactly one segment and nothing goes through global memory).  L.chunks[c] is the
// node index of chunk c's base node.
__global__ void __launch_bounds__(kRodChunk) rod_forces_fused_kernel(
    const RodLaunch L, const double* __restrict__ X, const double* __restrict__ D, double t_off,
    double* g64, double* m64, float* Xf, float* gf, float* mf)
{
    pdl_wait();
    __shared__ double sFN[kRodChunk * 6];
    __shared__ double sref[3];
    __shared__ double ssc[2];   // sin(f t), cos(f t) of the chunk's instance
    const long long k0 = L.chunks[blockIdx.x];
#if MRS_DEBUG_BOUNDS
    if (k0 < 0 || k0 >= L.N) {   // every thread reads the same chunk: the CTA leaves together
        if (threadIdx.x == 0 && L.err) atomicOr(L.err, MRS_FLAG_BOUNDS);
        return;
    }
#endif
    const int2 ni0 = L.node_info[k0];
    if (!node_checked(L, ni0, k0, L.N)) return;   // the same entry for every thread of the CTA
    const int M = ni0.y, t = threadIdx.x;
    const int s = ni0.x - 1 + t;   // segment index within the rod
    const int inst = (int)(k0 / L.nodes_per_inst);   // a chunk lies in one rod, hence in one instance
    static_assert(kRodChunk > 32, "the reference point is taken by a thread of the second warp");
    const bool centred = Xf && L.n_ref > 0;
    if (centred && t == 32) pack_reference(L, X + 3 * (size_t)inst * L.nodes_per_inst, sref);
    if (L.segsc) {
        if (t == 0) sincos(L.p.wave_f * (L.t0[inst] + (double)(*L.step) * L.dt + t_off), &ssc[0], &ssc[1]);
        __syncthreads();
    }
    if (s >= 0 && s < M - 1) segment_fn(L, X, D, t_off, k0 - 1 + t, s, M, sFN + 6 * t, L.segsc ? ssc : nullptr);
    __syncthreads();
    const int n = ni0.x + t - 1;   // node index within the rod
    if (t == 0 || n >= M) return;
    node_fn(X, k0 + t - 1, n < M - 1 ? sFN + 6 * t : nullptr, n > 0 ? sFN + 6 * (t - 1) : nullptr,
            g64, m64, Xf, gf, mf, centred ? sref : nullptr);
}

// ---------------------------------------------------------------------------------------------
// Warp-cooperative force kernel for small systems.  The float64 pipe executes one warp
// instruction in about 64 cycles per scheduler whatever the active mask, so a segment computed
// by one thread costs its ~190 float64 instructions on one scheduler, and a rod of a few
// hundred nodes keeps only a few dozen of the GPU's 608 schedulers busy.  Here the lanes of a
// warp share the arithmetic of a segment instead: a CTA covers kWNodes consecutive nodes of one
// rod (the kWNodes + 1 segments around them; chunks overlap by one segment) with four warps.
//   * warps 0..2: three segments each, ten lanes per segment (lanes 30, 31 idle).  Nine lanes
//     form A = D_{k+1} D_k^T (one entry each), the quaternion of A and the half-angle quaternion
//     are formed redundantly by every lane (the same instructions, no extra cost), nine lanes
//     form the rotation S and the mid frame Dh = S D_k, six lanes the three force and three
//     moment coefficients and then the six components of F and N (Eqs. mid_triad,
//     F_comp_discrete, N_comp_discrete; the same expressions as segment_core);
//   * warp 3: the preferred curvature Omega_2 of every segment (one lane each, in parallel with
//     the segment warps), the pack reference point, and after the segments the node force and
//     torque of the CTA's nodes (three lanes per node, one per component; node_fn's terms).
// The longest float64 path of a CTA is then about 70 instructions instead of ~230.
// ---------------------------------------------------------------------------------------------
constexpr int kWSegLanes = 10;   // lanes per segment in a segment warp
constexpr int kWSegPerWarp = 3;  // segments per segment warp
constexpr int kWSegs = kWNodes + 1;
static_assert(kWSegs == 3 * kWSegPerWarp, "three segment warps cover a chunk's segments");
static_assert(3 * kWNodes <= 32, "one lane per node component in the node phase");

struct WSeg {          // per-segment shared scratch of rod_forces_warp_kernel
    double A[9];       // D_{k+1} D_k^T
    double S[9];       // its principal square root
    double Dh[9];      // mid frame S D_k
    double q[4];       // quaternion of A (before the sign is fixed)
    double h[4];       // half-angle quaternion (a, b, c, d)
    double c[6];       // F_i (0..2), N_i (3..5)
    double FN[6];      // F (lab), N (lab)
    double om2;        // Omega_2 at the segment midpoint
};

// x with its sign flipped when neg (an exact operation, kept off the float64 pipe)
__device__ __forceinline__ double flip_if(double x, bool neg)
{
    return __longlong_as_double(__double_as_longlong(x) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
}

__device__ __forceinline__ double sel4(int i, double a, double b, double c, double d)
{
    return i == 0 ? a : i == 1 ? b : i == 2 ? c : d;
}

// Segment warps, first part: A (nine lanes); the quaternion of A and the half-angle quaternion
// (rot_to_quat and rot_sqrt_dev without branches, so that the three groups of a warp, which may
// take different branches, run one instruction stream: every lane forms the branch, x and the
// norm, lane j < 4 component j); S (nine lanes) and Dh = S D_k (nine lanes).
__device__ __forceinline__ void wseg_frame(const double* __restrict__ Dk, bool valid, int sl, WSeg& W)
{
    const double* Dk1 = Dk + 9;
    if (valid && sl < 9) {
        const int r = sl / 3, c = sl - 3 * (sl / 3);
        W.A[sl] = Dk1[r] * Dk[c] + Dk1[3 + r] * Dk[3 + c] + Dk1[6 + r] * Dk[6 + c];
    }
    __syncwarp();
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    if (valid) {
        double A[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) A[q] = W.A[q];
        const double tr = A[0] + A[4] + A[8];
        const int br = (tr >= A[0] && tr >= A[4] && tr >= A[8]) ? 0
                       : (A[0] >= A[4] && A[0] >= A[8]) ? 1
                       : (A[4] >= A[8]) ? 2 : 3;
        // x of the branch: 1 + tr, or 1 +- A0 +- A4 +- A8 with + on the branch's own entry
        const double u1 = br == 0 ? tr : flip_if(A[0], br != 1);
        const double u2 = br == 0 ? 0.0 : flip_if(A[4], br != 2);
        const double u3 = br == 0 ? 0.0 : flip_if(A[8], br != 3);
        const double x = fmax(((1.0 + u1) + u2) + u3, 0.0), ir = rsqrt(x);
        const double s = 0.5 * ir;
        if (sl < 4) {
            // component j = sl: x s on the branch's own component, else (A[p] +- A[m]) s, the
            // pair depending on {br, j} only
            const int j = sl;
            const int key = br < j ? 4 * br + j : 4 * j + br;
            const double P = j == br ? x
                             : key == 1 ? A[7] : key == 2 ? A[2] : key == 3 ? A[3]
                             : key == 6 ? A[1] : key == 7 ? A[2] : A[5];
            const double M = j == br ? 0.0
                             : key == 1 ? -A[5] : key == 2 ? -A[6] : key == 3 ? -A[1]
                             : key == 6 ? A[3] : key == 7 ? A[6] : A[7];
            W.q[j] = (P + M) * s;
        }
    }
    __syncwarp();
    if (valid) {
        // half-angle quaternion (1 + q) / |1 + q| with w >= 0: every lane the norm, lane j < 4
        // component j
        const bool ng = W.q[0] < 0.0;
        const double q0 = flip_if(W.q[0], ng), q1 = flip_if(W.q[1], ng), q2 = flip_if(W.q[2], ng),
                     q3 = flip_if(W.q[3], ng);
        const double w1 = 1.0 + q0;
        const double inv = rsqrt(w1 * w1 + q1 * q1 + q2 * q2 + q3 * q3);
        if (sl < 4) W.h[sl] = (sl == 0 ? w1 : sl == 1 ? q1 : sl == 2 ? q2 : q3) * inv;
    }
    __syncwarp();
    if (valid) {
        a = W.h[0];
        b = W.h[1];
        c = W.h[2];
        d = W.h[3];
    }
    if (valid && sl < 9) {
        // S[e] = alpha + beta (x1 y1 +- x2 y2) with (x1, y1, x2, y2) from (a, b, c, d):
        //   e:  0     1     2     3     4     5     6     7     8
        //      cc+dd bc-ad bd+ac bc+ad bb+dd cd-ab bd-ac cd+ab bb+cc
        // alpha = 1, beta = -2 on the diagonal, alpha = 0, beta = 2 off it (2-bit fields by e)
        const int e = sl;
        const double x1 = sel4((0x19956 >> (2 * e)) & 3, a, b, c, d);
        const double y1 = sel4((0x1fdba >> (2 * e)) & 3, a, b, c, d);
        const double x2 = sel4((0x20303 >> (2 * e)) & 3, a, b, c, d);
        const double y2 = sel4((0x267ef >> (2 * e)) & 3, a, b, c, d);
        const bool diag = e == 0 || e == 4 || e == 8;
        const double t = fma(x1, y1, flip_if(x2 * y2, (0x62 >> e) & 1));
        W.S[e] = fma(diag ? -2.0 : 2.0, t, diag ? 1.0 : 0.0);
    }
    __syncwarp();
    if (valid && sl < 9) {
        const int i = sl / 3, r = sl - 3 * (sl / 3);
        W.Dh[sl] = W.S[3 * r] * Dk[3 * i] + W.S[3 * r + 1] * Dk[3 * i + 1] + W.S[3 * r + 2] * Dk[3 * i + 2];
    }
    __syncwarp();
}

// Segment warps, second part (after Omega_2 is known): the coefficients F_i = b_i (e.Dh_i -
// delta_i3), N_i = a_i ((d_j(k+1) - d_j(k)).Dh_l / ds - delta_i2 Omega_2) (six lanes, one
// instruction stream: u = P - Q scaled before or after the dot product), then F = sum F_i Dh_i
// and N = sum N_i Dh_i (six lanes, one component each).
__device__ __forceinline__ void wseg_forces(const mrs_rod_params& P, const double* __restrict__ Xk,
                                            const double* __restrict__ Dk, double ids, bool valid,
                                            int sl, WSeg& W)
{
    if (valid && sl < 6) {
        const int i = sl % 3;
        const bool isN = sl >= 3;
        const int jd = (i + 1) % 3, l = (i + 2) % 3;
        const double* Pp = isN ? Dk + 9 + 3 * jd : Xk + 3;
        const double* Qp = isN ? Dk + 3 * jd : Xk;
        const double sc1 = isN ? 1.0 : ids, sc2 = isN ? ids : 1.0;
        const double* w = W.Dh + 3 * (isN ? l : i);
        const double u0 = (Pp[0] - Qp[0]) * sc1, u1 = (Pp[1] - Qp[1]) * sc1, u2 = (Pp[2] - Qp[2]) * sc1;
        const double dotv = u0 * w[0] + u1 * w[1] + u2 * w[2];
        const double coef = isN ? P.a[i] : P.b[i];
        const double off = isN ? (i == 1 ? W.om2 : 0.0) : (i == 2 ? 1.0 : 0.0);
        W.c[sl] = coef * (dotv * sc2 - off);
    }
    __syncwarp();
    if (valid && sl < 6) {
        const int cc = sl % 3;
        const double* cf = W.c + (sl >= 3 ? 3 : 0);
        W.FN[sl] = fma(cf[2], W.Dh[6 + cc], fma(cf[1], W.Dh[3 + cc], cf[0] * W.Dh[cc]));
    }
}

__global__ void __launch_bounds__(128) rod_forces_warp_kernel(
    const RodLaunch L, const double* __restrict__ X, const double* __restrict__ D, double t_off,
    double* g64, double* m64, float* Xf, float* gf, float* mf)
{
    pdl_wait();
    constexpr int NW = kWNodes + 2;   // the chunk's nodes and one on each side
    __shared__ WSeg sW[kWSegs];
    __shared__ double sX[NW * 3], sD[NW * 9];   // window node w = node k0 - 1 + w
    __shared__ double sRX[24];                  // positions of the pack reference nodes
    __shared__ double sref[3];
    const int4 ch = L.wchunks[blockIdx.x];   // (k0, M, b0, instance): the same for every thread
    const long long k0 = ch.x;
    const int M = ch.y, b0 = ch.z, inst = ch.w;
#if MRS_DEBUG_BOUNDS
    {
        bool bad = k0 < 0 || k0 >= L.N;
        if (!bad) {
            const int2 ni0 = L.node_info[k0];
            bad = !rod_node_ok(ni0, k0, L.N) || ni0.x != b0 || ni0.y != M ||
                  inst != (int)(k0 / L.nodes_per_inst);
        }
        if (bad) {   // every thread sees the same entry: the CTA leaves together
            if (threadIdx.x == 0 && L.err) atomicOr(L.err, MRS_FLAG_BOUNDS);
            return;
        }
    }
#endif
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double ids = (double)(M - 1) * L.inv_L;
    const bool centred = Xf && L.n_ref > 0;
    // window node w exists when b0 - 1 + w is a node of the rod
    const int wlo = b0 == 0 ? 1 : 0, whi = min(NW, M - b0 + 1);
    // one round of loads: the window's positions and frames, the reference nodes' positions
    for (int idx = threadIdx.x; idx < NW * 12; idx += blockDim.x) {
        const int wn = idx / 12, r = idx - 12 * (idx / 12);
        if (wn >= wlo && wn < whi) {
            const long long k = k0 - 1 + wn;
            if (r < 3) sX[wn * 3 + r] = X[3 * k + r];
            else sD[wn * 9 + r - 3] = D[9 * k + r - 3];
        }
    }
    if (warp == 3 && centred && lane < 3 * L.n_ref) {
        const int i = lane / 3, c = lane - 3 * (lane / 3);
        sRX[lane] = X[3 * ((size_t)inst * L.nodes_per_inst + L.ref[i]) + c];
    }
    __syncthreads();

    // segment s of the chunk is segment b0 - 1 + s of the rod (window nodes s and s + 1)
    const int g = lane / kWSegLanes, sl = lane - kWSegLanes * g;
    const int s = kWSegPerWarp * warp + g;
    const bool seg_valid = warp < 3 && g < kWSegPerWarp && b0 - 1 + s >= 0 && b0 - 1 + s < M - 1;
    const double* Xk = sX + 3 * (seg_valid ? s : 0);
    const double* Dk = sD + 9 * (seg_valid ? s : 0);

    if (warp < 3) {
        wseg_frame(Dk, seg_valid, sl, sW[g < kWSegPerWarp ? s : 0]);
    } else if (lane < kWSegs && b0 - 1 + lane >= 0 && b0 - 1 + lane < M - 1) {
        // Omega_2 of segment `lane` (segment_fn's two forms)
        const double amp = -L.p.wave_k * L.p.wave_k * L.p.wave_A;
        const double t = L.t0[inst] + (double)(*L.step) * L.dt + t_off;
        double om2;
        if (L.segsc) {
            double sft, cft;
            sincos(L.p.wave_f * t, &sft, &cft);
            const double2 v = L.segsc[k0 - 1 + lane];
            om2 = amp * (v.x * cft + v.y * sft);
        } else {
            const double s_mid = ((double)(b0 - 1 + lane) + 0.5) * (L.p.L / (double)(M - 1));
            om2 = amp * sin(L.p.wave_k * s_mid + L.p.wave_f * t);
        }
        sW[lane].om2 = om2;
    }
    __syncthreads();
    if (warp < 3) {
        wseg_forces(L.p, Xk, Dk, ids, seg_valid, sl, sW[g < kWSegPerWarp ? s : 0]);
    } else if (centred && lane < 3) {
        // pack_reference, component `lane`, summed in the same order
        double acc = 0.0;
        for (int i = 0; i < L.n_ref; ++i) acc += sRX[3 * i + lane];
        sref[lane] = acc * L.ref_w;
    }
    __syncthreads();
    if (warp != 3 || lane >= 3 * kWNodes) return;
    // node phase: node nn of the chunk (window node nn + 1), component c (node_fn's terms)
    const int nn = lane / 3, c = lane - 3 * (lane / 3);
    const int nb = b0 + nn;
    if (nb >= M) return;
    const long long k = k0 + nn;
    const double* Xn = sX + 3 * (nn + 1);
    const int c1 = c == 2 ? 0 : c + 1, c2 = c == 0 ? 2 : c - 1;
    double gv = 0.0, mv = 0.0;
    if (nb < M - 1) {   // segment k+1/2 = chunk segment nn + 1
        const double* fp = sW[nn + 1].FN;
        const double dX1 = Xn[3 + c1] - Xn[c1], dX2 = Xn[3 + c2] - Xn[c2];
        gv += fp[c];
        mv += fp[3 + c] + 0.5 * (dX1 * fp[c2] - dX2 * fp[c1]);
    }
    if (nb > 0) {       // segment k-1/2 = chunk segment nn
        const double* fm = sW[nn].FN;
        const double dX1 = Xn[c1] - Xn[c1 - 3], dX2 = Xn[c2] - Xn[c2 - 3];
        gv -= fm[c];
        mv += -fm[3 + c] + 0.5 * (dX1 * fm[c2] - dX2 * fm[c1]);
    }
    if (g64) {
        g64[3 * (size_t)k + c] = gv;
        m64[3 * (size_t)k + c] = mv;
    }
    if (Xf) {
        Xf[3 * (size_t)k + c] = (float)(centred ? Xn[c] - sref[c] : Xn[c]);
        gf[3 * (size_t)k + c] = (float)gv;
        mf[3 * (size_t)k + c] = (float)mv;
    }
}

// Eq. (newD): rotate the three directors of node k by |w| h about w / |w| (unchanged if w = 0),
// written without normalising w: with theta^2 = |w|^2 h^2,
//   D' = cos(theta) D + (sin(theta)/theta) h (w x D) + ((1 - cos(theta))/theta^2) h^2 (w.D) w,
// the two ratios taken from their Taylor series in theta^2 when theta^2 < 1e-3 (the next terms
// are below 1e-22, i.e. exact in float64) and from sincos otherwise.  Small angles -- the usual
// case, |w| dt ~ 1e-4..1e-3 -- then need no sqrt, division or trigonometric call, which matters
// because the float64 pipe bounds this kernel.
__device__ __forceinline__ void rodrigues(const double* D0, double wx, double wy, double wz,
                                          double h, double* D1)
{
    double ct, a, b;   // rodrigues_coefficients (rod_update.cuh)
    if (!rodrigues_coefficients(wx, wy, wz, h, ct, a, b)) {
#pragma unroll
        for (int q = 0; q < 9; ++q) D1[q] = D0[q];
        return;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double* v = D0 + 3 * i;
        const double wv = b * (wx * v[0] + wy * v[1] + wz * v[2]);
        const double c0 = wy * v[2] - wz * v[1];
        const double c1 = wz * v[0] - wx * v[2];
        const double c2 = wx * v[1] - wy * v[0];
        D1[3 * i + 0] = ct * v[0] + a * c0 + wv * wx;
        D1[3 * i + 1] = ct * v[1] + a * c1 + wv * wy;
        D1[3 * i + 2] = ct * v[2] + a * c2 + wv * wz;
    }
}

// (X1, D1) = (X0 + u h, Rodrigues(D0, w, h)).  X1/D1 may alias X0/D0.  When bump_step is set,
// one thread advances the step counter (after every other kernel of the step has read it).
template <typename VT>
__global__ void rod_update_kernel(const RodLaunch L, const double* X0, const double* D0,
                                  const VT* __restrict__ u, const VT* __restrict__ w,
                                  double h, double* X1, double* D1, int bump_step)
{
    pdl_wait();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (bump_step && k == 0) *L.step += 1;
    if (k >= L.N) return;
    double Dn[9], Dl[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) Dl[q] = D0[9 * (size_t)k + q];
    rodrigues(Dl, (double)w[3 * (size_t)k], (double)w[3 * (size_t)k + 1],
              (double)w[3 * (size_t)k + 2], h, Dn);
#pragma unroll
    for (int c = 0; c < 3; ++c) X1[3 * (size_t)k + c] = X0[3 * (size_t)k + c] + (double)u[3 * (size_t)k + c] * h;
#pragma unroll
    for (int q = 0; q < 9; ++q) D1[9 * (size_t)k + q] = Dn[q];
}

// Warp-cooperative update for small systems (same float64-pipe argument as
// rod_forces_warp_kernel): nine lanes per node, one entry (director i, component c) of the new
// frame each (rodrigues_entry), three nodes per warp.  Every lane of a node forms Rodrigues'
// coefficients (the same instructions, no extra cost); a lane then needs only its director's
// projection on w and one component of w x d_i.  Each lane loads everything it reads before any lane of the warp
// stores, so X1/D1 may alias X0/D0.  When bump_step is set, lane 0 of node 0 advances the step
// counter.
constexpr int kUNodesPerWarp = 3;   // nine lanes each; lanes 27..31 idle

template <typename VT>
__global__ void __launch_bounds__(128) rod_update_warp_kernel(const RodLaunch L, const double* X0,
                                                              const double* D0, const VT* __restrict__ u,
                                                              const VT* __restrict__ w, double h,
                                                              double* X1, double* D1, int bump_step)
{
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int sub = lane / 9, e = lane - 9 * (lane / 9);
    const long long k = gw * kUNodesPerWarp + sub;
    const bool active = sub < kUNodesPerWarp && k < L.N;
    if (bump_step && k == 0 && e == 0) *L.step += 1;
    const int i = e / 3, c = e - 3 * (e / 3);
    double d1 = 0.0, x1 = 0.0;
    if (active) {
        const double* v = D0 + 9 * k + 3 * i;
        d1 = rodrigues_entry(v[0], v[1], v[2], (double)w[3 * k], (double)w[3 * k + 1], (double)w[3 * k + 2],
                             h, c);
        if (e < 3) x1 = X0[3 * k + e] + (double)u[3 * k + e] * h;
    }
    __syncwarp();   // every lane of the warp has read X0/D0 before any lane stores
    if (active) {
        D1[9 * k + e] = d1;
        if (e < 3) X1[3 * k + e] = x1;
    }
}

// ---------------------------------------------------------------------------------------------
// Fused fine propagator for small systems: one CTA advances one instance (a Parareal slice, or
// the single system of a rod_step call) through all its time steps inside one launch.  The
// instance's whole state lives in shared memory -- X, D, the RK2 midpoint state, the segment
// forces, the float32 packs of positions, forces and torques, and the velocities -- and every
// stage runs the same arithmetic as the batched kernels: segment_core (rotation square root,
// internal force and moment), node_fn (node force and torque, float32 packs), the regularized
// Stokeslet pair sum over the instance's points (float32, per-target accumulation in 32-source
// chunks folded into Kahan pairs; the kernels written with d s^2 = 1 as in mrs_kernels.cu), the
// Lennard-Jones repulsion between its rods when enabled, and rodrigues (Eqs. newx, newD).  Only __syncthreads separates the phases: no launches per step.
// ---------------------------------------------------------------------------------------------
struct FusedConst {   // pair-sum constants of the instance's system (see SysConst)
    float e2, c1, c2, c3, c5, scale;
};

__device__ __forceinline__ float fused_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void fused_kahan(float& sum, float& comp, float v)
{
    const float y = __fsub_rn(v, comp);
    const float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

// Pair sum of point i over the sources [jb, je) of the instance (float32 packs in shared
// memory), in 32-source chunks whose float32 partials are folded into Kahan pairs (sum, cmp),
// both scaled by 8 pi mu (the kernels written with d s^2 = 1, as in mrs_kernels.cu).
__device__ __forceinline__ void fused_pair_range(const FusedConst& K, const float* sXf,
                                                 const float* sgf, const float* smf, int i,
                                                 int jb, int je, float* sum, float* cmp)
{
    const float xi = sXf[3 * i], yi = sXf[3 * i + 1], zi = sXf[3 * i + 2];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        sum[q] = 0.f;
        cmp[q] = 0.f;
    }
    for (int j0 = jb; j0 < je; j0 += 32) {
        const int j1 = min(je, j0 + 32);
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int j = j0; j < j1; ++j) {
            const float rx = xi - sXf[3 * j], ry = yi - sXf[3 * j + 1], rz = zi - sXf[3 * j + 2];
            const float fx = sgf[3 * j], fy = sgf[3 * j + 1], fz = sgf[3 * j + 2];
            const float nx = smf[3 * j], ny = smf[3 * j + 1], nz = smf[3 * j + 2];
            const float d = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, K.e2)));
            const float s1 = fused_rsqrt(d);
            const float s2 = s1 * s1;
            const float s3 = s1 * s2, s5 = s3 * s2;
            const float h1 = fmaf(K.e2, s3, s1);
            const float h3 = fmaf(K.c1, s5, s3);
            const float h4 = s3 * fmaf(s2, fmaf(K.c2, s2, K.c3), -0.5f);
            const float h5 = s5 * fmaf(K.c5, s2, 1.5f);
            const float bf = s3 * fmaf(fx, rx, fmaf(fy, ry, fz * rz));
            const float bn = h5 * fmaf(nx, rx, fmaf(ny, ry, nz * rz));
            const float hx = h3 * rx, hy = h3 * ry, hz = h3 * rz;
            // u += H1 f + H2 (f.r) r + H3 (n x r);  w += H3 (f x r) + H4 n + H5 (n.r) r
            acc[0] += h1 * fx + bf * rx + (ny * hz - nz * hy);
            acc[1] += h1 * fy + bf * ry + (nz * hx - nx * hz);
            acc[2] += h1 * fz + bf * rz + (nx * hy - ny * hx);
            acc[3] += h4 * nx + bn * rx + (fy * hz - fz * hy);
            acc[4] += h4 * ny + bn * ry + (fz * hx - fx * hz);
            acc[5] += h4 * nz + bn * rz + (fx * hy - fy * hx);
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) fused_kahan(sum[q], cmp[q], acc[q]);
    }
}

// Velocities (u, w) of the instance's points for the state (sXs, sDs) at time t.  sseg[k] =
// (1/ds of node k's rod, sin(k_w s_mid), cos(k_w s_mid)) for the segment k+1/2, so that
// Omega_2 = -k_w^2 A (sin(k_w s_mid) cos(f t) + cos(k_w s_mid) sin(f t)) needs one sincos per
// stage (one thread, shared through stime) instead of one sin per segment.
template <int BLOCK>
__device__ void fused_velocity(const RodLaunch& L, const FusedConst& K, int N1,
                               const int2* sni, const double* sseg, const double* sXs,
                               const double* sDs, double t, double* stime, double* sref,
                               double* sFN, float* sXf, float* sgf, float* smf, float* su, float* sw)
{
    const mrs_rod_params& P = L.p;
    const int tid = threadIdx.x;
    static_assert(BLOCK > 32, "the reference point is taken by a thread of the second warp");
    if (tid == 0) sincos(P.wave_f * t, &stime[0], &stime[1]);
    if (tid == 32) pack_reference(L, sXs, sref);   // reference point of this stage's float32 packs
    __syncthreads();
    const double sft = stime[0], cft = stime[1];
    const double amp = -P.wave_k * P.wave_k * P.wave_A;
    for (int k = tid; k < N1; k += BLOCK) {
        const int2 ni = sni[k];
        if (ni.x < ni.y - 1) {
            const double om2 = amp * (sseg[3 * k + 1] * cft + sseg[3 * k + 2] * sft);
            segment_core(P, sXs + 3 * k, sDs + 9 * k, sseg[3 * k], om2, sFN + 6 * k);
        }
    }
    __syncthreads();
    for (int k = tid; k < N1; k += BLOCK) {
        const int2 ni = sni[k];
        node_fn(sXs, k, ni.x < ni.y - 1 ? sFN + 6 * k : nullptr, ni.x > 0 ? sFN + 6 * (k - 1) : nullptr,
                nullptr, nullptr, sXf, sgf, smf, sref);
    }
    __syncthreads();
    if (P.lj_eps > 0.0) {
        // Section IV-A repulsion between nodes of different rods of the instance, as in
        // rod_lj_kernel: float32 screen against r_c^2 with a 1 % margin, float64 force for the
        // close pairs, added to the force the node applies to the fluid
        const double s2 = P.lj_sigma * P.lj_sigma;
        const double rc2 = 1.2599210498948732 * s2;            // (2^{1/6} sigma)^2
        const float rc2f = (float)(1.01 * rc2);
        for (int k = tid; k < N1; k += BLOCK) {
            const int key = k - sni[k].x;
            const float xf = sXf[3 * k], yf = sXf[3 * k + 1], zf = sXf[3 * k + 2];
            double a0 = 0.0, a1 = 0.0, a2 = 0.0;
            for (int j = 0; j < N1; ++j) {
                const float dx = xf - sXf[3 * j], dy = yf - sXf[3 * j + 1], dz = zf - sXf[3 * j + 2];
                if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rc2f && j - sni[j].x != key) {
                    const double rx = sXs[3 * k] - sXs[3 * j], ry = sXs[3 * k + 1] - sXs[3 * j + 1],
                                 rz = sXs[3 * k + 2] - sXs[3 * j + 2];
                    const double r2 = rx * rx + ry * ry + rz * rz;
                    if (r2 < rc2 && r2 > 0.0) {
                        const double sr2 = s2 / r2, sr6 = sr2 * sr2 * sr2;
                        const double c = 24.0 * P.lj_eps * (2.0 * sr6 * sr6 - sr6) / r2;
                        a0 += c * rx;
                        a1 += c * ry;
                        a2 += c * rz;
                    }
                }
            }
            sgf[3 * k] = (float)((double)sgf[3 * k] + a0);
            sgf[3 * k + 1] = (float)((double)sgf[3 * k + 1] + a1);
            sgf[3 * k + 2] = (float)((double)sgf[3 * k + 2] + a2);
        }
        __syncthreads();
    }
    if (2 * N1 <= BLOCK) {
        // two threads per point: the first half of the CTA sums sources [0, half), the second
        // [half, N1) (whole 32-source chunks), then the first adds the second's folded partial.
        // For N1 < 32 the rounded split point would pass N1; it is clamped so that the first
        // half takes every source and the second an empty range (a zero partial).
        constexpr int H = BLOCK / 2;
        const int part = tid >= H ? 1 : 0, i = tid - part * H;
        const int half = min(N1, (N1 / 2 + 31) & ~31);
        float sum[6], cmp[6];
        if (i < N1) {
            fused_pair_range(K, sXf, sgf, smf, i, part ? half : 0, part ? N1 : half, sum, cmp);
            if (part) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    su[3 * i + c] = __fsub_rn(sum[c], cmp[c]);
                    sw[3 * i + c] = __fsub_rn(sum[3 + c], cmp[3 + c]);
                }
            }
        }
        __syncthreads();
        if (!part && i < N1) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                fused_kahan(sum[c], cmp[c], su[3 * i + c]);
                fused_kahan(sum[3 + c], cmp[3 + c], sw[3 * i + c]);
                su[3 * i + c] = __fsub_rn(sum[c], cmp[c]) * K.scale;
                sw[3 * i + c] = __fsub_rn(sum[3 + c], cmp[3 + c]) * K.scale;
            }
        }
    } else {
        for (int i = tid; i < N1; i += BLOCK) {
            float sum[6], cmp[6];
            fused_pair_range(K, sXf, sgf, smf, i, 0, N1, sum, cmp);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                su[3 * i + c] = __fsub_rn(sum[c], cmp[c]) * K.scale;
                sw[3 * i + c] = __fsub_rn(sum[3 + c], cmp[3 + c]) * K.scale;
            }
        }
    }
    __syncthreads();
}

// (X1, D1) = (X0 + u h, Rodrigues(D0, w, h)) for the instance's points; X1/D1 may alias X0/D0.
template <int BLOCK>
__device__ void fused_update(int N1, const double* sX0, const double* sD0, const float* su,
                             const float* sw, double h, double* sX1, double* sD1)
{
    for (int k = threadIdx.x; k < N1; k += BLOCK) {
        double Dl[9], Dn[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) Dl[q] = sD0[9 * k + q];
        rodrigues(Dl, (double)sw[3 * k], (double)sw[3 * k + 1], (double)sw[3 * k + 2], h, Dn);
#pragma unroll
        for (int c = 0; c < 3; ++c) sX1[3 * k + c] = sX0[3 * k + c] + (double)su[3 * k + c] * h;
#pragma unroll
        for (int q = 0; q < 9; ++q) sD1[9 * k + q] = Dn[q];
    }
    __syncthreads();
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) rod_fine_fused_kernel(const RodLaunch L, double* X,
                                                                double* D, int nsteps, int scheme,
                                                                const FusedConst K)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    const int N1 = L.nodes_per_inst;
    const int inst = blockIdx.x;
    double* sX = reinterpret_cast<double*>(fsm);
    double* sD = sX + 3 * N1;
    double* sXh = sD + 9 * N1;
    double* sDh = sXh + 3 * N1;
    double* sFN = sDh + 9 * N1;
    double* sseg = sFN + 6 * N1;
    double* stime = sseg + 3 * N1;   // sin(f t), cos(f t) of the current stage
    double* sref = stime + 2;        // reference point of the current stage's float32 packs
    int2* sni = reinterpret_cast<int2*>(sref + 3);
    float* sXf = reinterpret_cast<float*>(sni + N1);
    float* sgf = sXf + 3 * N1;
    float* smf = sgf + 3 * N1;
    float* su = smf + 3 * N1;
    float* sw = su + 3 * N1;
    double* gX = X + (size_t)inst * 3 * N1;
    double* gD = D + (size_t)inst * 9 * N1;
    for (int q = threadIdx.x; q < 3 * N1; q += BLOCK) sX[q] = gX[q];
    for (int q = threadIdx.x; q < 9 * N1; q += BLOCK) sD[q] = gD[q];
    for (int k = threadIdx.x; k < N1; k += BLOCK) {
        int2 ni = L.node_info[k];
        if (!node_checked(L, ni, k, N1)) ni = make_int2(0, 1);   // skipped: a node with no segment
        sni[k] = ni;
        const double ds = L.p.L / (double)(ni.y - 1);
        double sk, ck;
        sincos(L.p.wave_k * ((double)ni.x + 0.5) * ds, &sk, &ck);
        sseg[3 * k] = 1.0 / ds;
        sseg[3 * k + 1] = sk;
        sseg[3 * k + 2] = ck;
    }
    const double t0 = L.t0[inst] + (double)(*L.step) * L.dt;
    __syncthreads();
    for (int st = 0; st < nsteps; ++st) {
        const double t = t0 + (double)st * L.dt;
        fused_velocity<BLOCK>(L, K, N1, sni, sseg, sX, sD, t, stime, sref, sFN, sXf, sgf, smf, su, sw);
        if (scheme == MRS_EULER) {
            fused_update<BLOCK>(N1, sX, sD, su, sw, L.dt, sX, sD);
        } else {
            fused_update<BLOCK>(N1, sX, sD, su, sw, 0.5 * L.dt, sXh, sDh);
            fused_velocity<BLOCK>(L, K, N1, sni, sseg, sXh, sDh, t + 0.5 * L.dt, stime, sref, sFN,
                                  sXf, sgf, smf, su, sw);
            fused_update<BLOCK>(N1, sX, sD, su, sw, L.dt, sX, sD);
        }
    }
    for (int q = threadIdx.x; q < 3 * N1; q += BLOCK) gX[q] = sX[q];
    for (int q = threadIdx.x; q < 9 * N1; q += BLOCK) gD[q] = sD[q];
}

__global__ void rod_bump_step_kernel(long long* step, int nsteps) { *step += nsteps; }

constexpr int kFusedBlock = 256;

size_t fused_smem_bytes(int N1)
{
    return 5 * sizeof(double) + (size_t)N1 * (33 * sizeof(double) + sizeof(int2) + 15 * sizeof(float));
}

bool fused_fits(int N1)
{
    return N1 >= 2 && fused_smem_bytes(N1) <= kFusedMaxSmem;
}

cudaError_t launch_rod_fine_fused(const RodLaunch& L, double* X, double* D, int nsteps, int scheme,
                                  double mu, double eps, cudaStream_t s)
{
    const int N1 = L.nodes_per_inst;
    const int n_inst = L.N / N1;
    if (L.N == 0 || nsteps <= 0) return cudaSuccess;
    const size_t bytes = fused_smem_bytes(N1);
    // raise the kernel's dynamic shared-memory limit once per device (not per launch)
    static bool raised[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!raised[dev]) {
        e = cudaFuncSetAttribute(rod_fine_fused_kernel<kFusedBlock>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedMaxSmem);
        if (e != cudaSuccess) return e;
        raised[dev] = true;
    }
    FusedConst K;
    const double e2 = eps * eps;
    K.e2 = (float)e2;
    K.c1 = (float)(1.5 * e2);
    K.c2 = (float)(3.75 * e2 * e2);
    K.c3 = (float)(-0.75 * e2);
    K.c5 = (float)(3.75 * e2);
    K.scale = (float)(1.0 / (8.0 * M_PI * mu));
    rod_fine_fused_kernel<kFusedBlock><<<n_inst, kFusedBlock, bytes, s>>>(L, X, D, nsteps, scheme, K);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    rod_bump_step_kernel<<<1, 1, 0, s>>>(L.step, nsteps);
    return cudaGetLastError();
}

// Start times of the instances of a batch, t0[i] = t_first + i * dT, and the step counter reset:
// a kernel rather than a host copy so that enqueueing never waits for the stream.
__global__ void rod_set_times_kernel(double* t0, int n_inst, double t_first, double dT,
                                     long long* step)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *step = 0;
    if (i < n_inst) t0[i] = t_first + (double)i * dT;
}

// Section IV-A: Lennard-Jones repulsion U = 4 e [(s/r)^12 - (s/r)^6] for r < r_c = 2^{1/6} s
// between nodes of different rods of the same instance, added to the force each node applies to
// the fluid (the rod is massless: elastic + LJ + fluid force = 0 on every node).  Every pair is
// screened in float32 against r_c^2 with a 1 % margin (the screen only has to be conservative);
// the rare close pairs are evaluated in float64 from the float64 positions.  Two nodes belong to
// the same rod when their rods start at the same node (node index minus index within the rod).
constexpr int kLJTile = 256;

__global__ void rod_lj_kernel(const RodLaunch L, const double* __restrict__ X, double* g64, float* gf)
{
    pdl_wait();
    __shared__ float sx[kLJTile * 3];
    __shared__ int skey[kLJTile];
    const int inst = blockIdx.y;
    const int N1 = L.nodes_per_inst;
    const int kl = blockIdx.x * kLJTile + threadIdx.x;
    const bool valid = kl < N1;
    const long long k = (long long)inst * N1 + (valid ? kl : N1 - 1);
    const double xi = X[3 * k], yi = X[3 * k + 1], zi = X[3 * k + 2];
    const float xf = (float)xi, yf = (float)yi, zf = (float)zi;
    const int key = (int)k - L.node_info[k].x;
    const double s2 = L.p.lj_sigma * L.p.lj_sigma;
    const double rc2 = 1.2599210498948732 * s2;            // (2^{1/6} sigma)^2
    const float rc2f = (float)(1.01 * rc2);
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
    for (int j0 = 0; j0 < N1; j0 += kLJTile) {
        const int cnt = min(kLJTile, N1 - j0);
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            const long long j = (long long)inst * N1 + j0 + threadIdx.x;
            sx[3 * threadIdx.x] = (float)X[3 * j];
            sx[3 * threadIdx.x + 1] = (float)X[3 * j + 1];
            sx[3 * threadIdx.x + 2] = (float)X[3 * j + 2];
            skey[threadIdx.x] = (int)j - L.node_info[j].x;
        }
        __syncthreads();
        for (int t = 0; t < cnt; ++t) {
            const float dx = xf - sx[3 * t], dy = yf - sx[3 * t + 1], dz = zf - sx[3 * t + 2];
            const float r2f = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (r2f < rc2f && skey[t] != key) {
                const long long j = (long long)inst * N1 + j0 + t;
                const double rx = xi - X[3 * j], ry = yi - X[3 * j + 1], rz = zi - X[3 * j + 2];
                const double r2 = rx * rx + ry * ry + rz * rz;
                if (r2 < rc2 && r2 > 0.0) {
                    const double sr2 = s2 / r2, sr6 = sr2 * sr2 * sr2;
                    const double c = 24.0 * L.p.lj_eps * (2.0 * sr6 * sr6 - sr6) / r2;
                    acc0 += c * rx;
                    acc1 += c * ry;
                    acc2 += c * rz;
                }
            }
        }
    }
    if (!valid) return;
    if (g64) {
        g64[3 * k] += acc0;
        g64[3 * k + 1] += acc1;
        g64[3 * k + 2] += acc2;
    }
    if (gf) {
        gf[3 * k] = (float)((double)gf[3 * k] + acc0);
        gf[3 * k + 1] = (float)((double)gf[3 * k + 1] + acc1);
        gf[3 * k + 2] = (float)((double)gf[3 * k + 2] + acc2);
    }
}

static inline int nblk(int n, int b) { return (n + b - 1) / b; }

cudaError_t launch_set_times(double* t0, int n_inst, double t_first, double dT, long long* step,
                             cudaStream_t s)
{
    rod_set_times_kernel<<<nblk(n_inst, 128), 128, 0, s>>>(t0, n_inst, t_first, dT, step);
    return cudaGetLastError();
}

cudaError_t launch_rod_forces(const RodLaunch& L, const double* X, const double* D, double t_off,
                              double* g64, double* m64, float* Xf, float* gf, float* mf,
                              cudaStream_t s)
{
    if (L.N == 0) return cudaSuccess;
    if (L.wchunks != nullptr) {
        cudaError_t e = launch_pdl(rod_forces_warp_kernel, dim3(L.n_wchunks), dim3(128), 0, s, L, X, D, t_off,
                                   g64, m64, Xf, gf, mf);
        if (e != cudaSuccess) return e;
    } else if (L.chunks != nullptr) {
        cudaError_t e = launch_pdl(rod_forces_fused_kernel, dim3(L.n_chunks), dim3(kRodChunk), 0, s,
                                   L, X, D, t_off, g64, m64, Xf, gf, mf);
        if (e != cudaSuccess) return e;
    } else {
        cudaError_t e = launch_pdl(rod_segment_kernel, dim3(nblk(L.N, 128)), dim3(128), 0, s, L, X, D, t_off);
        if (e == cudaSuccess)
            e = launch_pdl(rod_node_kernel, dim3(nblk(L.N, 128)), dim3(128), 0, s, L, X, g64, m64, Xf, gf, mf);
        if (e != cudaSuccess) return e;
    }
    if (L.p.lj_eps > 0.0) {
        const dim3 grid(nblk(L.nodes_per_inst, kLJTile), L.N / L.nodes_per_inst);
        return launch_pdl(rod_lj_kernel, grid, dim3(kLJTile), 0, s, L, X, g64, gf);
    }
    return cudaSuccess;
}

cudaError_t launch_rod_update(const RodLaunch& L, const double* X0, const double* D0,
                              const float* u, const float* w, double h, double* X1, double* D1,
                              bool bump_step, cudaStream_t s)
{
    if (L.N == 0) return cudaSuccess;
    if (L.wchunks != nullptr)   // small batch: warp-cooperative (see rod_forces_warp_kernel)
        return launch_pdl(rod_update_warp_kernel<float>, dim3(nblk(L.N, 4 * kUNodesPerWarp)), dim3(128), 0, s,
                          L, X0, D0, u, w, h, X1, D1, bump_step ? 1 : 0);
    return launch_pdl(rod_update_kernel<float>, dim3(nblk(L.N, 128)), dim3(128), 0, s, L, X0, D0, u, w,
                      h, X1, D1, bump_step ? 1 : 0);
}

cudaError_t launch_rod_update64(const RodLaunch& L, const double* X0, const double* D0,
                                const double* u, const double* w, double h, double* X1,
                                double* D1, bool bump_step, cudaStream_t s)
{
    if (L.N == 0) return cudaSuccess;
    if (L.wchunks != nullptr)
        return launch_pdl(rod_update_warp_kernel<double>, dim3(nblk(L.N, 4 * kUNodesPerWarp)), dim3(128), 0,
                          s, L, X0, D0, u, w, h, X1, D1, bump_step ? 1 : 0);
    return launch_pdl(rod_update_kernel<double>, dim3(nblk(L.N, 128)), dim3(128), 0, s, L, X0, D0, u,
                      w, h, X1, D1, bump_step ? 1 : 0);
}

cudaError_t launch_segment_table(int N, const int2* node_info, double wave_k, double Lrod,
                                 double2* out, cudaStream_t s)
{
    if (N == 0) return cudaSuccess;
    rod_segsc_kernel<<<nblk(N, 128), 128, 0, s>>>(N, node_info, wave_k, Lrod, out);
    return cudaGetLastError();
}

cudaError_t launch_rot_sqrt_batch(int n, const double* R, double* S, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    rot_sqrt_batch_kernel<<<nblk(n, 128), 128, 0, s>>>(n, R, S);
    return cudaGetLastError();
}

}  // namespace mrs
