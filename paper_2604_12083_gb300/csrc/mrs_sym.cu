// mrs_sym.cu -- the regularized-Stokeslet pair sum with each unordered pair evaluated once.
//
// Section II-C, Eqs. (velocity_field), (angular_velocity_field), (superposition).  When the
// targets are the sources (the rod nodes themselves, the paper's setting), the pair (i, j) and
// the pair (j, i) share everything that depends on the separation alone: with q = X_j - x_i,
// the separation of the reversed pair is -q, and
//   mu u_j     += f_i H1 + (f_i.q) q H2 - H3 (q x n_i)
//   mu omega_j += -H3 (q x f_i) + n_i H4 + (n_i.q) q H5
// against mu u_i += f_j H1 + (f_j.q) q H2 + H3 (q x n_j) and
//         mu omega_i += H3 (q x f_j) + n_j H4 + (n_j.q) q H5 for the forward pair.
// The separation, the SFU rsqrt, the kernel values H1..H5 and the scaled separation H3 q are
// computed once (19 FP32 instructions) and each direction adds 32, so one unordered pair costs
// 83 FP32 instructions instead of 2 x 50.
//
// Layout of the work: see SymTile in mrs_internal.h.  Inside a CTA, each thread holds TPT
// points of the row's tile as TPT/2 packs (the two lanes of every float2 are two different
// points), each source is staged in shared memory with every component duplicated into both
// lanes, and all f32x2 instructions of a pair act on two (point, source) pairs.  The source's
// share of a pair sum is folded over the thread's packs, reduced over the warp by a
// transposing shuffle reduction (8 shuffles for 6 values) and over the CTA's warps through
// shared memory, then written to the column partial of its work unit.  The tile's points keep
// their share in registers, folded per chunk into Kahan pairs in MRS_F32_COMP.
#include "mrs_checks.h"
#include "mrs_device.cuh"
#include "mrs_internal.h"

namespace mrs {

namespace {

struct PairConsts {
    float2 e2, c1, c2, c3, c5, mhalf, three_halves;
};

// Shared part of one pair for a pack of two points x (lanes) and one source X (duplicated):
// q = X - x, the kernel values and the scaled separation.
struct PairCore {
    float2 q0, q1, q2, s3, h1, h4, h5, hq0, hq1, hq2;
};

template <bool SQ>
__device__ __forceinline__ PairCore pair_core(const float2* x, const float2* S, const PairConsts& K)
{
    PairCore c;
    c.q0 = __fadd2_rn(S[0], neg2(x[0]));
    c.q1 = __fadd2_rn(S[1], neg2(x[1]));
    c.q2 = __fadd2_rn(S[2], neg2(x[2]));
    const float2 d = __ffma2_rn(c.q0, c.q0, __ffma2_rn(c.q1, c.q1, __ffma2_rn(c.q2, c.q2, K.e2)));
    const float2 s = make_float2(sfu_rsqrt(d.x), sfu_rsqrt(d.y));
    const float2 s2 = SQ ? __fmul2_rn(s, s) : make_float2(sfu_rcp(d.x), sfu_rcp(d.y));
    c.s3 = __fmul2_rn(s, s2);
    const float2 s5 = __fmul2_rn(c.s3, s2);
    c.h1 = __ffma2_rn(K.e2, c.s3, s);                                          // 8 pi H1
    const float2 h3 = __ffma2_rn(K.c1, s5, c.s3);                              // 8 pi H3
    c.h4 = __fmul2_rn(c.s3, __ffma2_rn(s2, __ffma2_rn(K.c2, s2, K.c3), K.mhalf));  // 8 pi H4
    c.h5 = __fmul2_rn(s5, __ffma2_rn(K.c5, s2, K.three_halves));               // 8 pi H5
    c.hq0 = __fmul2_rn(h3, c.q0);
    c.hq1 = __fmul2_rn(h3, c.q1);
    c.hq2 = __fmul2_rn(h3, c.q2);
    return c;
}

// One direction of a pair: acc += H1 F + H2 (F.q) q + SGN H3 (q x N) (u) and
// H4 N + H5 (N.q) q + SGN H3 (q x F) (omega), SGN = +1 for the forward pair (F, N of the
// source), -1 for the reversed pair (F, N of the points).
template <bool REV>
__device__ __forceinline__ void pair_dir(const PairCore& c, const float2* F, const float2* N,
                                         float2* acc)
{
    const float2 fq = __ffma2_rn(F[0], c.q0, __ffma2_rn(F[1], c.q1, __fmul2_rn(F[2], c.q2)));
    const float2 nq = __ffma2_rn(N[0], c.q0, __ffma2_rn(N[1], c.q1, __fmul2_rn(N[2], c.q2)));
    const float2 bf = __fmul2_rn(c.s3, fq);
    const float2 bn = __fmul2_rn(c.h5, nq);
    acc[0] = __ffma2_rn(c.h1, F[0], acc[0]);
    acc[1] = __ffma2_rn(c.h1, F[1], acc[1]);
    acc[2] = __ffma2_rn(c.h1, F[2], acc[2]);
    acc[0] = __ffma2_rn(bf, c.q0, acc[0]);
    acc[1] = __ffma2_rn(bf, c.q1, acc[1]);
    acc[2] = __ffma2_rn(bf, c.q2, acc[2]);
    acc[3] = __ffma2_rn(c.h4, N[0], acc[3]);
    acc[4] = __ffma2_rn(c.h4, N[1], acc[4]);
    acc[5] = __ffma2_rn(c.h4, N[2], acc[5]);
    acc[3] = __ffma2_rn(bn, c.q0, acc[3]);
    acc[4] = __ffma2_rn(bn, c.q1, acc[4]);
    acc[5] = __ffma2_rn(bn, c.q2, acc[5]);
    if (!REV) {
        // + (H3 q) x N and + (H3 q) x F
        acc[0] = __ffma2_rn(c.hq1, N[2], acc[0]);
        acc[1] = __ffma2_rn(c.hq2, N[0], acc[1]);
        acc[2] = __ffma2_rn(c.hq0, N[1], acc[2]);
        acc[0] = __ffma2_rn(neg2(c.hq2), N[1], acc[0]);
        acc[1] = __ffma2_rn(neg2(c.hq0), N[2], acc[1]);
        acc[2] = __ffma2_rn(neg2(c.hq1), N[0], acc[2]);
        acc[3] = __ffma2_rn(c.hq1, F[2], acc[3]);
        acc[4] = __ffma2_rn(c.hq2, F[0], acc[4]);
        acc[5] = __ffma2_rn(c.hq0, F[1], acc[5]);
        acc[3] = __ffma2_rn(neg2(c.hq2), F[1], acc[3]);
        acc[4] = __ffma2_rn(neg2(c.hq0), F[2], acc[4]);
        acc[5] = __ffma2_rn(neg2(c.hq1), F[0], acc[5]);
    } else {
        // - (H3 q) x N and - (H3 q) x F
        acc[0] = __ffma2_rn(c.hq2, N[1], acc[0]);
        acc[1] = __ffma2_rn(c.hq0, N[2], acc[1]);
        acc[2] = __ffma2_rn(c.hq1, N[0], acc[2]);
        acc[0] = __ffma2_rn(neg2(c.hq1), N[2], acc[0]);
        acc[1] = __ffma2_rn(neg2(c.hq2), N[0], acc[1]);
        acc[2] = __ffma2_rn(neg2(c.hq0), N[1], acc[2]);
        acc[3] = __ffma2_rn(c.hq2, F[1], acc[3]);
        acc[4] = __ffma2_rn(c.hq0, F[2], acc[4]);
        acc[5] = __ffma2_rn(c.hq1, F[0], acc[5]);
        acc[3] = __ffma2_rn(neg2(c.hq1), F[2], acc[3]);
        acc[4] = __ffma2_rn(neg2(c.hq2), F[0], acc[4]);
        acc[5] = __ffma2_rn(neg2(c.hq0), F[1], acc[5]);
    }
}

// Sum of v[0..5] over the 32 lanes of a warp by halving exchanges: after the exchange across
// lane bit 4 each lane holds three of the six partial sums, after bit 3 two (one of them a zero
// pad), after bit 2 one, and bits 1 and 0 finish with plain butterflies.  Returns the total of
// component *c (valid when *c < 6; lanes 4m..4m+3 hold the same value).
__device__ __forceinline__ float warp_sum6(const float* v, int lane, int* c)
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float a0 = b4 ? v[3] : v[0], a1 = b4 ? v[4] : v[1], a2 = b4 ? v[5] : v[2];
    const float o0 = b4 ? v[0] : v[3], o1 = b4 ? v[1] : v[4], o2 = b4 ? v[2] : v[5];
    a0 += __shfl_xor_sync(0xffffffffu, o0, 16);
    a1 += __shfl_xor_sync(0xffffffffu, o1, 16);
    a2 += __shfl_xor_sync(0xffffffffu, o2, 16);
    float k0 = b3 ? a2 : a0, k1 = b3 ? 0.f : a1;
    const float s0 = b3 ? a0 : a2, s1 = b3 ? a1 : 0.f;
    k0 += __shfl_xor_sync(0xffffffffu, s0, 8);
    k1 += __shfl_xor_sync(0xffffffffu, s1, 8);
    float m = b2 ? k1 : k0;
    const float o = b2 ? k0 : k1;
    m += __shfl_xor_sync(0xffffffffu, o, 4);
    m += __shfl_xor_sync(0xffffffffu, m, 2);
    m += __shfl_xor_sync(0xffffffffu, m, 1);
    *c = (b3 && b2) ? 6 : (b4 ? 3 : 0) + (b3 ? 2 : 0) + (b2 ? 1 : 0);   // 6: the pad
    return m;
}

template <int BLOCK, int TPT>
struct SymMinBlocks {   // CTAs per SM the register allocation must allow
    static constexpr int value = BLOCK >= 384 ? 1 : BLOCK >= 128 ? (TPT >= 4 ? 3 : 4) : (TPT >= 4 ? 6 : 8);
};

template <int BLOCK, int TPT, bool COMP>
constexpr size_t sym_smem_bytes()
{
    // staged sources, per-warp source partials, Kahan pairs
    return sizeof(float2) * 9 * kSymChunk + sizeof(float) * (BLOCK / 32) * kSymChunk * 6 +
           (COMP ? sizeof(float2) * 6 * TPT * BLOCK : 0);
}

}  // namespace

// SKEW = false: every lane takes the same source (shared-memory broadcast) and the source's
// share is summed over the warp by warp_sum6.  SKEW = true: within each group of 32 sources,
// lane l takes source (t + l) mod 32 at step t, so the lanes of a warp work on 32 different
// sources at every step and each adds its share to the source's per-warp accumulator in
// shared memory without any exchange between lanes (no shuffles, no dependent chain).
// UNR: unroll of the skewed source loop; MINB: CTAs per SM the register allocation must allow
// (0: SymMinBlocks).
template <int BLOCK, int TPT, bool COMP, bool SQ, bool SKEW, int UNR = 2, int MINB = 0>
__global__ void __launch_bounds__(BLOCK, (MINB ? MINB : SymMinBlocks<BLOCK, TPT>::value))
mrs_f32_sym(const SymLaunch L)
{
    pdl_wait();
    static_assert(TPT % 2 == 0, "points are held in packs of two");
    constexpr int NP = TPT / 2;
    constexpr int TM = BLOCK * TPT;
    constexpr int NW = BLOCK / 32;
    constexpr int CH = kSymChunk;
    // dynamic shared memory (sym_smem_bytes): the staged sources [component][source] with both
    // lanes equal; the per-warp source partials [warp][source][component] (SKEW:
    // [warp][component][source]); the Kahan pairs of the tile's points (MRS_F32_COMP)
    extern __shared__ __align__(16) unsigned char sym_smem[];
    float2* ssrc = reinterpret_cast<float2*>(sym_smem);
    float* swp = reinterpret_cast<float*>(sym_smem + sizeof(float2) * 9 * CH);
    float2* kah = reinterpret_cast<float2*>(sym_smem + sizeof(float2) * 9 * CH + sizeof(float) * NW * CH * 6);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int p = blockIdx.x;
    long long ubeg = L.U0 + unit_start(L.W, L.P, p);
    const long long uend = L.U0 + unit_start(L.W, L.P, p + 1);
    if (ubeg >= uend) return;

    int ti;
    {
        int lo = L.ta, hi = L.tb - 1;   // the pass's tiles
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (L.tiles[mid].u0 <= ubeg) lo = mid; else hi = mid - 1;
        }
        ti = lo;
    }

    while (ubeg < uend) {
#if MRS_DEBUG_BOUNDS
        // every thread of the CTA reads the same tile, so the CTA leaves together
        if (ti < L.ta || ti >= L.tb) {
            if (tid == 0) atomicOr(L.err, MRS_FLAG_BOUNDS);
            return;
        }
#endif
        const SymTile T = L.tiles[ti];
#if MRS_DEBUG_BOUNDS
        if (!sym_tile_ok(T, TM, L.n_points, L.U0, L.col_units, L.row_segs) || ubeg < T.u0 ||
            ubeg >= T.u0 + T.nu || p < T.qlo || p - T.qlo >= T.nseg) {
            if (tid == 0) atomicOr(L.err, MRS_FLAG_BOUNDS);
            return;
        }
#endif
        const long long seg_end = min(uend, T.u0 + (long long)T.nu);
        const int ua = (int)(ubeg - T.u0), ub = (int)(seg_end - T.u0);
        const SysConst sys = L.sc[T.sys];
        PairConsts K;
        K.e2 = f2(sys.e2);
        K.c1 = f2(sys.c1);
        K.c2 = f2(sys.c2);
        K.c3 = f2(sys.c3);
        K.c5 = f2(sys.c5);
        K.mhalf = f2(-0.5f);
        K.three_halves = f2(1.5f);

        // the tile's points: positions, and f, n for the reversed pairs (zero for the padding
        // of a ragged tile, so that padded points give nothing to the sources)
        float2 xp[NP][3], fp[NP][3], np_[NP][3], acc[NP][6];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float xa[2][3], fa[2][3], na[2][3];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int li = (2 * k + h) * BLOCK + tid;
                const bool ok = li < T.tn;
                const long long gi = (long long)T.t0 + (ok ? li : T.tn - 1);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    xa[h][c] = L.X[gi * 3 + c];
                    fa[h][c] = ok ? L.f[gi * 3 + c] : 0.f;
                    na[h][c] = ok ? L.n[gi * 3 + c] : 0.f;
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xp[k][c] = make_float2(xa[0][c], xa[1][c]);
                fp[k][c] = make_float2(fa[0][c], fa[1][c]);
                np_[k][c] = make_float2(na[0][c], na[1][c]);
            }
#pragma unroll
            for (int q = 0; q < 6; ++q) acc[k][q] = make_float2(0.f, 0.f);
        }
        if (COMP) {
#pragma unroll
            for (int k = 0; k < TPT; ++k)
#pragma unroll
                for (int q = 0; q < 6; ++q) kah[(q * TPT + k) * BLOCK + tid] = make_float2(0.f, 0.f);
        }

        const int jbeg = T.t0 + ua * kUnitSources;
        const int jend = min(T.t0 + ub * kUnitSources, T.send);
        const int jdiag = T.t0 + T.nd * kUnitSources;   // end of the diagonal block
        for (int j0 = jbeg; j0 < jend;) {
            const bool diag = j0 < jdiag;
            const int cend = min(min(j0 + CH, jend), diag ? jdiag : jend);
            const int cnt = cend - j0;
            __syncthreads();   // the previous chunk's sources and partials are no longer read
            for (int idx = tid; idx < cnt * 3; idx += BLOCK) {
                const int s = idx / 3, c = idx - s * 3;
                ssrc[c * CH + s] = f2(__ldg(L.X + (long long)j0 * 3 + idx));
                ssrc[(3 + c) * CH + s] = f2(__ldg(L.f + (long long)j0 * 3 + idx));
                ssrc[(6 + c) * CH + s] = f2(__ldg(L.n + (long long)j0 * 3 + idx));
            }
            const int cnt32 = (cnt + 31) & ~31;
            if (SKEW && !diag) {
                // zero sources up to a whole group of 32 (they add nothing to the points; their
                // own partials are never written out), and zero this warp's accumulators
                for (int s = cnt + tid; s < cnt32; s += BLOCK)
#pragma unroll
                    for (int c = 0; c < 9; ++c) ssrc[c * CH + s] = make_float2(0.f, 0.f);
                for (int idx = lane; idx < 6 * CH; idx += 32) swp[warp * CH * 6 + idx] = 0.f;
            }
            __syncthreads();

            if (diag) {
                // the tile against itself: ordered pairs, the tile's points as targets only
#pragma unroll 2
                for (int j = 0; j < cnt; ++j) {
                    float2 S[9];
#pragma unroll
                    for (int c = 0; c < 9; ++c) S[c] = ssrc[c * CH + j];
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        const PairCore pc = pair_core<SQ>(xp[k], S, K);
                        pair_dir<false>(pc, S + 3, S + 6, acc[k]);
                    }
                }
            } else if (SKEW) {
                float* wp = swp + warp * CH * 6;
                for (int g = 0; g < cnt32; g += 32) {
#pragma unroll UNR
                    for (int t = 0; t < 32; ++t) {
                        const int j = g + ((t + lane) & 31);
                        float2 S[9];
#pragma unroll
                        for (int c = 0; c < 9; ++c) S[c] = ssrc[c * CH + j];
                        float2 sacc[6];
#pragma unroll
                        for (int q = 0; q < 6; ++q) sacc[q] = make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k < NP; ++k) {
                            const PairCore pc = pair_core<SQ>(xp[k], S, K);
                            pair_dir<false>(pc, S + 3, S + 6, acc[k]);
                            pair_dir<true>(pc, fp[k], np_[k], sacc);
                        }
#pragma unroll
                        for (int q = 0; q < 6; ++q)
                            wp[q * CH + j] = __fadd_rn(wp[q * CH + j], __fadd_rn(sacc[q].x, sacc[q].y));
                    }
                }
            } else {
                for (int j = 0; j < cnt; ++j) {
                    float2 S[9];
#pragma unroll
                    for (int c = 0; c < 9; ++c) S[c] = ssrc[c * CH + j];
                    float2 sacc[6];
#pragma unroll
                    for (int q = 0; q < 6; ++q) sacc[q] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        const PairCore pc = pair_core<SQ>(xp[k], S, K);
                        pair_dir<false>(pc, S + 3, S + 6, acc[k]);
                        pair_dir<true>(pc, fp[k], np_[k], sacc);
                    }
                    float v[6];
#pragma unroll
                    for (int q = 0; q < 6; ++q) v[q] = __fadd_rn(sacc[q].x, sacc[q].y);
                    int c;
                    const float tot = warp_sum6(v, lane, &c);
                    if ((lane & 3) == 0 && c < 6) swp[(warp * CH + j) * 6 + c] = tot;
                }
            }
            if (!diag) {
                __syncthreads();
                // column partials of this chunk: the sum over the CTA's warps, in warp order
                float* cp = L.colpart + ((T.u0 - L.U0) * kUnitSources + (j0 - T.t0)) * 6;
                for (int idx = tid; idx < cnt * 6; idx += BLOCK) {
                    // idx = 6 j + q; SKEW keeps the partials component-major
                    const int sidx = SKEW ? (idx % 6) * CH + idx / 6 : idx;
                    float s = swp[sidx];
#pragma unroll
                    for (int w = 1; w < NW; ++w) s = __fadd_rn(s, swp[w * CH * 6 + sidx]);
                    cp[idx] = s;
                }
            }
            if (COMP) {
#pragma unroll
                for (int k = 0; k < NP; ++k)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
#pragma unroll
                        for (int q = 0; q < 6; ++q) {
                            float2& kk = kah[(q * TPT + 2 * k + h) * BLOCK + tid];
                            float sum = kk.x, cmp = kk.y;
                            kahan_add(sum, cmp, h ? acc[k][q].y : acc[k][q].x);
                            kk = make_float2(sum, cmp);
                        }
#pragma unroll
                for (int k = 0; k < NP; ++k)
#pragma unroll
                    for (int q = 0; q < 6; ++q) acc[k][q] = make_float2(0.f, 0.f);
            }
            j0 = cend;
        }

        // row partial of this segment
        float* rp = L.rowpart + ((long long)(T.seg0 + (p - T.qlo)) * TM) * 6;
#pragma unroll
        for (int k = 0; k < NP; ++k)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int li = (2 * k + h) * BLOCK + tid;
                if (li < T.tn) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        float v;
                        if (COMP) {
                            const float2 kk = kah[(q * TPT + 2 * k + h) * BLOCK + tid];
                            v = __fsub_rn(kk.x, kk.y);
                        } else {
                            v = h ? acc[k][q].y : acc[k][q].x;
                        }
                        rp[li * 6 + q] = v;
                    }
                }
            }
        ubeg = seg_end;
        ++ti;
    }
}

// Sum per point and component over one pass: the Kahan pair carried from earlier passes (none
// in the first pass touching the point's system), then -- for a point of the pass's own tiles
// -- its row's partials (CTA order) and the column partials of the earlier tiles of its system
// that lie in the pass (tile order); for a later point of a system the pass touches, the
// column partials of all the pass's tiles of that system.  Own points are final: scaled by
// 1/(8 pi mu) and written out; later points carry their pair to the next pass.
// kRedSplit consecutive lanes share one (point, component): lane r sums the terms r, r + R,
// r + 2R, ... of that sequence into its own Kahan pair (lane 0 starting from the carried
// pair), fetching kRedAhead terms at a time so that their L2 latencies overlap, and lane 0
// then adds the other lanes' compensated sums in lane order -- a fixed order, so the result
// is deterministic.
constexpr int kRedAhead = 8;
constexpr int kRedSplit = 4;

__global__ void __launch_bounds__(256) mrs_sym_reduce(const SymLaunch L)
{
    pdl_wait();
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(L.tc - L.ta) * L.TM * 6 * kRedSplit) return;   // whole lane groups
    const int r = (int)(idx % kRedSplit);
    const long long pq = idx / kRedSplit;
    const long long pt = pq / 6;
    const int q = (int)(pq - pt * 6);
    const int tl = (int)(pt / L.TM), li = (int)(pt - (long long)tl * L.TM);
    const int ti = L.ta + tl;
#if MRS_DEBUG_BOUNDS
    if (ti >= L.n_tiles) {
        atomicOr(L.err, MRS_FLAG_BOUNDS);
        return;
    }
#endif
    const SymTile T = L.tiles[ti];
    if (li >= T.tn) return;   // the whole lane group leaves together
    const int j = T.t0 + li;
    const bool own = ti < L.tb;
#if MRS_DEBUG_BOUNDS
    // the units of a later tile lie in a later pass: only its extent is checked
    if (!sym_tile_ok(T, L.TM, L.n_points, own ? L.U0 : T.u0, own ? L.col_units : T.nu, L.row_segs) ||
        T.tfirst > ti) {
        if (r == 0) atomicOr(L.err, MRS_FLAG_BOUNDS);
        return;   // the whole lane group reads the same tile and leaves together
    }
#endif
    float sum = 0.f, cmp = 0.f;
    if (r == 0 && T.tfirst < L.ta) {   // an earlier pass holds tiles of this system
        const float2 a = L.acc[(long long)j * 6 + q];
        sum = a.x;
        cmp = a.y;
    }
    const int nrow = own ? T.nseg : 0;
    const int c0 = max(T.tfirst, L.ta), c1 = own ? ti : L.tb;   // column tiles [c0, c1)
    const int nterm = nrow + max(0, c1 - c0);
    for (int k0 = r; k0 < nterm; k0 += kRedSplit * kRedAhead) {
        float v[kRedAhead];
#pragma unroll
        for (int a = 0; a < kRedAhead; ++a) {
            const int k = k0 + a * kRedSplit;
            v[a] = 0.f;
            if (k < nrow) {
                v[a] = __ldcg(L.rowpart + ((long long)(T.seg0 + k) * L.TM + li) * 6 + q);
            } else if (k < nterm) {
                const SymTile& R = L.tiles[c0 + (k - nrow)];
#if MRS_DEBUG_BOUNDS
                if (!sym_tile_ok(R, L.TM, L.n_points, L.U0, L.col_units, L.row_segs) || j < R.t0 ||
                    j >= R.send) {
                    atomicOr(L.err, MRS_FLAG_BOUNDS);
                    continue;   // the term is skipped
                }
#endif
                v[a] = __ldcg(L.colpart + ((R.u0 - L.U0) * kUnitSources + (j - R.t0)) * 6 + q);
            }
        }
#pragma unroll
        for (int a = 0; a < kRedAhead; ++a)
            if (k0 + a * kRedSplit < nterm) kahan_add(sum, cmp, v[a]);
    }
    // lane 0 of the group folds in lanes 1..R-1, in lane order
    const unsigned lane = threadIdx.x & 31u;
    const unsigned mask = ((1u << kRedSplit) - 1u) << (lane & ~(unsigned)(kRedSplit - 1));
    float part = __fsub_rn(sum, cmp);
#pragma unroll
    for (int o = 1; o < kRedSplit; ++o) {
        const float other = __shfl_down_sync(mask, part, o, kRedSplit);
        if (r == 0) kahan_add(sum, cmp, other);
    }
    if (r != 0) return;
    if (!own) {
        L.acc[(long long)j * 6 + q] = make_float2(sum, cmp);
        return;
    }
    const float val = __fsub_rn(sum, cmp) * L.sc[T.sys].scale;
    if (!isfinite(val)) atomicOr(L.err, 1u);
    if (q < 3) L.u[(long long)j * 3 + q] = val; else L.w[(long long)j * 3 + q - 3] = val;
}

int cta_of_unit_host(long long W, int P, long long x)
{
    auto start = [&](int p) { return (W * (long long)p) / (long long)P; };
    int q = (int)((x * (long long)P) / W);
    if (q > P - 1) q = P - 1;
    while (q + 1 < P && start(q + 1) <= x) ++q;
    while (q > 0 && start(q) > x) --q;
    return q;
}

template <int BLOCK, int TPT, bool COMP, bool SQ, bool SKEW, int UNR, int MINB>
static cudaError_t sym_prepare()
{
    constexpr size_t bytes = sym_smem_bytes<BLOCK, TPT, COMP>();
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(mrs_f32_sym<BLOCK, TPT, COMP, SQ, SKEW, UNR, MINB>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// The dynamic shared-memory limit above 48 KB is raised by occupancy_sym, which every plan and
// server calls when it is built, so a launch makes no attribute call (stream capture safe).
template <int BLOCK, int TPT, bool COMP, bool SQ, bool SKEW, int UNR, int MINB>
static cudaError_t launch_sym_t(const SymLaunch& L, cudaStream_t s)
{
    cudaError_t e = launch_pdl(mrs_f32_sym<BLOCK, TPT, COMP, SQ, SKEW, UNR, MINB>, dim3(L.P), dim3(BLOCK),
                               sym_smem_bytes<BLOCK, TPT, COMP>(), s, L);
    if (e != cudaSuccess) return e;
    const long long n = (long long)(L.tc - L.ta) * L.TM * 6 * kRedSplit;
    if (n == 0) return cudaSuccess;
    return launch_pdl(mrs_sym_reduce, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, L);
}

template <int BLOCK, int TPT, bool COMP, bool SQ, bool SKEW, int UNR, int MINB>
static int occ_sym_t(int* n)
{
    if (sym_prepare<BLOCK, TPT, COMP, SQ, SKEW, UNR, MINB>() != cudaSuccess) return MRS_ECUDA;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        n, mrs_f32_sym<BLOCK, TPT, COMP, SQ, SKEW, UNR, MINB>, BLOCK, sym_smem_bytes<BLOCK, TPT, COMP>());
    return e == cudaSuccess ? MRS_OK : MRS_ECUDA;
}

#define MRS_SYM_CASE_X(id, B, T, Q, K, U, M, FN, ...) \
    case id:                                          \
        return comp ? FN<B, T, true, Q, K, U, M>(__VA_ARGS__) : FN<B, T, false, Q, K, U, M>(__VA_ARGS__);
#define MRS_SYM_CASE(id, B, T, Q, K, FN, ...) MRS_SYM_CASE_X(id, B, T, Q, K, 2, 0, FN, __VA_ARGS__)

// Symmetric configurations (ids continue the ordered table of mrs_kernels.cu).  Measured on the
// 32768-point system (ms per call, both kernels): 17: 1.80 (warp-shuffle reduction of each
// source's share), 18: 1.68, 19: 1.67, 20: 1.68 (one 384-thread CTA per SM), 21: 1.653,
// 22: 1.651, 23: 1.630, and 23 launched as 2 / 4 / 8 waves of CTAs (24, 25, 26): 1.622, 1.610
// (the default), 1.628.  On the 512-system batch 26 is the fastest (21.2 ms).  Computing the next
// source's kernel values while accumulating the current one's (software pipelining, 2 packs,
// 200 registers) was slower: 1.74 ms; unrolling 25's source loop twice changed nothing (1.612);
// keeping the tile's f and n in shared memory (126 registers, 16 warps per SM, 64-source
// chunks) was slower too: 1.68 ms at 4 points per thread, 1.64 ms at 6.
#define MRS_SYM_DISPATCH(cfg, comp, FN, ...)                             \
    switch (cfg) {                                                       \
        MRS_SYM_CASE(17, 128, 4, false, false, FN, __VA_ARGS__)          \
        MRS_SYM_CASE(18, 128, 4, false, true, FN, __VA_ARGS__)           \
        MRS_SYM_CASE(19, 128, 4, true, true, FN, __VA_ARGS__)            \
        MRS_SYM_CASE(20, 384, 4, false, true, FN, __VA_ARGS__)           \
        MRS_SYM_CASE_X(21, 128, 6, true, true, 1, 2, FN, __VA_ARGS__)    \
        MRS_SYM_CASE_X(22, 128, 8, true, true, 1, 2, FN, __VA_ARGS__)    \
        MRS_SYM_CASE_X(23, 64, 6, true, true, 1, 4, FN, __VA_ARGS__)     \
        MRS_SYM_CASE_X(24, 64, 6, true, true, 1, 4, FN, __VA_ARGS__)     \
        MRS_SYM_CASE_X(25, 64, 6, true, true, 1, 4, FN, __VA_ARGS__)     \
        MRS_SYM_CASE_X(26, 64, 6, true, true, 1, 4, FN, __VA_ARGS__)     \
    default: break;                                                      \
    }

cudaError_t launch_mrs_sym(int config, bool comp, const SymLaunch& L, cudaStream_t s)
{
    MRS_SYM_DISPATCH(config, comp, launch_sym_t, L, s);
    return cudaErrorInvalidValue;
}

int occupancy_sym(int config, bool comp, int* ctas_per_sm)
{
    MRS_SYM_DISPATCH(config, comp, occ_sym_t, ctas_per_sm);
    return MRS_EINVAL;
}

}  // namespace mrs
