// mrs_kernels.cu -- the regularized-Stokeslet pair sum on sm_103a.
//
// Section II-C, Eqs. (velocity_field), (angular_velocity_field), (superposition); Section
// III-C-2.  For every target i and every source j of its system (self pair included):
//   mu u_i     += f_j H1 + (f_j.r) r H2 + (n_j x r) H3
//   mu omega_i += (f_j x r) H3 + n_j H4 + (n_j.r) r H5,         r = x_i - X_j.
//
// Arithmetic.  With d = r^2 + eps^2, s = d^{-1/2} (SFU rsqrt), s2 = 1/d (SFU rcp), s3 = s s2,
// s5 = s3 s2 and e2 = eps^2, the identity d s2 = 1 turns every polynomial in r^2 = d - e2 of
// the kernels into one in s2:
//   8 pi H1 = s + e2 s3                      8 pi H2 = s3
//   8 pi H3 = s3 + (3/2) e2 s5               8 pi H5 = s5 (3/2 + (15/4) e2 s2)
//   8 pi H4 = s3 (-1/2 + s2 (-(3/4) e2 + (15/4) e2^2 s2))
// and with the scaled separation H3 r serving both cross products (H3 (n x r) = n x (H3 r),
// likewise for f), one pair costs 50 FP32 instructions (FFMA/FMUL/FADD) and 2 SFU
// instructions; the common factor 1/(8 pi mu) is applied once per target.  No tensor cores: the pair sum is not
// a dense contraction.
//
// Float32 path (MRS_F32 / MRS_F32_COMP): one persistent kernel over all systems of a batch.
//   * CTA p of P processes the contiguous range [W p/P, W (p+1)/P) of the W work units (a
//     unit = one target tile x kUnitSources sources), so every CTA gets the same number of
//     pairs whatever the system sizes (no tail of idle SMs).
//   * Each thread holds TPT targets in registers (targets tid, tid+BLOCK, ... of the tile);
//     sources are staged kChunk at a time in shared memory as three float4 per source and read
//     by warp-wide broadcast, so each shared load is reused TPT times.
//   * Accumulation: per-chunk float32 partials; in MRS_F32_COMP each chunk's partial is folded
//     into a per-target Kahan pair (sum, compensation) held in shared memory.
//   * A tile whose units are spread over several CTAs: each CTA writes its partial to its own
//     scratch slot, then adds its unit count to the tile's counter; the CTA that completes the
//     count sums all slots in CTA order (float32 Kahan) and writes the result, then zeroes the
//     counter for the next launch.  No CTA ever waits for another.
//
// Float64 path (MRS_F64): one CTA per 128 targets, all sources of the system staged through
// shared memory, float64 arithmetic with the kernels written in r^2.
#include "mrs_device.cuh"
#include "mrs_checks.h"
#include "mrs_internal.h"
#include "rod_update.cuh"

namespace mrs {

// One (target, source) pair accumulated into acc[0..2] (u) and acc[3..5] (omega), both scaled
// by 8 pi mu.  a = (X.x, X.y, X.z, f.x), b = (f.y, f.z, n.x, n.y), nz = n.z.
__device__ __forceinline__ void pair_f32(float xi, float yi, float zi, const float4 a,
                                         const float4 b, float nz, float e2, float c1, float c2,
                                         float c3, float c5, float* acc)
{
    const float rx = xi - a.x, ry = yi - a.y, rz = zi - a.z;
    const float fx = a.w, fy = b.x, fz = b.y, nx = b.z, ny = b.w;
    const float d = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, e2)));
    const float s = sfu_rsqrt(d);
    const float s2 = sfu_rcp(d);
    const float s3 = s * s2;
    const float s5 = s3 * s2;
    const float h1 = fmaf(e2, s3, s);                        // 8 pi H1
    const float h3 = fmaf(c1, s5, s3);                       // 8 pi H3
    const float h4 = s3 * fmaf(s2, fmaf(c2, s2, c3), -0.5f);  // 8 pi H4
    const float h5 = s5 * fmaf(c5, s2, 1.5f);                // 8 pi H5
    const float fr = fmaf(fx, rx, fmaf(fy, ry, fz * rz));
    const float nr = fmaf(nx, rx, fmaf(ny, ry, nz * rz));
    const float bf = s3 * fr;                                // 8 pi H2 (f.r)
    const float bn = h5 * nr;                                // 8 pi H5 (n.r)
    // H3 (n x r) = n x (H3 r) and H3 (f x r) = f x (H3 r): one scaled separation serves both
    const float hrx = h3 * rx, hry = h3 * ry, hrz = h3 * rz;
    // u += H1 f + H2 (f.r) r + H3 (n x r)
    acc[0] = fmaf(h1, fx, acc[0]);
    acc[1] = fmaf(h1, fy, acc[1]);
    acc[2] = fmaf(h1, fz, acc[2]);
    acc[0] = fmaf(bf, rx, acc[0]);
    acc[1] = fmaf(bf, ry, acc[1]);
    acc[2] = fmaf(bf, rz, acc[2]);
    acc[0] = fmaf(ny, hrz, acc[0]);
    acc[1] = fmaf(nz, hrx, acc[1]);
    acc[2] = fmaf(nx, hry, acc[2]);
    acc[0] = fmaf(-nz, hry, acc[0]);
    acc[1] = fmaf(-nx, hrz, acc[1]);
    acc[2] = fmaf(-ny, hrx, acc[2]);
    // omega += H3 (f x r) + H4 n + H5 (n.r) r
    acc[3] = fmaf(h4, nx, acc[3]);
    acc[4] = fmaf(h4, ny, acc[4]);
    acc[5] = fmaf(h4, nz, acc[5]);
    acc[3] = fmaf(bn, rx, acc[3]);
    acc[4] = fmaf(bn, ry, acc[4]);
    acc[5] = fmaf(bn, rz, acc[5]);
    acc[3] = fmaf(fy, hrz, acc[3]);
    acc[4] = fmaf(fz, hrx, acc[4]);
    acc[5] = fmaf(fx, hry, acc[5]);
    acc[3] = fmaf(-fz, hry, acc[3]);
    acc[4] = fmaf(-fx, hrz, acc[4]);
    acc[5] = fmaf(-fy, hrx, acc[5]);
}

// Packed form of pair_f32: the two lanes of every float2 hold two different sources (j, j+1)
// for the same target, so each f32x2 instruction does the work of two scalar ones.  q = X - x
// (the negated separation; every term below is written in q: (f.r) r = (f.q) q and
// n x r = q x n), so the staged positions need no negation.
template <bool SQ>
__device__ __forceinline__ void pair_f32x2(const float2 xt, const float2 yt, const float2 zt,  // targets
                                           const float2 X0, const float2 X1, const float2 X2,
                                           const float2 F0, const float2 F1, const float2 F2,
                                           const float2 N0, const float2 N1, const float2 N2,
                                           const float2 e2, const float2 c1, const float2 c2,
                                           const float2 c3, const float2 c5, float2* acc)
{
    const float2 qx = __fadd2_rn(X0, neg2(xt)), qy = __fadd2_rn(X1, neg2(yt)),
                 qz = __fadd2_rn(X2, neg2(zt));
    const float2 d = __ffma2_rn(qx, qx, __ffma2_rn(qy, qy, __ffma2_rn(qz, qz, e2)));
    const float2 s = make_float2(sfu_rsqrt(d.x), sfu_rsqrt(d.y));
    // SQ: s2 = s s (one packed multiply) instead of a second SFU op per lane
    const float2 s2 = SQ ? __fmul2_rn(s, s) : make_float2(sfu_rcp(d.x), sfu_rcp(d.y));
    const float2 s3 = __fmul2_rn(s, s2);
    const float2 s5 = __fmul2_rn(s3, s2);
    const float2 h1 = __ffma2_rn(e2, s3, s);
    const float2 h3 = __ffma2_rn(c1, s5, s3);
    const float2 h4 = __fmul2_rn(s3, __ffma2_rn(s2, __ffma2_rn(c2, s2, c3), f2(-0.5f)));
    const float2 h5 = __fmul2_rn(s5, __ffma2_rn(c5, s2, f2(1.5f)));
    const float2 fq = __ffma2_rn(F0, qx, __ffma2_rn(F1, qy, __fmul2_rn(F2, qz)));
    const float2 nq = __ffma2_rn(N0, qx, __ffma2_rn(N1, qy, __fmul2_rn(N2, qz)));
    const float2 bf = __fmul2_rn(s3, fq);
    const float2 bn = __fmul2_rn(h5, nq);
    // H3 (q x n) = (H3 q) x n and H3 (q x f) = (H3 q) x f: one scaled separation serves both
    const float2 hq0 = __fmul2_rn(h3, qx), hq1 = __fmul2_rn(h3, qy), hq2 = __fmul2_rn(h3, qz);
    // u += H1 f + H2 (f.q) q + H3 (q x n)
    acc[0] = __ffma2_rn(h1, F0, acc[0]);
    acc[1] = __ffma2_rn(h1, F1, acc[1]);
    acc[2] = __ffma2_rn(h1, F2, acc[2]);
    acc[0] = __ffma2_rn(bf, qx, acc[0]);
    acc[1] = __ffma2_rn(bf, qy, acc[1]);
    acc[2] = __ffma2_rn(bf, qz, acc[2]);
    acc[0] = __ffma2_rn(hq1, N2, acc[0]);
    acc[1] = __ffma2_rn(hq2, N0, acc[1]);
    acc[2] = __ffma2_rn(hq0, N1, acc[2]);
    acc[0] = __ffma2_rn(neg2(hq2), N1, acc[0]);
    acc[1] = __ffma2_rn(neg2(hq0), N2, acc[1]);
    acc[2] = __ffma2_rn(neg2(hq1), N0, acc[2]);
    // omega += H3 (q x f) + H4 n + H5 (n.q) q
    acc[3] = __ffma2_rn(h4, N0, acc[3]);
    acc[4] = __ffma2_rn(h4, N1, acc[4]);
    acc[5] = __ffma2_rn(h4, N2, acc[5]);
    acc[3] = __ffma2_rn(bn, qx, acc[3]);
    acc[4] = __ffma2_rn(bn, qy, acc[4]);
    acc[5] = __ffma2_rn(bn, qz, acc[5]);
    acc[3] = __ffma2_rn(hq1, F2, acc[3]);
    acc[4] = __ffma2_rn(hq2, F0, acc[4]);
    acc[5] = __ffma2_rn(hq0, F1, acc[5]);
    acc[3] = __ffma2_rn(neg2(hq2), F1, acc[3]);
    acc[4] = __ffma2_rn(neg2(hq0), F2, acc[4]);
    acc[5] = __ffma2_rn(neg2(hq1), F0, acc[5]);
}

// The CTA whose unit range contains unit x.
__device__ __forceinline__ int cta_of_unit(long long W, int P, long long x)
{
    int q = (int)((x * (long long)P) / W);
    if (q > P - 1) q = P - 1;
    while (q + 1 < P && unit_start(W, P, q + 1) <= x) ++q;
    while (q > 0 && unit_start(W, P, q) > x) --q;
    return q;
}

template <int BLOCK, int TPT>
struct MinBlocks {   // CTAs per SM the register allocation must allow
    static constexpr int value = TPT == 1 ? (BLOCK >= 256 ? 3 : 6)
                                          : (BLOCK >= 256 ? 2 : (BLOCK >= 128 ? (TPT >= 8 ? 3 : 4) : 8));
};

// PAIRED: the inner loop runs on packed f32x2 instructions, two sources per instruction
// (pair_f32x2); sources are then staged structure-of-arrays (nine rows of kChunk floats) so
// that four consecutive sources of one component are one 16-byte shared load.
template <int BLOCK, int TPT, bool COMP, bool PAIRED, int UNROLL, bool SQ = false>
__global__ void __launch_bounds__(BLOCK, (MinBlocks<BLOCK, TPT>::value))
mrs_f32_persistent(const MrsLaunch L)
{
    pdl_wait();
    constexpr int TM = BLOCK * TPT;
    __shared__ __align__(16) float sflat[kChunk * 12];
    __shared__ float2 kah[COMP ? 6 * TPT * BLOCK : 1];
    __shared__ int s_last;

    const int tid = threadIdx.x;
    const int p = blockIdx.x;
    long long ubeg = unit_start(L.W, L.P, p);
    const long long uend = unit_start(L.W, L.P, p + 1);
    if (ubeg >= uend) return;

    if (!PAIRED) {
        // lanes 9..11 of every staged source stay zero
        for (int i = tid; i < kChunk; i += BLOCK) {
            sflat[i * 12 + 9] = 0.f;
            sflat[i * 12 + 10] = 0.f;
            sflat[i * 12 + 11] = 0.f;
        }
    }
    // first tile: the last one whose first unit is <= ubeg
    int ti;
    {
        int lo = 0, hi = L.n_tiles - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (L.tiles[mid].u0 <= ubeg) lo = mid; else hi = mid - 1;
        }
        ti = lo;
    }
    bool first_seg = true;

    while (ubeg < uend) {
#if MRS_DEBUG_BOUNDS
        // every thread of the CTA reads the same tile, so the CTA leaves together
        if (ti < 0 || ti >= L.n_tiles) {
            if (tid == 0) atomicOr(L.err, MRS_FLAG_BOUNDS);
            return;
        }
#endif
        const TileDesc T = L.tiles[ti];
#if MRS_DEBUG_BOUNDS
        if (!ordered_tile_ok(T, TM, L.n_points) || ubeg < T.u0 || ubeg >= T.u0 + T.nu) {
            if (tid == 0) atomicOr(L.err, MRS_FLAG_BOUNDS);
            return;
        }
#endif
        const long long send = min(uend, T.u0 + (long long)T.nu);
        const int ua = (int)(ubeg - T.u0), ub = (int)(send - T.u0);
        const bool full = (ua == 0 && ub == T.nu);
        const SysConst sc = L.sc[T.sys];

        float xt[TPT][3];
        float acc[TPT][6];
        float2 acc2[TPT][6];
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            const int li = k * BLOCK + tid;
            const long long gi = (long long)T.t0 + (li < T.tn ? li : T.tn - 1);
#pragma unroll
            for (int c = 0; c < 3; ++c) xt[k][c] = L.Xt[gi * 3 + c];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                acc[k][q] = 0.f;
                acc2[k][q] = make_float2(0.f, 0.f);
            }
            if (COMP) {
#pragma unroll
                for (int q = 0; q < 6; ++q) kah[(q * TPT + k) * BLOCK + tid] = make_float2(0.f, 0.f);
            }
        }

        const long long jbeg = (long long)T.s0 + (long long)ua * kUnitSources;
        const long long jend = (long long)T.s0 + min((long long)ub * kUnitSources, (long long)T.sn);
        for (long long j0 = jbeg; j0 < jend; j0 += kChunk) {
            const int cnt = (int)min((long long)kChunk, jend - j0);
            const int cntp = (cnt + 3) & ~3;
            __syncthreads();  // the previous chunk is no longer read
            const float* gX = L.X + j0 * 3;
            const float* gf = L.f + j0 * 3;
            const float* gn = L.n + j0 * 3;
            for (int idx = tid; idx < cnt * 3; idx += BLOCK) {
                const int sidx = idx / 3, c = idx - sidx * 3;
                if (PAIRED) {
                    sflat[c * kChunk + sidx] = __ldg(gX + idx);
                    sflat[(3 + c) * kChunk + sidx] = __ldg(gf + idx);
                    sflat[(6 + c) * kChunk + sidx] = __ldg(gn + idx);
                } else {
                    sflat[sidx * 12 + c] = __ldg(gX + idx);
                    sflat[sidx * 12 + 3 + c] = __ldg(gf + idx);
                    sflat[sidx * 12 + 6 + c] = __ldg(gn + idx);
                }
            }
            for (int sidx = cnt + tid; sidx < cntp; sidx += BLOCK) {
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    if (PAIRED) sflat[c * kChunk + sidx] = 0.f;   // zero source: adds 0
                    else sflat[sidx * 12 + c] = 0.f;
                }
            }
            __syncthreads();

            if (PAIRED) {
                const float2 e2 = f2(sc.e2), c1 = f2(sc.c1), c2 = f2(sc.c2), c3 = f2(sc.c3),
                             c5 = f2(sc.c5);
                float2 xn[TPT][3];
#pragma unroll
                for (int k = 0; k < TPT; ++k)
#pragma unroll
                    for (int c = 0; c < 3; ++c) xn[k][c] = f2(xt[k][c]);
#pragma unroll UNROLL
                for (int j = 0; j < cntp; j += 4) {
                    float4 v[9];
#pragma unroll
                    for (int c = 0; c < 9; ++c)
                        v[c] = *reinterpret_cast<const float4*>(&sflat[c * kChunk + j]);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float2 s9[9];
#pragma unroll
                        for (int c = 0; c < 9; ++c)
                            s9[c] = h == 0 ? make_float2(v[c].x, v[c].y) : make_float2(v[c].z, v[c].w);
#pragma unroll
                        for (int k = 0; k < TPT; ++k)
                            pair_f32x2<SQ>(xn[k][0], xn[k][1], xn[k][2], s9[0], s9[1], s9[2], s9[3],
                                       s9[4], s9[5], s9[6], s9[7], s9[8], e2, c1, c2, c3, c5,
                                       acc2[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < TPT; ++k)
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        acc[k][q] = __fadd_rn(acc[k][q], __fadd_rn(acc2[k][q].x, acc2[k][q].y));
                        acc2[k][q] = make_float2(0.f, 0.f);
                    }
            } else {
                const float e2 = sc.e2, c1 = sc.c1, c2 = sc.c2, c3 = sc.c3, c5 = sc.c5;
#pragma unroll 2
                for (int j = 0; j < cntp; ++j) {
                    const float4 a = *reinterpret_cast<const float4*>(&sflat[j * 12]);
                    const float4 b = *reinterpret_cast<const float4*>(&sflat[j * 12 + 4]);
                    const float nz = sflat[j * 12 + 8];
#pragma unroll
                    for (int k = 0; k < TPT; ++k)
                        pair_f32(xt[k][0], xt[k][1], xt[k][2], a, b, nz, e2, c1, c2, c3, c5, acc[k]);
                }
            }
            if (COMP) {
                // Kahan fold of this chunk's partial into (sum, compensation)
#pragma unroll
                for (int k = 0; k < TPT; ++k) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        float2 sc2 = kah[(q * TPT + k) * BLOCK + tid];
                        const float y = __fsub_rn(acc[k][q], sc2.y);
                        const float t = __fadd_rn(sc2.x, y);
                        sc2.y = __fsub_rn(__fsub_rn(t, sc2.x), y);
                        sc2.x = t;
                        kah[(q * TPT + k) * BLOCK + tid] = sc2;
                        acc[k][q] = 0.f;
                    }
                }
            }
        }

        // --- result of this segment -------------------------------------------------------
        if (full) {
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                const int li = k * BLOCK + tid;
                if (li < T.tn) {
                    const long long gi = (long long)T.t0 + li;
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        float v;
                        if (COMP) {
                            const float2 sc2 = kah[(q * TPT + k) * BLOCK + tid];
                            v = __fsub_rn(sc2.x, sc2.y);
                        } else {
                            v = acc[k][q];
                        }
                        v *= sc.scale;
                        if (!isfinite(v)) atomicOr(L.err, 1u);
                        if (q < 3) L.u[gi * 3 + q] = v; else L.w[gi * 3 + q - 3] = v;
                    }
                }
            }
        } else {
            const int slot = 2 * p + (first_seg ? 0 : 1);
            float* part = L.partial + (size_t)slot * 6 * TM;
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                const int li = k * BLOCK + tid;
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    if (COMP) {
                        const float2 sc2 = kah[(q * TPT + k) * BLOCK + tid];
                        part[q * TM + li] = __fsub_rn(sc2.x, sc2.y);
                    } else {
                        part[q * TM + li] = acc[k][q];
                    }
                }
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                const int mine = ub - ua;
                const int old = atomicAdd(&L.counters[ti], mine);
                s_last = (old + mine == T.nu) ? 1 : 0;
            }
            __syncthreads();
            if (s_last) {
                __threadfence();
                // float32 Kahan sum over the slots, in CTA order (float64 is a slow pipe here).
                // Contributors are the consecutive CTAs q_lo..q_hi (every CTA range is non-empty
                // because P <= W).  Only q_lo can have started before this tile, in which case
                // the tile is its second segment (slot 2 q_lo + 1); for every later CTA it is the
                // first segment (slot 2 qc).  A slot holds one float per target and component
                // (in MRS_F32_COMP the segment's Kahan pair folded to sum - compensation); they
                // are read eight at a time to keep loads in flight, and the sum order stays the
                // CTA order.
                const int q_lo = cta_of_unit(L.W, L.P, T.u0);
                const int q_hi = cta_of_unit(L.W, L.P, T.u0 + T.nu - 1);
#if MRS_DEBUG_BOUNDS
                if (q_lo < 0 || q_hi >= L.P || q_lo > q_hi) {   // contributor slots outside [0, 2P)
                    if (tid == 0) atomicOr(L.err, MRS_FLAG_BOUNDS);
                    return;
                }
#endif
                const int sl_lo = 2 * q_lo + (unit_start(L.W, L.P, q_lo) < T.u0 ? 1 : 0);
                constexpr int NB = 8;
#pragma unroll 1
                for (int k = 0; k < TPT; ++k) {
                    const int li = k * BLOCK + tid;
                    float tot[6], cmp[6];
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        tot[q] = 0.f;
                        cmp[q] = 0.f;
                    }
                    for (int qb = q_lo; qb <= q_hi; qb += NB) {
                        float v[NB][6];
#pragma unroll
                        for (int bq = 0; bq < NB; ++bq) {
                            const int qc = qb + bq;
                            const int sl = qc == q_lo ? sl_lo : 2 * qc;
                            const float* pp = L.partial + (size_t)sl * 6 * TM + li;
#pragma unroll
                            for (int q = 0; q < 6; ++q) v[bq][q] = qc <= q_hi ? __ldcg(pp + q * TM) : 0.f;
                        }
#pragma unroll
                        for (int bq = 0; bq < NB; ++bq)
#pragma unroll
                            for (int q = 0; q < 6; ++q) kahan_add(tot[q], cmp[q], v[bq][q]);
                    }
                    if (li < T.tn) {
                        const long long gi = (long long)T.t0 + li;
#pragma unroll
                        for (int q = 0; q < 6; ++q) {
                            const float val = __fsub_rn(tot[q], cmp[q]) * sc.scale;
                            if (!isfinite(val)) atomicOr(L.err, 1u);
                            if (q < 3) L.u[gi * 3 + q] = val; else L.w[gi * 3 + q - 3] = val;
                        }
                    }
                }
                if (tid == 0) L.counters[ti] = 0;
            }
        }
        first_seg = false;
        ubeg = send;
        ++ti;
    }
}

// ---------------------------------------------------------------------------------------------
// Cluster kernel for small systems (KernelConfig::cluster > 0).  One thread-block cluster of
// L.cl CTAs per target tile of TM targets; a CTA has TM x G threads, G groups of TM threads with
// one target each.  CTA r of the cluster sweeps the units [nu r / cl, nu (r+1) / cl) of the
// tile's sources, group g taking every G-th 4-source block of each staged chunk, with the
// packed inner loop and the per-chunk Kahan folding of mrs_f32_persistent.  The groups'
// partials (sum - compensation) are summed in group order in shared memory into the CTA's
// partial, one float per target and component.  After a cluster barrier, CTA r reduces targets
// [r tpr, (r+1) tpr) of the tile, tpr = ceil(TM / cl): it reads the partial of every CTA of the
// cluster through distributed shared memory (mapa + ld.shared::cluster) and sums them in rank
// order with float32 Kahan, as the persistent kernel's finishing CTA sums its slots.  A second
// barrier keeps every CTA resident until its partials have been read.  For a system of a few
// hundred to a few thousand points this replaces the scratch slots in global memory, the
// atomic tile counter and the finishing CTA's reads with on-chip traffic: the call is then a
// load of the sources, the sweep and two cluster barriers, with G warps per tile and SM for
// latency hiding.
//
// Every thread of every CTA reaches both barriers: nothing returns early (a CTA with no units
// contributes zero partials; the debug build's index checks skip work instead of returning).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_index()
{
    unsigned c;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(c));
    return c;
}

__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// float at shared-memory address `p` (this CTA's) in the shared memory of CTA `rank`
__device__ __forceinline__ float ld_cluster_f32(const float* p, unsigned rank)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    unsigned ra;
    float v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(ra) : "memory");
    return v;
}

constexpr int kMaxCluster = 16;

template <int TM, int G, bool COMP, int UNROLL>
__global__ void __launch_bounds__(TM * G) mrs_f32_cluster(const MrsLaunch L)
{
    pdl_wait();
    constexpr int BLOCK = TM * G;
    __shared__ __align__(16) float sflat[kChunk * 9];
    __shared__ float sgrp[G > 1 ? G * 6 * TM : 1];   // each group's partial: [group][component][target]
    __shared__ float spart[6 * TM];                  // the CTA's partial: [component][target]
    __shared__ float sv[6 * TM];                     // completed velocities (update epilogue)

    const int tid = threadIdx.x;
    const int lt = tid % TM, g = tid / TM;   // target of the tile, source group
    const int cl = L.cl;
    const int ti = (int)cluster_index();
    const int r = (int)cluster_rank();
    bool ok = true;
#if MRS_DEBUG_BOUNDS
    ok = ti >= 0 && ti < L.n_tiles && cl >= 1 && cl <= kMaxCluster && r < cl;
    if (ok) ok = ordered_tile_ok(L.tiles[ti], TM, L.n_points);
    if (!ok && tid == 0) atomicOr(L.err, MRS_FLAG_BOUNDS);
#endif
    const TileDesc T = L.tiles[ok ? ti : 0];
    const SysConst sc = L.sc[ok ? T.sys : 0];
    const int ua = (int)((long long)T.nu * r / cl), ub = (int)((long long)T.nu * (r + 1) / cl);

    float xt[3];
    {
        const long long gi = (long long)T.t0 + (lt < T.tn ? lt : T.tn - 1);
#pragma unroll
        for (int c = 0; c < 3; ++c) xt[c] = L.Xt[gi * 3 + c];
    }
    float acc[6], ks[6], kc[6];
    float2 acc2[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        acc[q] = ks[q] = kc[q] = 0.f;
        acc2[q] = make_float2(0.f, 0.f);
    }
    const long long jbeg = (long long)T.s0 + (long long)ua * kUnitSources;
    const long long jend = ok ? (long long)T.s0 + min((long long)ub * kUnitSources, (long long)T.sn) : jbeg;
    const float2 e2 = f2(sc.e2), c1 = f2(sc.c1), c2 = f2(sc.c2), c3 = f2(sc.c3), c5 = f2(sc.c5);
    const float2 xn[3] = {f2(xt[0]), f2(xt[1]), f2(xt[2])};
    for (long long j0 = jbeg; j0 < jend; j0 += kChunk) {
        const int cnt = (int)min((long long)kChunk, jend - j0);
        const int cntp = (cnt + 3) & ~3;
        __syncthreads();   // the previous chunk is no longer read
        const float* gX = L.X + j0 * 3;
        const float* gf = L.f + j0 * 3;
        const float* gn = L.n + j0 * 3;
        for (int idx = tid; idx < cnt * 3; idx += BLOCK) {
            const int sidx = idx / 3, c = idx - sidx * 3;
            sflat[c * kChunk + sidx] = __ldg(gX + idx);
            sflat[(3 + c) * kChunk + sidx] = __ldg(gf + idx);
            sflat[(6 + c) * kChunk + sidx] = __ldg(gn + idx);
        }
        for (int sidx = cnt + tid; sidx < cntp; sidx += BLOCK) {
#pragma unroll
            for (int c = 0; c < 9; ++c) sflat[c * kChunk + sidx] = 0.f;   // zero source: adds 0
        }
        __syncthreads();
        // group g takes the 4-source blocks g, g + G, g + 2G, ... of the chunk
#pragma unroll UNROLL
        for (int j = 4 * g; j < cntp; j += 4 * G) {
            float4 v[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) v[c] = *reinterpret_cast<const float4*>(&sflat[c * kChunk + j]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float2 s9[9];
#pragma unroll
                for (int c = 0; c < 9; ++c)
                    s9[c] = h == 0 ? make_float2(v[c].x, v[c].y) : make_float2(v[c].z, v[c].w);
                pair_f32x2<false>(xn[0], xn[1], xn[2], s9[0], s9[1], s9[2], s9[3], s9[4], s9[5], s9[6],
                                  s9[7], s9[8], e2, c1, c2, c3, c5, acc2);
            }
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            acc[q] = __fadd_rn(acc[q], __fadd_rn(acc2[q].x, acc2[q].y));
            acc2[q] = make_float2(0.f, 0.f);
            if (COMP) {   // Kahan fold of this chunk's partial
                kahan_add(ks[q], kc[q], acc[q]);
                acc[q] = 0.f;
            }
        }
    }
    if (G > 1) {
        // the groups' partials summed in group order (float32 Kahan) into the CTA's partial
#pragma unroll
        for (int q = 0; q < 6; ++q) sgrp[(g * 6 + q) * TM + lt] = COMP ? __fsub_rn(ks[q], kc[q]) : acc[q];
        __syncthreads();
        for (int e = tid; e < 6 * TM; e += BLOCK) {
            float tot = 0.f, cmp = 0.f;
#pragma unroll
            for (int gg = 0; gg < G; ++gg) kahan_add(tot, cmp, sgrp[gg * 6 * TM + e]);
            spart[e] = __fsub_rn(tot, cmp);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 6; ++q) spart[q * TM + lt] = COMP ? __fsub_rn(ks[q], kc[q]) : acc[q];
    }

    cluster_barrier();   // every CTA's partials are written and visible to the cluster

    const int tpr = (TM + cl - 1) / cl;
    const int lo = r * tpr, hi = min(TM, lo + tpr);
    for (int e = tid; e < (hi - lo) * 6; e += BLOCK) {
        const int li = lo + e / 6, q = e - (e / 6) * 6;
        const float* src = spart + q * TM + li;
        float v[kMaxCluster];
#pragma unroll
        for (int k = 0; k < kMaxCluster; ++k) v[k] = k < cl ? ld_cluster_f32(src, (unsigned)k) : 0.f;
        float tot = 0.f, cmp = 0.f;
#pragma unroll
        for (int k = 0; k < kMaxCluster; ++k)
            if (k < cl) kahan_add(tot, cmp, v[k]);
        if (ok && li < T.tn) {
            const long long gi = (long long)T.t0 + li;
            const float val = __fsub_rn(tot, cmp) * sc.scale;
            if (!isfinite(val)) atomicOr(L.err, 1u);
            if (q < 3) L.u[gi * 3 + q] = val; else L.w[gi * 3 + q - 3] = val;
            sv[(li - lo) * 6 + q] = val;
        }
    }

    if (L.upX0) {
        // update epilogue: nine threads per completed target, one entry (director i, component
        // c) of its new frame each, the first three also one position component; every thread
        // reads what it needs before any thread of the CTA stores (in-place update)
        if (L.up_step && blockIdx.x == 0 && tid == 0) *L.up_step += 1;
        const int nloc = ok ? max(0, min(hi, T.tn) - lo) : 0;
        __syncthreads();   // sv complete
        for (int base = 0; base < nloc * 9; base += BLOCK) {
            const int idx = base + tid;
            const bool act = idx < nloc * 9;
            const int nl = idx / 9, e = idx - 9 * (idx / 9);
            const long long gk = (long long)T.t0 + lo + (act ? nl : 0);
            double d1 = 0.0, x1 = 0.0;
            if (act) {
                const int i = e / 3, c = e - 3 * (e / 3);
                const float* vv = sv + nl * 6;
                const double* v = L.upD0 + 9 * gk + 3 * i;
                d1 = rodrigues_entry(v[0], v[1], v[2], (double)vv[3], (double)vv[4], (double)vv[5], L.up_h, c);
                if (e < 3) x1 = L.upX0[3 * gk + e] + (double)vv[e] * L.up_h;
            }
            __syncthreads();
            if (act) {
                L.upD1[9 * gk + e] = d1;
                if (e < 3) L.upX1[3 * gk + e] = x1;
            }
        }
    }

    // no CTA leaves while another still reads its partials; the reads above have completed
    // (their values are consumed), so the arrival needs no release ordering
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\t"
                 "barrier.cluster.wait.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------------------------
// Configuration table and dispatch.
// ---------------------------------------------------------------------------------------------
const KernelConfig kConfigs[] = {
    {128, 4, 0, 1}, {128, 2, 0, 1}, {128, 8, 0, 1}, {64, 4, 0, 1}, {256, 2, 0, 1}, {128, 1, 0, 1},
    {128, 2, 1, 1}, {128, 4, 1, 1}, {64, 4, 1, 1}, {256, 2, 1, 1},
    {256, 2, 1, 2}, {128, 2, 1, 2}, {128, 1, 1, 1}, {128, 1, 1, 2}, {256, 1, 1, 2},
    {256, 2, 1, 1, 1}, {256, 1, 1, 2, 1},
    // symmetric (mrs_sym.cu): packs of two points per thread, duplicated sources
    {128, 4, 1, 1, 0, 1}, {128, 4, 1, 1, 0, 1}, {128, 4, 1, 1, 1, 1}, {384, 4, 1, 1, 0, 1},
    {128, 6, 1, 1, 1, 1}, {128, 8, 1, 1, 1, 1}, {64, 6, 1, 1, 1, 1},
    // ... the last three launched as 2, 4 and 8 waves of CTAs (KernelConfig::over)
    {64, 6, 1, 1, 1, 1, 2}, {64, 6, 1, 1, 1, 1, 4}, {64, 6, 1, 1, 1, 1, 8},
    // cluster kernel (small systems): 256 threads per CTA as 32 targets x 8 source groups and
    // as 64 targets x 4, clusters of up to 16 CTAs
    {256, 1, 1, 1, 0, 0, 0, 16, 8}, {256, 1, 1, 1, 0, 0, 0, 16, 4},
};
const int kNumConfigs = (int)(sizeof(kConfigs) / sizeof(kConfigs[0]));

template <int BLOCK, int TPT, bool COMP, bool PAIRED, int UNROLL, bool SQ>
static cudaError_t launch_t(const MrsLaunch& L, cudaStream_t s)
{
    return launch_pdl(mrs_f32_persistent<BLOCK, TPT, COMP, PAIRED, UNROLL, SQ>, dim3(L.P), dim3(BLOCK), 0,
                      s, L);
}

template <int BLOCK, int TPT, bool COMP, bool PAIRED, int UNROLL, bool SQ>
static int occ_t(int* n)
{
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        n, mrs_f32_persistent<BLOCK, TPT, COMP, PAIRED, UNROLL, SQ>, BLOCK, 0);
    return e == cudaSuccess ? MRS_OK : MRS_ECUDA;
}

#define MRS_CASE_SQ(id, B, T, P, U, Q, FN, ...)                                           \
    case id:                                                                              \
        return comp ? FN<B, T, true, P, U, Q>(__VA_ARGS__) : FN<B, T, false, P, U, Q>(__VA_ARGS__);
#define MRS_CASE(id, B, T, P, U, FN, ...) MRS_CASE_SQ(id, B, T, P, U, false, FN, __VA_ARGS__)

#define MRS_DISPATCH(cfg, comp, FN, ...)                                                  \
    switch (cfg) {                                                                        \
        MRS_CASE(0, 128, 4, false, 1, FN, __VA_ARGS__)                                    \
        MRS_CASE(1, 128, 2, false, 1, FN, __VA_ARGS__)                                    \
        MRS_CASE(2, 128, 8, false, 1, FN, __VA_ARGS__)                                    \
        MRS_CASE(3, 64, 4, false, 1, FN, __VA_ARGS__)                                     \
        MRS_CASE(4, 256, 2, false, 1, FN, __VA_ARGS__)                                    \
        MRS_CASE(5, 128, 1, false, 1, FN, __VA_ARGS__)                                    \
        MRS_CASE(6, 128, 2, true, 1, FN, __VA_ARGS__)                                     \
        MRS_CASE(7, 128, 4, true, 1, FN, __VA_ARGS__)                                     \
        MRS_CASE(8, 64, 4, true, 1, FN, __VA_ARGS__)                                      \
        MRS_CASE(9, 256, 2, true, 1, FN, __VA_ARGS__)                                     \
        MRS_CASE(10, 256, 2, true, 2, FN, __VA_ARGS__)                                    \
        MRS_CASE(11, 128, 2, true, 2, FN, __VA_ARGS__)                                    \
        MRS_CASE(12, 128, 1, true, 1, FN, __VA_ARGS__)                                    \
        MRS_CASE(13, 128, 1, true, 2, FN, __VA_ARGS__)                                    \
        MRS_CASE(14, 256, 1, true, 2, FN, __VA_ARGS__)                                    \
        MRS_CASE_SQ(15, 256, 2, true, 1, true, FN, __VA_ARGS__)                           \
        MRS_CASE_SQ(16, 256, 1, true, 2, true, FN, __VA_ARGS__)                           \
    default: break;                                                                       \
    }

template <int TM, int G, bool COMP, int UNROLL>
static cudaError_t launch_cl_t(const MrsLaunch& L, cudaStream_t s)
{
    return launch_pdl_cl(mrs_f32_cluster<TM, G, COMP, UNROLL>, dim3(L.P), dim3(TM * G), 0, s, L.cl, L);
}

template <int TM, int G, bool COMP, int UNROLL>
static int occ_cl_t(int* n)
{
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, mrs_f32_cluster<TM, G, COMP, UNROLL>,
                                                                  TM * G, 0);
    return e == cudaSuccess ? MRS_OK : MRS_ECUDA;
}

template <int TM, int G, bool COMP, int UNROLL>
static int setup_cl_t(int cl, int* n)
{
    *n = 0;
    if (cl < 1 || cl > kMaxCluster) return MRS_EINVAL;
    cudaError_t e = cudaFuncSetAttribute(mrs_f32_cluster<TM, G, COMP, UNROLL>,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cl);
        cfg.blockDim = dim3(TM * G);
        cudaLaunchAttribute a[1];
        a[0].id = cudaLaunchAttributeClusterDimension;
        a[0].val.clusterDim.x = (unsigned)cl;
        a[0].val.clusterDim.y = 1;
        a[0].val.clusterDim.z = 1;
        cfg.attrs = a;
        cfg.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(n, mrs_f32_cluster<TM, G, COMP, UNROLL>, &cfg);
    }
    return e == cudaSuccess ? MRS_OK : MRS_ECUDA;
}

#define MRS_CASE_CL(id, TM, G, U, FN, ...) \
    case id:                              \
        return comp ? FN<TM, G, true, U>(__VA_ARGS__) : FN<TM, G, false, U>(__VA_ARGS__);
#define MRS_DISPATCH_CL(cfg, comp, FN, ...)          \
    switch (cfg) {                                   \
        MRS_CASE_CL(27, 32, 8, 1, FN, __VA_ARGS__)   \
        MRS_CASE_CL(28, 64, 4, 1, FN, __VA_ARGS__)   \
    default: break;                                  \
    }

cudaError_t launch_mrs_f32(int config, bool comp, const MrsLaunch& L, cudaStream_t s)
{
    if (config >= 0 && config < kNumConfigs && kConfigs[config].cluster) {
        MRS_DISPATCH_CL(config, comp, launch_cl_t, L, s);
        return cudaErrorInvalidValue;
    }
    MRS_DISPATCH(config, comp, launch_t, L, s);
    return cudaErrorInvalidValue;
}

int occupancy_f32(int config, bool comp, int* ctas_per_sm)
{
    if (config >= 0 && config < kNumConfigs && kConfigs[config].cluster) {
        MRS_DISPATCH_CL(config, comp, occ_cl_t, ctas_per_sm);
        return MRS_EINVAL;
    }
    MRS_DISPATCH(config, comp, occ_t, ctas_per_sm);
    return MRS_EINVAL;
}

int cluster_setup_f32(int config, bool comp, int cl, int* max_clusters)
{
    MRS_DISPATCH_CL(config, comp, setup_cl_t, cl, max_clusters);
    return MRS_EINVAL;
}

// ---------------------------------------------------------------------------------------------
// Float64 kernel.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kF64Block) mrs_f64_kernel(const MrsLaunch64 L)
{
    pdl_wait();
    __shared__ double sx[kF64Block * 9];
    const int b = blockIdx.x;
    const int sys = L.tile_sys[b];
    const long long s0 = L.offsets[sys], s1 = L.offsets[sys + 1];
    const long long i = (long long)L.tile_t0[b] + threadIdx.x;
    const bool valid = i < s1;
    const long long ii = valid ? i : s1 - 1;
    const double xi = L.Xt[ii * 3 + 0], yi = L.Xt[ii * 3 + 1], zi = L.Xt[ii * 3 + 2];
    const double e2 = L.eps[sys] * L.eps[sys];
    double u0 = 0, u1 = 0, u2 = 0, w0 = 0, w1 = 0, w2 = 0;
    for (long long j0 = s0; j0 < s1; j0 += kF64Block) {
        const int cnt = (int)min((long long)kF64Block, s1 - j0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < cnt * 3; idx += kF64Block) {
            const int sidx = idx / 3, c = idx - sidx * 3;
            sx[sidx * 9 + c] = L.X[j0 * 3 + idx];
            sx[sidx * 9 + 3 + c] = L.f[j0 * 3 + idx];
            sx[sidx * 9 + 6 + c] = L.n[j0 * 3 + idx];
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const double* q = sx + j * 9;
            const double rx = xi - q[0], ry = yi - q[1], rz = zi - q[2];
            const double r2 = rx * rx + ry * ry + rz * rz;
            const double s = rsqrt(r2 + e2);
            const double s2 = s * s, s3 = s2 * s, s5 = s3 * s2, s7 = s5 * s2;
            // 8 pi H1..H5
            const double h1 = (r2 + 2.0 * e2) * s3;
            const double h2 = s3;
            const double h3 = 0.5 * (2.0 * r2 + 5.0 * e2) * s5;
            const double h4 = 0.25 * (10.0 * e2 * e2 - 7.0 * e2 * r2 - 2.0 * r2 * r2) * s7;
            const double h5 = 0.25 * (6.0 * r2 + 21.0 * e2) * s7;
            const double fx = q[3], fy = q[4], fz = q[5], nx = q[6], ny = q[7], nz = q[8];
            const double fr = fx * rx + fy * ry + fz * rz;
            const double nr = nx * rx + ny * ry + nz * rz;
            u0 += h1 * fx + h2 * fr * rx + h3 * (ny * rz - nz * ry);
            u1 += h1 * fy + h2 * fr * ry + h3 * (nz * rx - nx * rz);
            u2 += h1 * fz + h2 * fr * rz + h3 * (nx * ry - ny * rx);
            w0 += h3 * (fy * rz - fz * ry) + h4 * nx + h5 * nr * rx;
            w1 += h3 * (fz * rx - fx * rz) + h4 * ny + h5 * nr * ry;
            w2 += h3 * (fx * ry - fy * rx) + h4 * nz + h5 * nr * rz;
        }
    }
    if (valid) {
        const double sc = L.inv_mu / (8.0 * 3.14159265358979323846);
        if (!isfinite(u0 + u1 + u2 + w0 + w1 + w2)) atomicOr(L.err, 1u);
        L.u[i * 3 + 0] = u0 * sc;
        L.u[i * 3 + 1] = u1 * sc;
        L.u[i * 3 + 2] = u2 * sc;
        L.w[i * 3 + 0] = w0 * sc;
        L.w[i * 3 + 1] = w1 * sc;
        L.w[i * 3 + 2] = w2 * sc;
    }
}

cudaError_t launch_mrs_f64(const MrsLaunch64& L, cudaStream_t s)
{
    if (L.n_blocks == 0) return cudaSuccess;
    cudaError_t e = launch_pdl(mrs_f64_kernel, dim3(L.n_blocks), dim3(kF64Block), 0, s, L);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace mrs
