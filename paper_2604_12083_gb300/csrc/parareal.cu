// parareal.cu -- Parareal on one GPU (Section II-D, Eqs. initial, intermediate, serial_correct;
// Eq. true_err for the stopping increment).
//
// States of all slice ends live on the device: U[n] = (X, D) at T_n, n = 0..Ns, and the coarse
// values G(T_n, T_{n-1}, U^{k-1}_{n-1}) kept from the previous iteration.  Iteration k:
//   1. the fine solves of the open slices n = k..Ns start from U[k-1..Ns-1] (contiguous rows)
//      and run together as Ns-k+1 independent systems of one batched workspace: every stage
//      of every RK2 step is one rod-force pass and ONE persistent pair-sum launch over all
//      instances (replayed from a captured graph);
//   2. U[k] = F'[k]; then serially for n = k+1..Ns: G(U^k_{n-1}) by explicit Euler, and
//      U[n] = F'[n] + G(U^k_{n-1}) - G(U^{k-1}_{n-1}) in float64, followed by polar
//      re-orthonormalisation of every frame (Newton-Schulz iteration);
//   3. eta~^k = max over nodes and slices n >= k of |x^k - x^{k-1}| / |x^k| (positions) is
//      reduced on the device and read back; stop when it falls below tol.
#include <chrono>
#include <cmath>
#include <cstring>

#include "rod_internal.h"

namespace mrs {

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* a, double v)
{
    // non-negative doubles order like their bit patterns
    if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000LL);   // NaN -> +inf
    atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// Nearest rotation of a 3x3 matrix close to one: Q <- (3I - Q Q^T) Q / 2, four times.
__device__ __forceinline__ void polar_newton_schulz(double* Q)
{
#pragma unroll
    for (int it = 0; it < 4; ++it) {
        double S[9], Qn[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                S[3 * r + c] = (r == c ? 3.0 : 0.0) -
                               (Q[3 * r] * Q[3 * c] + Q[3 * r + 1] * Q[3 * c + 1] + Q[3 * r + 2] * Q[3 * c + 2]);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Qn[3 * r + c] = 0.5 * (S[3 * r] * Q[c] + S[3 * r + 1] * Q[3 + c] + S[3 * r + 2] * Q[6 + c]);
#pragma unroll
        for (int q = 0; q < 9; ++q) Q[q] = Qn[q];
    }
}

// Slice n of iteration k.  Fp*: the fine result F'[n]; Gn*: G(U^k_{n-1}) (NULL for n = k, where
// U[k] = F'[k]); Go*: G(U^{k-1}_{n-1}) on entry, replaced by Gn* on exit; U*: U^{k-1}[n] on
// entry, U^k[n] on exit.
__global__ void parareal_correct_kernel(int N1, const double* __restrict__ FpX,
                                        const double* __restrict__ FpD, const double* GnX,
                                        const double* GnD, double* GoX, double* GoD, double* UX,
                                        double* UD, unsigned long long* incr)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N1) return;
    double x[3], Dm[9];
    if (GnX) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t i = 3 * (size_t)k + c;
            x[c] = FpX[i] + GnX[i] - GoX[i];
            GoX[i] = GnX[i];
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const size_t i = 9 * (size_t)k + q;
            Dm[q] = FpD[i] + GnD[i] - GoD[i];
            GoD[i] = GnD[i];
        }
        polar_newton_schulz(Dm);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) x[c] = FpX[3 * (size_t)k + c];
#pragma unroll
        for (int q = 0; q < 9; ++q) Dm[q] = FpD[9 * (size_t)k + q];
    }
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double d = x[c] - UX[3 * (size_t)k + c];
        num += d * d;
        den += x[c] * x[c];
        UX[3 * (size_t)k + c] = x[c];
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) UD[9 * (size_t)k + q] = Dm[q];
    atomic_max_nonneg(incr, den > 0.0 ? sqrt(num / den) : sqrt(num));
}

cudaError_t launch_parareal_correct(int N1, const double* FpX, const double* FpD, const double* GnX,
                                    const double* GnD, double* GoX, double* GoD, double* UX,
                                    double* UD, double* incr, cudaStream_t s)
{
    parareal_correct_kernel<<<(N1 + 127) / 128, 128, 0, s>>>(N1, FpX, FpD, GnX, GnD, GoX, GoD, UX, UD,
                                                             (unsigned long long*)incr);
    return cudaGetLastError();
}

}  // namespace mrs

using namespace mrs;

namespace {

struct DevBuf {
    double* p = nullptr;
    ~DevBuf() { cudaFree(p); }
};

int alloc_d(DevBuf& b, size_t n)
{
    cudaError_t e = cudaMalloc((void**)&b.p, n * sizeof(double));
    if (e != cudaSuccess) {
        b.p = nullptr;
        set_error("cudaMalloc of %zu bytes failed: %s", n * sizeof(double), cudaGetErrorString(e));
        return MRS_ENOMEM;
    }
    return MRS_OK;
}

}  // namespace

extern "C" int parareal_run(mrs_ctx* ctx, int n_rods, const int64_t* rod_off,
                            const mrs_rod_params* p, double* X, double* D, double T0, double T1,
                            int n_slices, double dt_fine, int coarse_ratio, int max_iter,
                            double tol, mrs_parareal_stats* out, void* stream)
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
    MRS_REQUIRE(std::isfinite(T0) && std::isfinite(T1) && T1 > T0, "need T1 > T0");
    MRS_REQUIRE(dt_fine > 0.0 && coarse_ratio >= 1, "need dt_fine > 0 and coarse_ratio >= 1");
    MRS_REQUIRE(max_iter >= 1, "max_iter must be >= 1");
    const double dT = (T1 - T0) / n_slices;
    const long long n_fine = llround(dT / dt_fine);
    MRS_REQUIRE(n_fine >= 1 && std::fabs(n_fine * dt_fine - dT) <= 1e-9 * dT,
                "the slice length must be a whole number of fine steps");
    MRS_REQUIRE(n_fine % coarse_ratio == 0, "the slice length must be a whole number of coarse steps");
    MRS_REQUIRE(n_fine <= 0x7fffffff, "too many fine steps per slice");
    const int n_coarse = (int)(n_fine / coarse_ratio);
    const double dt_coarse = dt_fine * coarse_ratio;
    MRS_CHECK_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int Ns = n_slices;
    const size_t N1 = (size_t)rod_off[n_rods];
    const size_t sx = 3 * N1, sd = 9 * N1;   // doubles per state (positions, frames)

    int st;
    DevBuf UX, UD, GoX, GoD, FX, FD, WX, WD, INC;
    if ((st = alloc_d(UX, sx * (Ns + 1))) || (st = alloc_d(UD, sd * (Ns + 1))) ||
        (st = alloc_d(GoX, sx * (Ns + 1))) || (st = alloc_d(GoD, sd * (Ns + 1))) ||
        (st = alloc_d(FX, sx * Ns)) || (st = alloc_d(FD, sd * Ns)) || (st = alloc_d(WX, sx)) ||
        (st = alloc_d(WD, sd)) || (st = alloc_d(INC, 1)))
        return st;
    RodWorkspace* wsG = nullptr;
    if ((st = rod_ws_get(ctx, n_rods, rod_off, 1, MRS_F32_COMP, p->mu, p->eps, &wsG))) return st;

    const int nb = (int)((N1 + 127) / 128);
    long long fine_steps = 0, coarse_steps = 0;
    // coarse propagation of the work state (WX, WD) over slice n (from T_{n-1})
    auto coarse = [&](int n) -> int {
        int r = rod_ws_set_times(wsG, T0 + (n - 1) * dT, 0.0, s);
        if (r) return r;
        coarse_steps += n_coarse;
        return rod_ws_steps(wsG, p, WX.p, WD.p, dt_coarse, n_coarse, MRS_EULER, s);
    };
    auto cpy = [&](double* dst, const double* src, size_t n) -> int {
        MRS_CHECK_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        return MRS_OK;
    };

    // U[0] = x0; initial coarse sweep (Eq. initial)
    if ((st = cpy(UX.p, X, sx)) || (st = cpy(UD.p, D, sd))) return st;
    if ((st = cpy(WX.p, X, sx)) || (st = cpy(WD.p, D, sd))) return st;
    for (int n = 1; n <= Ns; ++n) {
        if ((st = coarse(n))) return st;
        if ((st = cpy(UX.p + n * sx, WX.p, sx)) || (st = cpy(UD.p + n * sd, WD.p, sd)) ||
            (st = cpy(GoX.p + n * sx, WX.p, sx)) || (st = cpy(GoD.p + n * sd, WD.p, sd)))
            return st;
    }

    mrs_parareal_stats stats;
    std::memset(&stats, 0, sizeof(stats));
    double last = INFINITY;
    int status = MRS_OK;
    for (int k = 1; k <= max_iter && k <= Ns; ++k) {
        // 1. fine solves of slices k..Ns from U[k-1..Ns-1], batched (Eq. intermediate)
        const int n_open = Ns - k + 1;
        RodWorkspace* wsF = nullptr;
        if ((st = rod_ws_get(ctx, n_rods, rod_off, n_open, MRS_F32_COMP, p->mu, p->eps, &wsF)))
            return st;
        if ((st = cpy(FX.p, UX.p + (k - 1) * sx, sx * n_open)) ||
            (st = cpy(FD.p, UD.p + (k - 1) * sd, sd * n_open)))
            return st;
        if ((st = rod_ws_set_times(wsF, T0 + (k - 1) * dT, dT, s))) return st;
        if ((st = rod_ws_steps(wsF, p, FX.p, FD.p, dt_fine, (int)n_fine, MRS_RK2, s))) return st;
        fine_steps += n_fine * n_open;
        MRS_CHECK_CUDA(cudaMemsetAsync(INC.p, 0, sizeof(double), s));
        // 2. U[k] = F'[k]; serial correction for n > k (Eq. serial_correct)
        parareal_correct_kernel<<<nb, 128, 0, s>>>((int)N1, FX.p, FD.p, nullptr, nullptr, nullptr,
                                                   nullptr, UX.p + k * sx, UD.p + k * sd,
                                                   (unsigned long long*)INC.p);
        MRS_CHECK_CUDA(cudaGetLastError());
        for (int n = k + 1; n <= Ns; ++n) {
            if ((st = cpy(WX.p, UX.p + (n - 1) * sx, sx)) || (st = cpy(WD.p, UD.p + (n - 1) * sd, sd)))
                return st;
            if ((st = coarse(n))) return st;
            parareal_correct_kernel<<<nb, 128, 0, s>>>(
                (int)N1, FX.p + (n - k) * sx, FD.p + (n - k) * sd, WX.p, WD.p, GoX.p + n * sx,
                GoD.p + n * sd, UX.p + n * sx, UD.p + n * sd, (unsigned long long*)INC.p);
            MRS_CHECK_CUDA(cudaGetLastError());
        }
        // 3. the increment (Eq. true_err, relative increment)
        double incr = 0.0;
        MRS_CHECK_CUDA(cudaMemcpyAsync(&incr, INC.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        MRS_CHECK_CUDA(cudaStreamSynchronize(s));
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
    if ((st = cpy(X, UX.p + Ns * sx, sx)) || (st = cpy(D, UD.p + Ns * sd, sd))) return st;
    MRS_CHECK_CUDA(cudaStreamSynchronize(s));
    stats.final_incr = last;
    stats.fine_steps = fine_steps;
    stats.coarse_steps = coarse_steps;
    stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - wall0).count();
    if (out) *out = stats;
    return status;
}
