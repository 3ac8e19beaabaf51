// autotune.cu -- choice of the pair-sum kernel configuration by measurement.
//
// mrs_autotune times every compiled configuration (threads per CTA, targets per thread, scalar
// or packed f32x2 inner loop) on the caller's batch shape, with synthetic inputs generated on
// the device, and records the fastest per shape bucket in the context.  Plans built with
// config = -1 look the bucket up first and fall back to the built-in heuristic.  The table can
// be written to / read from a small JSON file.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "mrs_internal.h"

namespace mrs {

static int ilog2_ceil(int64_t v)
{
    int l = 0;
    while (((int64_t)1 << l) < v) ++l;
    return l;
}

TuneKey tune_key(int n_sys, const int64_t* offsets, int precision)
{
    int64_t mx = 0;
    for (int s = 0; s < n_sys; ++s) mx = std::max<int64_t>(mx, offsets[s + 1] - offsets[s]);
    TuneKey k;
    k.precision = precision;
    k.sys_log2 = ilog2_ceil(n_sys);
    k.n_log2 = ilog2_ceil(offsets[n_sys]);
    k.max_log2 = ilog2_ceil(mx);
    return k;
}

int tuned_config(const mrs_ctx* ctx, const TuneKey& k)
{
    for (const TuneEntry& e : ctx->tuned)
        if (e.key == k) return e.config;
    return -1;
}

// Deterministic synthetic inputs: points on a jittered lattice of spacing h, unit-size forces.
__global__ void autotune_fill_kernel(int N, float h, float* X, float* f, float* n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int side = 64;
    const float jx = 0.25f * __sinf(1.7f * i), jy = 0.25f * __cosf(2.3f * i), jz = 0.25f * __sinf(0.9f * i + 1.f);
    X[3 * i + 0] = h * ((i % side) + jx);
    X[3 * i + 1] = h * (((i / side) % side) + jy);
    X[3 * i + 2] = h * ((i / (side * side)) + jz);
    for (int c = 0; c < 3; ++c) {
        f[3 * i + c] = __sinf(0.37f * i + c);
        n[3 * i + c] = __cosf(0.53f * i + 2.f * c);
    }
}

}  // namespace mrs

using namespace mrs;

extern "C" {

int mrs_autotune(mrs_ctx* ctx, int n_sys, const int64_t* offsets, double mu, double eps,
                 const double* eps_per_sys, int precision, int reps, int* best_config,
                 float* best_ms)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr && offsets != nullptr && n_sys >= 1, "bad arguments");
    MRS_REQUIRE(precision == MRS_F32 || precision == MRS_F32_COMP,
                "autotuning applies to the float32 pair sum");
    MRS_REQUIRE(reps >= 1 && reps <= 1000, "reps must be in 1..1000");
    const int64_t N = offsets[n_sys];
    MRS_REQUIRE(N >= 1, "empty batch");
    MRS_CHECK_CUDA(cudaSetDevice(ctx->device));
    float *X = nullptr, *f = nullptr, *n = nullptr, *u = nullptr, *w = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    int st = MRS_OK;
    cudaError_t e = cudaMalloc(&X, 12 * N);
    if (!e) e = cudaMalloc(&f, 12 * N);
    if (!e) e = cudaMalloc(&n, 12 * N);
    if (!e) e = cudaMalloc(&u, 12 * N);
    if (!e) e = cudaMalloc(&w, 12 * N);
    if (!e) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreate(&a);
    if (!e) e = cudaEventCreate(&b);
    if (!e) {
        autotune_fill_kernel<<<(int)((N + 127) / 128), 128, 0, s>>>((int)N, 0.01f, X, f, n);
        e = cudaGetLastError();
    }
    int best = -1;
    float best_t = INFINITY;
    for (int cfg = 0; cfg < kNumConfigs && !e && st == MRS_OK; ++cfg) {
        mrs_plan* p = nullptr;
        st = plan_build(ctx, n_sys, offsets, mu, eps, eps_per_sys, precision, cfg, &p);
        if (st) break;
        float t = INFINITY;
        st = plan_run(p, X, f, n, nullptr, u, w, s);   // warm-up
        for (int r = 0; r < reps && st == MRS_OK && !e; ++r) {
            e = cudaEventRecord(a, s);
            if (!e) st = plan_run(p, X, f, n, nullptr, u, w, s);
            if (!e) e = cudaEventRecord(b, s);
            if (!e) e = cudaEventSynchronize(b);
            float ms = 0.f;
            if (!e) e = cudaEventElapsedTime(&ms, a, b);
            if (!e && ms < t) t = ms;
        }
        cudaStreamSynchronize(s);
        plan_free(p);
        if (t < best_t) {
            best_t = t;
            best = cfg;
        }
    }
    cudaFree(X);
    cudaFree(f);
    cudaFree(n);
    cudaFree(u);
    cudaFree(w);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
    if (e) {
        set_error("autotuning failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    if (st) return st;
    const TuneKey k = tune_key(n_sys, offsets, precision);
    bool found = false;
    for (TuneEntry& te : ctx->tuned)
        if (te.key == k) {
            te.config = best;
            te.ms = best_t;
            found = true;
        }
    if (!found) ctx->tuned.push_back(TuneEntry{k, best, best_t});
    if (best_config) *best_config = best;
    if (best_ms) *best_ms = best_t;
    return MRS_OK;
}

int mrs_autotune_save(const mrs_ctx* ctx, const char* path)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr && path != nullptr, "NULL argument");
    FILE* fp = std::fopen(path, "w");
    MRS_REQUIRE(fp != nullptr, "cannot open %s for writing", path);
    std::fprintf(fp, "{\"sm\": \"%d%d\", \"entries\": [", ctx->cc_major, ctx->cc_minor);
    for (size_t i = 0; i < ctx->tuned.size(); ++i) {
        const TuneEntry& t = ctx->tuned[i];
        std::fprintf(fp, "%s\n {\"precision\": %d, \"sys_log2\": %d, \"n_log2\": %d, \"max_log2\": %d, "
                         "\"config\": %d, \"ms\": %.6f}",
                     i ? "," : "", t.key.precision, t.key.sys_log2, t.key.n_log2, t.key.max_log2,
                     t.config, t.ms);
    }
    std::fprintf(fp, "\n]}\n");
    std::fclose(fp);
    return MRS_OK;
}

int mrs_autotune_load(mrs_ctx* ctx, const char* path)
{
    clear_error();
    MRS_REQUIRE(ctx != nullptr && path != nullptr, "NULL argument");
    FILE* fp = std::fopen(path, "r");
    MRS_REQUIRE(fp != nullptr, "cannot open %s", path);
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof(buf), fp)) > 0) text.append(buf, got);
    std::fclose(fp);
    char want[16];
    std::snprintf(want, sizeof(want), "\"%d%d\"", ctx->cc_major, ctx->cc_minor);
    MRS_REQUIRE(text.find(want) != std::string::npos, "%s was tuned for another architecture", path);
    size_t pos = 0;
    int loaded = 0;
    while ((pos = text.find("{\"precision\"", pos)) != std::string::npos) {
        TuneEntry t;
        if (std::sscanf(text.c_str() + pos,
                        "{\"precision\": %d, \"sys_log2\": %d, \"n_log2\": %d, \"max_log2\": %d, "
                        "\"config\": %d, \"ms\": %f}",
                        &t.key.precision, &t.key.sys_log2, &t.key.n_log2, &t.key.max_log2, &t.config,
                        &t.ms) == 6 &&
            t.config >= 0 && t.config < kNumConfigs) {
            bool found = false;
            for (TuneEntry& te : ctx->tuned)
                if (te.key == t.key) {
                    te = t;
                    found = true;
                }
            if (!found) ctx->tuned.push_back(t);
            ++loaded;
        }
        ++pos;
    }
    MRS_REQUIRE(loaded > 0, "no tuning entries in %s", path);
    return MRS_OK;
}

}  // extern "C"
