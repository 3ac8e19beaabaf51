// noalloc.cu -- mrs_velocity_noalloc: the float32 compensated pair sum with no device allocation.
//
// Some callers cannot call cudaMalloc: code whose device memory is entirely owned by another
// allocator (a framework's caching pool, a fixed budget carved out at start-up), latency-
// critical loops that cannot afford cudaMalloc's implicit device synchronisation, and code
// that runs while another component is capturing the stream.  For them this file keeps the
// scratch of the persistent pair-sum kernel -- its work table, per-system constants, partial
// result slots and per-tile counters -- in one file-scope __device__ array of fixed size that
// every GPU loading the library holds until the process exits.
//
// The entry point launches two kernels on the caller's stream: a set-up kernel that writes the
// work table into the array and zeroes the tile counters, then the same persistent pair-sum
// kernel mrs_velocity uses (config: 128 threads x 2 targets per thread).  It calls no
// cudaMalloc, cudaFree or allocating library routine.  Host code never uses the array's name as
// an address: the device address comes from cudaGetSymbolAddress, taken once per device (with
// that device current) by the first call on that device.
#include <cmath>
#include <mutex>

#include "mrs_internal.h"

namespace mrs {

namespace {

constexpr int kNaConfig = 1;                         // 128 threads x 2 targets per thread
constexpr int kNaTM = 256;                           // targets per tile for that config
constexpr long long kNaMaxPoints = 1LL << 20;        // largest accepted system
constexpr int kNaMaxTiles = (int)(kNaMaxPoints / kNaTM);
constexpr int kNaMaxCTAs = 768;                      // persistent CTAs (>= 5 per SM x 152 SMs)
constexpr size_t kNaPartialBytes = (size_t)2 * kNaMaxCTAs * 6 * kNaTM * sizeof(float);
constexpr size_t kNaTilesBytes = (size_t)kNaMaxTiles * sizeof(TileDesc);
constexpr size_t kNaCountersBytes = (size_t)kNaMaxTiles * sizeof(int);
constexpr size_t kNaOffTiles = 0;
constexpr size_t kNaOffCounters = kNaOffTiles + kNaTilesBytes;
constexpr size_t kNaOffConst = kNaOffCounters + kNaCountersBytes;
constexpr size_t kNaOffErr = kNaOffConst + sizeof(SysConst);
constexpr size_t kNaOffPartial = (kNaOffErr + sizeof(unsigned int) + 255) / 256 * 256;
constexpr size_t kNaScratchBytes = kNaOffPartial + kNaPartialBytes;   // ~9.1 MiB

}  // namespace

// The scratch every call shares (zero-initialised when the module loads).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

__global__ void noalloc_setup_kernel(TileDesc* tiles, int* counters, SysConst* sc, int n_points,
                                     int n_tiles, int nu, SysConst c)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *sc = c;
    if (i < n_tiles) {
        TileDesc T;
        T.sys = 0;
        T.t0 = i * kNaTM;
        T.tn = min(kNaTM, n_points - i * kNaTM);
        T.s0 = 0;
        T.sn = n_points;
        T.nu = nu;
        T.u0 = (long long)i * nu;
        tiles[i] = T;
        counters[i] = 0;   // every tile counter starts at zero
    }
}

namespace {

std::mutex g_na_lock;
unsigned char* g_na_addr[64] = {};   // device address of the array, per device ordinal
int g_na_ctas[64] = {};              // persistent grid size, per device ordinal

int na_setup(int dev, unsigned char** addr, int* ctas)
{
    std::lock_guard<std::mutex> g(g_na_lock);
    if (g_na_addr[dev] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("cudaGetSymbolAddress of the no-allocation scratch failed on device %d: %s",
                      dev, cudaGetErrorString(e));
            return MRS_ECUDA;
        }
        int sms = 0, occ = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            set_error("cudaDeviceGetAttribute failed: %s", cudaGetErrorString(e));
            return MRS_ECUDA;
        }
        if (occupancy_f32(kNaConfig, true, &occ) != MRS_OK || occ < 1) {
            set_error("occupancy query failed for the no-allocation pair sum");
            return MRS_ECUDA;
        }
        long long P = (long long)sms * occ;
        g_na_ctas[dev] = (int)(P < kNaMaxCTAs ? P : kNaMaxCTAs);
        g_na_addr[dev] = (unsigned char*)p;
    }
    *addr = g_na_addr[dev];
    *ctas = g_na_ctas[dev];
    return MRS_OK;
}

bool na_overlap(const void* a, size_t na, const void* b, size_t nb)
{
    const char* pa = (const char*)a;
    const char* pb = (const char*)b;
    return pa < pb + nb && pb < pa + na;
}

}  // namespace
}  // namespace mrs

using namespace mrs;

extern "C" int mrs_velocity_noalloc(int64_t n_points, const float* X, const float* f,
                                    const float* n, float* u, float* w, double mu, double eps,
                                    void* stream)
{
    clear_error();
    MRS_REQUIRE(n_points >= 0, "n_points must be >= 0");
    MRS_REQUIRE(n_points <= kNaMaxPoints,
                "mrs_velocity_noalloc accepts at most %lld points (got %lld): its scratch is a "
                "fixed %zu-byte device array; use mrs_velocity for larger systems",
                kNaMaxPoints, (long long)n_points, kNaScratchBytes);
    MRS_REQUIRE(std::isfinite(mu) && mu > 0.0, "mu must be > 0 (got %g)", mu);
    MRS_REQUIRE(std::isfinite(eps) && eps > 0.0, "eps must be > 0 (got %g)", eps);
    if (n_points == 0) return MRS_OK;
    MRS_REQUIRE(X && f && n && u && w, "NULL input or output pointer");
    // persistent CTAs write u, w for finished tiles while others still read X, f, n as
    // sources, so an output aliasing an input gives silently wrong sums; a float pointer that
    // is not 4-byte aligned would fault the kernel: both are rejected before any launch
    const size_t bytes = (size_t)n_points * 3 * sizeof(float);
    const void* ins[3] = {X, f, n};
    for (int i = 0; i < 3; ++i)
        MRS_REQUIRE(!na_overlap(ins[i], bytes, u, bytes) && !na_overlap(ins[i], bytes, w, bytes),
                    "outputs must not overlap the inputs");
    MRS_REQUIRE(!na_overlap(u, bytes, w, bytes), "u and w must not overlap");
    MRS_REQUIRE(((uintptr_t)X | (uintptr_t)f | (uintptr_t)n | (uintptr_t)u | (uintptr_t)w) %
                        sizeof(float) == 0,
                "pointers must be aligned to 4 bytes (float32)");
    int dev = 0;
    MRS_CHECK_CUDA(cudaGetDevice(&dev));
    MRS_REQUIRE(dev >= 0 && dev < 64, "device ordinal %d not supported", dev);
    unsigned char* base = nullptr;
    int P = 0;
    int st = na_setup(dev, &base, &P);
    if (st) return st;

    const int N = (int)n_points;
    const int n_tiles = (N + kNaTM - 1) / kNaTM;
    const int nu = (N + kUnitSources - 1) / kUnitSources;
    const long long W = (long long)n_tiles * nu;
    P = (int)ordered_ctas(P, W, nu);
    const double e2 = eps * eps;
    SysConst c;
    c.e2 = (float)e2;
    c.c1 = (float)(1.5 * e2);
    c.c2 = (float)(3.75 * e2 * e2);
    c.c3 = (float)(-0.75 * e2);
    c.c5 = (float)(3.75 * e2);
    c.scale = (float)(1.0 / (8.0 * 3.14159265358979323846 * mu));

    TileDesc* tiles = (TileDesc*)(base + kNaOffTiles);
    int* counters = (int*)(base + kNaOffCounters);
    SysConst* sc = (SysConst*)(base + kNaOffConst);
    float* partial = (float*)(base + kNaOffPartial);
    cudaStream_t s = (cudaStream_t)stream;
    noalloc_setup_kernel<<<(n_tiles + 127) / 128, 128, 0, s>>>(tiles, counters, sc, N, n_tiles, nu, c);
    MRS_CHECK_CUDA(cudaGetLastError());

    MrsLaunch L;
    L.tiles = tiles;
    L.n_tiles = n_tiles;
    L.W = W;
    L.P = P;
    L.sc = sc;
    L.X = X;
    L.f = f;
    L.n = n;
    L.Xt = X;
    L.u = u;
    L.w = w;
    L.partial = partial;
    L.counters = counters;
    L.n_points = N;
    // the kernel's non-finite-input flag goes to a word of the array that is never read back:
    // this entry point does not report non-finite inputs (the outputs carry the NaN/Inf)
    L.err = (unsigned int*)(base + kNaOffErr);
    cudaError_t e = launch_mrs_f32(kNaConfig, true, L, s);
    if (e != cudaSuccess) {
        set_error("pair-sum launch failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    return MRS_OK;
}
