// checkpoint.cu -- save / restore the state of a rod system (checkpoint and resume).
//
// File layout (little-endian): "MRSCKPT1" | int32 version = 1 | int32 n_rods | int64 N |
// float64 t | int64 rod_off[n_rods+1] | float64 X[N][3] | float64 D[N][3][3] |
// uint64 FNV-1a hash of everything before it.  X and D may live on the device or the host
// (copies use cudaMemcpyDefault).
#include <cstdio>
#include <cstring>
#include <vector>

#include "mrs_internal.h"

namespace {

constexpr char kMagic[8] = {'M', 'R', 'S', 'C', 'K', 'P', 'T', '1'};

uint64_t fnv1a(const void* p, size_t n, uint64_t h)
{
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ULL;
    }
    return h;
}

}  // namespace

using namespace mrs;

extern "C" {

int rod_checkpoint_save(const char* path, int n_rods, const int64_t* rod_off, const double* X,
                        const double* D, double t, void* stream)
{
    clear_error();
    MRS_REQUIRE(path && rod_off && X && D && n_rods >= 1 && rod_off[0] == 0, "bad arguments");
    const int64_t N = rod_off[n_rods];
    MRS_REQUIRE(N >= 1, "empty rod system");
    std::vector<double> hX(3 * (size_t)N), hD(9 * (size_t)N);
    cudaStream_t s = (cudaStream_t)stream;
    MRS_CHECK_CUDA(cudaMemcpyAsync(hX.data(), X, hX.size() * 8, cudaMemcpyDefault, s));
    MRS_CHECK_CUDA(cudaMemcpyAsync(hD.data(), D, hD.size() * 8, cudaMemcpyDefault, s));
    MRS_CHECK_CUDA(cudaStreamSynchronize(s));
    const int32_t version = 1, nr = n_rods;
    std::vector<unsigned char> buf;
    auto put = [&](const void* p, size_t n) {
        const unsigned char* b = (const unsigned char*)p;
        buf.insert(buf.end(), b, b + n);
    };
    put(kMagic, 8);
    put(&version, 4);
    put(&nr, 4);
    put(&N, 8);
    put(&t, 8);
    put(rod_off, 8 * (size_t)(n_rods + 1));
    put(hX.data(), hX.size() * 8);
    put(hD.data(), hD.size() * 8);
    const uint64_t h = fnv1a(buf.data(), buf.size(), 1469598103934665603ULL);
    put(&h, 8);
    std::FILE* fp = std::fopen(path, "wb");
    MRS_REQUIRE(fp != nullptr, "cannot open %s for writing", path);
    const size_t w = std::fwrite(buf.data(), 1, buf.size(), fp);
    const int cl = std::fclose(fp);
    MRS_REQUIRE(w == buf.size() && cl == 0, "short write to %s", path);
    return MRS_OK;
}

int rod_checkpoint_load(const char* path, int n_rods, const int64_t* rod_off, double* X, double* D,
                        double* t, void* stream)
{
    clear_error();
    MRS_REQUIRE(path && rod_off && X && D && t && n_rods >= 1, "bad arguments");
    std::FILE* fp = std::fopen(path, "rb");
    MRS_REQUIRE(fp != nullptr, "cannot open %s", path);
    std::vector<unsigned char> buf;
    unsigned char tmp[65536];
    size_t got;
    while ((got = std::fread(tmp, 1, sizeof(tmp), fp)) > 0) buf.insert(buf.end(), tmp, tmp + got);
    std::fclose(fp);
    const size_t head = 8 + 4 + 4 + 8 + 8;
    MRS_REQUIRE(buf.size() >= head + 8 && std::memcmp(buf.data(), kMagic, 8) == 0,
                "%s is not a rod checkpoint", path);
    int32_t version, nr;
    int64_t N;
    double tt;
    std::memcpy(&version, buf.data() + 8, 4);
    std::memcpy(&nr, buf.data() + 12, 4);
    std::memcpy(&N, buf.data() + 16, 8);
    std::memcpy(&tt, buf.data() + 24, 8);
    MRS_REQUIRE(version == 1, "unsupported checkpoint version %d", version);
    MRS_REQUIRE(nr == n_rods && N == rod_off[n_rods], "checkpoint holds %d rods / %lld nodes, caller "
                "expects %d / %lld", nr, (long long)N, n_rods, (long long)rod_off[n_rods]);
    const size_t body = head + 8 * (size_t)(nr + 1) + 8 * 12 * (size_t)N;
    MRS_REQUIRE(buf.size() == body + 8, "%s is truncated or has trailing data", path);
    uint64_t h;
    std::memcpy(&h, buf.data() + body, 8);
    MRS_REQUIRE(h == fnv1a(buf.data(), body, 1469598103934665603ULL), "%s is corrupted (hash mismatch)",
                path);
    MRS_REQUIRE(std::memcmp(buf.data() + head, rod_off, 8 * (size_t)(nr + 1)) == 0,
                "rod offsets differ from the checkpoint's");
    const unsigned char* px = buf.data() + head + 8 * (size_t)(nr + 1);
    cudaStream_t s = (cudaStream_t)stream;
    MRS_CHECK_CUDA(cudaMemcpyAsync(X, px, 24 * (size_t)N, cudaMemcpyDefault, s));
    MRS_CHECK_CUDA(cudaMemcpyAsync(D, px + 24 * (size_t)N, 72 * (size_t)N, cudaMemcpyDefault, s));
    MRS_CHECK_CUDA(cudaStreamSynchronize(s));
    *t = tt;
    return MRS_OK;
}

}  // extern "C"
