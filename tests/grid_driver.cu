// Host-only driver for tests/test_grid_rules.py: evaluates the persistent grid rules of the
// ordered pair sum (ordered_ctas: the per-tile split cap; balanced_ctas: one 256-thread CTA per
// SM when the full grid gives each little work) and the tile size of a configuration
// (tile_targets) on the shapes they were measured on, and prints "<case> <value>" lines.
#include <cstdio>

#include "mrs_internal.h"

using namespace mrs;

static long long grid(long long N, int TM, int occ, int threads, int sms = 152)
{
    const long long tiles = (N + TM - 1) / TM, nu = (N + kUnitSources - 1) / kUnitSources;
    const long long W = tiles * nu, full = (long long)sms * occ;
    return balanced_ctas(ordered_ctas(full, W, nu), full, W, sms, threads);
}

int main()
{
    // 256 threads x 1 target (256-target tiles), 3 CTAs per SM
    printf("p256_3072 %lld\n", grid(3072, 256, 3, 256));
    printf("p256_4096 %lld\n", grid(4096, 256, 3, 256));
    printf("p256_6144 %lld\n", grid(6144, 256, 3, 256));
    printf("p256_8192 %lld\n", grid(8192, 256, 3, 256));
    // 64 threads x 4 targets (256-target tiles), 8 CTAs per SM: the cap alone
    printf("p64_2560 %lld\n", grid(2560, 256, 8, 64));
    // fewer units than SMs: one unit per CTA
    printf("p256_300 %lld\n", grid(300, 256, 3, 256));
    // the cap alone (units >= 4 per CTA of the full grid is not met, 128-thread CTAs)
    printf("p128_2048 %lld\n", grid(2048, 128, 6, 128));
    KernelConfig a{256, 1, 1, 1, 0, 0, 0, 16, 8}, b{256, 1, 1, 1, 0, 0, 0, 16, 4}, c{64, 6, 1, 1, 1, 1, 4};
    printf("tm_cluster8 %d\n", tile_targets(a));
    printf("tm_cluster4 %d\n", tile_targets(b));
    printf("tm_sym %d\n", tile_targets(c));
    return 0;
}
