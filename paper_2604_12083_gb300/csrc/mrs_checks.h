// mrs_checks.h -- index checks of the debug build (compiled with -DMRS_DEBUG_BOUNDS=1).
//
// The kernels index their inputs, outputs and scratch through tables the host builds (work
// tiles, row and column partial slots, rod node tables).  In the debug build every kernel
// checks the entries it uses with the predicates below before touching memory through them; a
// failed check raises MRS_FLAG_BOUNDS in the context's device error word (reported by
// mrs_device_status) and the access is skipped -- nothing traps.  The release build compiles
// the checks out.  The predicates are plain host/device functions, so the host-side tests
// exercise them on tables with planted mistakes.
#pragma once

#include "mrs_internal.h"

#ifndef MRS_DEBUG_BOUNDS
#define MRS_DEBUG_BOUNDS 0
#endif

namespace mrs {

// A symmetric work tile (SymTile) against its pass: TM targets at most, inside its system and
// the point arrays, unit counts consistent with its extent, its units inside the pass's column
// buffer [U0, U0 + col_units) and its row segments inside the pass's row buffer.
__host__ __device__ inline bool sym_tile_ok(const SymTile& T, int TM, long long n_points,
                                            long long U0, long long col_units, long long row_segs)
{
    if (T.tn < 1 || T.tn > TM || T.t0 < 0) return false;
    if ((long long)T.t0 + T.tn > T.send || T.send > n_points) return false;
    if (T.nu != (T.send - T.t0 + kUnitSources - 1) / kUnitSources) return false;
    if (T.nd != (T.tn + kUnitSources - 1) / kUnitSources || T.nd > T.nu) return false;
    if (T.u0 < U0 || T.u0 - U0 + T.nu > col_units) return false;
    if (T.seg0 < 0 || T.nseg < 1 || (long long)T.seg0 + T.nseg > row_segs) return false;
    return T.tfirst >= 0 && T.kt >= 0;
}

// An ordered work tile (TileDesc): TM targets at most inside the target array, its system's
// sources inside the source array, unit count consistent with the system's size.
__host__ __device__ inline bool ordered_tile_ok(const TileDesc& T, int TM, long long n_points)
{
    if (T.tn < 1 || T.tn > TM || T.t0 < 0 || (long long)T.t0 + T.tn > n_points) return false;
    if (T.s0 < 0 || T.sn < 1 || (long long)T.s0 + T.sn > n_points) return false;
    return T.nu == (T.sn + kUnitSources - 1) / kUnitSources && T.u0 >= 0;
}

// A rod node table entry (index within its rod, nodes of the rod) of node k of N: the rod has
// at least two nodes and lies inside [0, N).
__host__ __device__ inline bool rod_node_ok(int2 ni, long long k, long long N)
{
    return ni.y >= 2 && ni.x >= 0 && ni.x < ni.y && k - ni.x >= 0 && k - ni.x + ni.y <= N;
}

}  // namespace mrs
