// Host-only driver for tests/test_debug_checks.py: evaluates the debug build's index
// predicates (csrc/mrs_checks.h) on a valid work tile / node entry and on copies with one
// planted mistake each, and prints one line "<case> <0|1>" per evaluation (1 = accepted).
#include <cstdio>

#include "mrs_checks.h"

using namespace mrs;

int main()
{
    // a valid symmetric tile: 384 targets from point 0 of a 1000-point system, 32 units
    // (1000 / 32 rounded up), 12 diagonal units, row segments 0..2 of a 10-segment buffer
    SymTile S{};
    S.sys = 0;
    S.t0 = 0;
    S.tn = 384;
    S.send = 1000;
    S.nu = 32;
    S.nd = 12;
    S.kt = 0;
    S.tfirst = 0;
    S.seg0 = 0;
    S.nseg = 3;
    S.qlo = 0;
    S.u0 = 40;
    const int TM = 384;
    const long long NP = 1000, U0 = 40, CU = 100, RS = 10;
    auto sym = [&](const char* name, const SymTile& T) {
        printf("sym_%s %d\n", name, sym_tile_ok(T, TM, NP, U0, CU, RS) ? 1 : 0);
    };
    sym("valid", S);
    SymTile T;
    T = S; T.tn = 385; sym("tn_above_TM", T);
    T = S; T.tn = 0; sym("tn_zero", T);
    T = S; T.t0 = -1; sym("t0_negative", T);
    T = S; T.send = 1001; T.nu = 32; sym("send_past_points", T);
    T = S; T.t0 = 700; T.nu = 10; T.nd = 10; sym("tile_past_system", T);
    T = S; T.nu = 31; sym("units_short", T);
    T = S; T.nd = 11; sym("diagonal_short", T);
    T = S; T.u0 = 39; sym("units_before_pass", T);
    T = S; T.u0 = 109; sym("units_past_buffer", T);
    T = S; T.seg0 = 8; sym("segments_past_buffer", T);
    T = S; T.nseg = 0; sym("no_segment", T);

    // a valid ordered tile: targets 256..511 of a 1000-point system starting at point 0
    TileDesc O{};
    O.sys = 0;
    O.t0 = 256;
    O.tn = 256;
    O.s0 = 0;
    O.sn = 1000;
    O.nu = 32;
    O.u0 = 32;
    auto ord = [&](const char* name, const TileDesc& D) {
        printf("ordered_%s %d\n", name, ordered_tile_ok(D, 256, NP) ? 1 : 0);
    };
    ord("valid", O);
    TileDesc D;
    D = O; D.tn = 257; ord("tn_above_TM", D);
    D = O; D.t0 = 800; ord("targets_past_points", D);
    D = O; D.s0 = 1; ord("sources_past_points", D);
    D = O; D.nu = 33; ord("units_wrong", D);
    D = O; D.s0 = -5; D.sn = 1005; D.nu = 32; ord("sources_negative", D);

    // node 13 of 20, index 3 in a rod of 10 nodes (nodes 10..19)
    auto node = [&](const char* name, int x, int y, long long k) {
        printf("node_%s %d\n", name, rod_node_ok(make_int2(x, y), k, 20) ? 1 : 0);
    };
    node("valid", 3, 10, 13);
    node("one_node_rod", 0, 1, 13);
    node("index_at_length", 10, 10, 13);
    node("index_negative", -1, 10, 13);
    node("rod_before_zero", 3, 10, 2);
    node("rod_past_end", 3, 10, 16);
    return 0;
}
