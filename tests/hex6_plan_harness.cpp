// Test harness: the six-directional window planner (csrc/hex6_plan.cpp) with a
// C interface, built on the CPU by tests/test_hex6_plan.py.
#include <string.h>

#include <vector>

#include "../paper_1003_2022_gb300/csrc/bsf_internal.h"

static std::vector<hex6_tile> g_tiles;
static std::vector<hex6_chunk> g_chunks;

extern "C" int plan_run(long long B, long long C, long long H, long long W, double h, const unsigned* ext,
                        unsigned long long budget, int* ntiles, int* nchunks) {
    const int s = hex6_plan(B, C, H, W, h, ext, (size_t)budget, g_tiles, g_chunks);
    *ntiles = (int)g_tiles.size();
    *nchunks = (int)g_chunks.size();
    return s;
}

// per tile: off, i_left, j0w, ncol, nrow, b, x0, y0, w, hh
extern "C" void plan_tiles(long long* out) {
    for (size_t t = 0; t < g_tiles.size(); ++t) {
        const hex6_tile& x = g_tiles[t];
        const long long v[10] = {x.off, x.i_left, x.j0w, x.ncol, x.nrow, x.b, x.x0, x.y0, x.w, x.hh};
        memcpy(out + 10 * t, v, sizeof(v));
    }
}

// per chunk: first, last, cols, bytes
extern "C" void plan_chunks(long long* out) {
    for (size_t k = 0; k < g_chunks.size(); ++k) {
        const hex6_chunk& c = g_chunks[k];
        const long long v[4] = {(long long)c.first, (long long)c.last, c.cols, (long long)c.bytes};
        memcpy(out + 4 * k, v, sizeof(v));
    }
}

extern "C" int plan_max_cols() { return hex6_max_cols(); }
