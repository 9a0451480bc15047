// Host-side planning of the six-directional filter's lattice windows
// (hex6.cu holds the kernels).  Pure host code: the tests build it on the CPU.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/bsf.h"
#include "bsf_internal.h"

// geometry of the window of one tile: every lattice point that the taps of
// its pixels read (host side; ex, ey = the tile's largest footprint half-extents)
void hex6_window(int tx0, int ty0, int tw, int th_, int H, int W, double ex, double ey, double h, hex6_tile* t) {
    const double SQ3 = 1.7320508075688772935;
    const int x0 = tx0, x1 = std::min(W, tx0 + tw) - 1;
    const int y0 = ty0, y1 = std::min(H, ty0 + th_) - 1;
    // taps: n + tau - x_q, in n + [-ex, ex] x [-ey, ey] - (h/2, 3 sqrt3 h / 2)
    const double xl = x0 - ex - 0.5 * h, xh = x1 + ex - 0.5 * h;
    const double yl = y0 - ey - 1.5 * SQ3 * h, yh = y1 + ey - 1.5 * SQ3 * h;
    const double tl = 2.0 * yl / (h * SQ3), th = 2.0 * yh / (h * SQ3);
    const int j0 = (int)std::floor(tl) - 4, j1 = (int)std::floor(th) + 5;
    t->j0w = j0;
    t->nrow = j1 - j0 + 1;
    // row j is read by taps with t in [j - 3, j + 3); their cells' columns i0 run
    // over floor(x/h - t/2) and the slots reach i0 - 2 .. i0 + 3
    long long ileft = (1LL << 40), ncol = 0;
    for (int r = 0; r < t->nrow; ++r) {
        const int j = j0 + r;
        const long long imin = (long long)std::floor(xl / h - 0.5 * (j + 3)) - 4;
        ileft = std::min(ileft, imin + 2LL * r);
    }
    for (int r = 0; r < t->nrow; ++r) {
        const int j = j0 + r;
        const long long imax = (long long)std::floor(xh / h - 0.5 * (j - 3)) + 5;
        ncol = std::max(ncol, imax - (ileft - 2LL * r) + 1);
    }
    t->i_left = (int)ileft;
    t->ncol = (int)ncol;
    t->x0 = tx0;
    t->y0 = ty0;
    t->w = tw;
    t->hh = th_;
}

// widest window: HEX6_PRE_CPT columns per thread, and four 128-bit state rows plus the
// warp totals in 227 KB of shared memory
int hex6_max_cols() {
    return std::min(HEX6_PRE_THREADS * HEX6_PRE_CPT,
                    (232448 - 32 * 16) / (4 * 16) * HEX6_PRE_PAD / (HEX6_PRE_PAD + 1) - 8);
}

// tile records and chunks from the largest footprint half-extents of every
// 16 x 16 block (ext: B * fy * fx pairs (ex, ey) as FP32 bits, fy x fx blocks)
int hex6_plan(int64_t B, int64_t C, int64_t H, int64_t W, double h, const unsigned* ext, size_t budget,
                     std::vector<hex6_tile>& tl, std::vector<hex6_chunk>& chunks) {
    const int fine = 16, coarse = 64, ratio = coarse / fine;
    const float split_below = 16.f;  // px: largest half-extent for which a 64-tile is cut into 16-tiles
    const float group_from = 32.f;   // px: smallest half-extent of a 64-tile that joins a group
    const int fx = (int)((W + fine - 1) / fine), fy = (int)((H + fine - 1) / fine);
    const int64_t nfine = (int64_t)fx * fy;
    auto ext_of = [&](int64_t b, int bx, int by, float* ex, float* ey) {
        const size_t t = (size_t)(b * nfine + (int64_t)by * fx + bx) * 2;
        memcpy(ex, &ext[t], sizeof(float));
        memcpy(ey, &ext[t + 1], sizeof(float));
    };
    // Tile records, one launch shape per class.  A window spans its tile plus
    // the footprint, sheared into a parallelogram (a row of the window is as
    // wide as the tile, twice the footprint, and sqrt(3) times the window's
    // height), so neighbouring 64-tiles with large footprints share one window:
    // groups of 4 x 2, 4 x 1 and 2 x 1 aligned 64-tiles (256 x 128, 256 x 64,
    // 128 x 64 pixels) are taken, largest first, where every tile of the group
    // has a footprint half-extent of at least group_from and at least half the
    // group's largest (a group's window is no larger, for the kernels of any
    // of its tiles, than a few times the tile's own: the conditioning of the
    // stencil grows with the window) and the window fits the
    // pre-integration's width; then single 64-tiles; tiles with small
    // footprints are cut into 16-tiles.
    for (size_t k = 0; k < (size_t)(B * nfine * 2); ++k) {  // finite, non-negative, below 1e5 px
        float v;
        memcpy(&v, &ext[k], sizeof(float));
        if (!(v >= 0.f && v < 1e5f)) return BSF_EINVAL;
    }
    static const int group[4][2] = {{4, 2}, {4, 1}, {2, 1}, {1, 1}};
    std::vector<hex6_tile> cls[5];
    const int cx = (int)((W + coarse - 1) / coarse), cy = (int)((H + coarse - 1) / coarse);
    std::vector<float> e64((size_t)cx * cy * 2);
    std::vector<unsigned char> taken((size_t)cx * cy);
    for (int64_t b = 0; b < B; ++b) {
        for (int ty = 0; ty < cy; ++ty)
            for (int tx = 0; tx < cx; ++tx) {
                float ex = 0.f, ey = 0.f;
                for (int by = ty * ratio; by < std::min(fy, (ty + 1) * ratio); ++by)
                    for (int bx = tx * ratio; bx < std::min(fx, (tx + 1) * ratio); ++bx) {
                        float a, e;
                        ext_of(b, bx, by, &a, &e);
                        ex = std::max(ex, a);
                        ey = std::max(ey, e);
                    }
                e64[((size_t)ty * cx + tx) * 2] = ex;
                e64[((size_t)ty * cx + tx) * 2 + 1] = ey;
            }
        std::fill(taken.begin(), taken.end(), 0);
        for (int g = 0; g < 4; ++g) {
            const int gw = group[g][0], gh = group[g][1];
            for (int ty = 0; ty + gh <= cy; ty += gh)
                for (int tx = 0; tx + gw <= cx; tx += gw) {
                    float ex = 0.f, ey = 0.f, lo = 1e30f, hi = 0.f;
                    bool free = true;
                    for (int yy = ty; yy < ty + gh; ++yy)
                        for (int xx = tx; xx < tx + gw; ++xx) {
                            const size_t k = (size_t)yy * cx + xx;
                            free = free && !taken[k];
                            ex = std::max(ex, e64[2 * k]);
                            ey = std::max(ey, e64[2 * k + 1]);
                            lo = std::min(lo, std::max(e64[2 * k], e64[2 * k + 1]));
                            hi = std::max(hi, std::max(e64[2 * k], e64[2 * k + 1]));
                        }
                    if (!free || lo < (g < 3 ? group_from : split_below) || (g < 3 && lo < 0.5f * hi)) continue;
                    hex6_tile t;
                    hex6_window(tx * coarse, ty * coarse, gw * coarse, gh * coarse, (int)H, (int)W, ex, ey, h, &t);
                    if (g < 3 && t.ncol > hex6_max_cols()) continue;  // too wide: smaller groups
                    t.b = (int)b;
                    cls[g].push_back(t);
                    for (int yy = ty; yy < ty + gh; ++yy)
                        for (int xx = tx; xx < tx + gw; ++xx) taken[(size_t)yy * cx + xx] = 1;
                }
        }
        for (int ty = 0; ty < cy; ++ty)
            for (int tx = 0; tx < cx; ++tx) {
                if (taken[(size_t)ty * cx + tx]) continue;
                for (int by = ty * ratio; by < std::min(fy, (ty + 1) * ratio); ++by)
                    for (int bx = tx * ratio; bx < std::min(fx, (tx + 1) * ratio); ++bx) {
                        float a, e;
                        ext_of(b, bx, by, &a, &e);
                        hex6_tile t;
                        hex6_window(bx * fine, by * fine, fine, fine, (int)H, (int)W, a, e, h, &t);
                        t.b = (int)b;
                        cls[4].push_back(t);
                    }
            }
    }
    tl.clear();
    for (auto& v : cls) tl.insert(tl.end(), v.begin(), v.end());
    // chunks of one tile shape, at most `budget` bytes of windows and 65535
    // tiles (a grid dimension)
    chunks.clear();
    for (size_t t = 0; t < tl.size(); ++t) {
        if (tl[t].ncol > hex6_max_cols()) return BSF_EINVAL;  // footprint too wide for one window
        const size_t bytes = (size_t)C * tl[t].ncol * tl[t].nrow * 16;
        if (bytes > budget) return BSF_EINVAL;
        if (chunks.empty() || tl[t].w != tl[chunks.back().first].w || tl[t].hh != tl[chunks.back().first].hh ||
            chunks.back().bytes + bytes > budget || t - chunks.back().first >= 65535)
            chunks.push_back({t, t, 0, 0});
        hex6_chunk& ch = chunks.back();
        tl[t].off = (long long)(ch.bytes / 16);
        ch.bytes += bytes;
        ch.last = t + 1;
        ch.cols = std::max(ch.cols, tl[t].ncol);
    }
    return BSF_OK;
}
