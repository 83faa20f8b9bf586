// Host-only driver for the set-up code (usr_setup.cpp): plans over boxes, grids, presets, cutoffs, forms,
// stencils, the multilevel option and the virial, then over extreme and out-of-range values, built with
// AddressSanitizer and UndefinedBehaviorSanitizer (float-to-int overflow included) by
// tests/test_host_sanitizers.py (no GPU).  For every plan of the first sweep it also checks that the
// spreading stencil of every wrapped coordinate fits the shared-memory tile of its block of cells.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include "usr_internal.h"

namespace {

float bits_to_float(uint32_t u)
{
    float f;
    std::memcpy(&f, &u, sizeof f);
    return f;
}

uint32_t float_to_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, sizeof u);
    return u;
}

/* The cell of a wrapped coordinate xw in [0, L] (the binning kernel's single-precision predicate). */
int cell_of(float xw, float cs, int nc)
{
    const float u = xw * cs;
    const int c = u >= 0.0f ? (int)u : 0;
    return c > nc - 1 ? nc - 1 : c;
}

/*
 * The spreading kernel adds an atom's P x P x P stencil into the shared-memory tile of the block of cells
 * that holds the atom; its base offset along an axis is floor(x gs) - P/2 + 1 - org.  For every block along
 * every axis, find the exact float interval of wrapped coordinates in [0, L] whose cell lies in the block
 * (the cell is monotone in x, so a binary search over the bit patterns of non-negative floats finds its
 * ends) and check that the stencil of both ends, hence of every coordinate between, lies inside the tile.
 * Returns the number of violations.
 */
int check_spread_tiles(const usr::Plan& P)
{
    int bad = 0;
    const int H = P.P / 2;
    // the tile's own layout: x extent a multiple of 4 (float4 zeroing), a plane stride of at least one plane
    // and a multiple of 4, at most kTileMaxSmem bytes, and at most 64 (z, y) rows of cells per block (the
    // spreading kernel's row table)
    const usr::TileGeom& tg = P.tile;
    if (tg.T[0] % 4 != 0 || tg.ps < tg.T[0] * tg.T[1] || tg.ps % 4 != 0 ||
        4.0 * tg.ps * tg.T[2] > usr::kTileMaxSmem || tg.kb[1] * tg.kb[2] > 64) {
        if (bad < 5) std::printf("tile layout violation: T %d %d %d ps %d kb %d %d %d\n", tg.T[0], tg.T[1], tg.T[2],
                                 tg.ps, tg.kb[0], tg.kb[1], tg.kb[2]);
        ++bad;
    }
    for (int a = 0; a < 3; ++a) {
        const float L = (float)P.L[a], cs = (float)((double)P.cells[a] / P.L[a]);
        const float gs = (float)((double)P.n[a] / P.L[a]);
        const int nc = P.cells[a], kb = P.tile.kb[a], T = P.tile.T[a];
        const uint32_t top = float_to_bits(L);
        for (int b = 0; b < P.tile.nbk[a]; ++b) {
            const int c0 = b * kb, c1 = std::min(nc, c0 + kb) - 1;
            uint32_t lo = 0, hi = top;                     // smallest x with cell(x) >= c0
            while (lo < hi) {
                const uint32_t mid = lo + (hi - lo) / 2;
                if (cell_of(bits_to_float(mid), cs, nc) >= c0) hi = mid; else lo = mid + 1;
            }
            const uint32_t xlo = lo;
            lo = 0, hi = top;                              // largest x with cell(x) <= c1
            while (lo < hi) {
                const uint32_t mid = lo + (hi - lo + 1) / 2;
                if (cell_of(bits_to_float(mid), cs, nc) <= c1) lo = mid; else hi = mid - 1;
            }
            const uint32_t xhi = lo;
            if (cell_of(bits_to_float(xlo), cs, nc) < c0 || cell_of(bits_to_float(xhi), cs, nc) > c1 || xlo > xhi)
                continue;                                  // no coordinate falls in this block
            const int org = P.tile_org[a][b];
            const int base_lo = (int)std::floor(bits_to_float(xlo) * gs) - H + 1 - org;
            const int base_hi = (int)std::floor(bits_to_float(xhi) * gs) - H + 1 - org;
            if (base_lo < 0 || base_hi + P.P > T) {
                if (bad < 5)
                    std::printf("tile violation: axis %d block %d base %d..%d + %d vs T %d\n", a, b, base_lo,
                                base_hi, P.P, T);
                ++bad;
            }
        }
    }
    return bad;
}

}  // namespace

int main()
{
    int ok = 0, rejected = 0, tile_bad = 0;
    const double boxes[][3] = {{31.0, 31.0, 31.0}, {80.0, 80.0, 100.0}, {58.5, 58.5, 58.5}, {220.0, 220.0, 220.0},
                               {100.0, 100.0, 100.0}, {27.0, 27.0, 27.0}};
    const int grids[][3] = {{32, 32, 32}, {64, 64, 80}, {48, 48, 48}, {176, 176, 176}, {96, 96, 96}, {24, 24, 24}};
    for (int b = 0; b < 6; ++b)
        for (int preset = 0; preset < 6; ++preset)
            for (double rc : {8.0, 9.0, 10.0, 13.0})
                for (int conv : {0, 1, 2})
                    for (int P : {0, 8, 10, 12, 16})
                        for (int ml : {0, 1})
                            for (int vir : {0, 1}) {
                                usr_params p = {};
                                if (usr_series_preset(preset, &p.series) != USR_OK) continue;
                                for (int a = 0; a < 3; ++a) { p.box[a] = boxes[b][a]; p.grid[a] = grids[b][a]; }
                                p.r_c = rc; p.conv = (usr_conv)conv; p.spread_points = P; p.spread_sigma_over_h = P ? 0.83 : 0.0;
                                p.multilevel = ml; p.virial = vir; p.max_atoms = 1000;
                                usr::Plan plan;
                                if (usr::make_plan(&p, &plan) == USR_OK) {
                                    ++ok;
                                    tile_bad += check_spread_tiles(plan);
                                } else {
                                    ++rejected;
                                }
                            }
    // extreme and out-of-range values: each must be planned or refused with a status, with no undefined
    // behaviour (float-to-int conversions included) and no unbounded host allocation
    const double ext_box[][3] = {{1e300, 1e300, 1e300}, {1e-300, 31.0, 31.0}, {4000.0, 4000.0, 4000.0},
                                 {31.0, 31.0, 31.0}};
    const int ext_grid[][3] = {{32, 32, 32}, {4096, 16, 16}, {4097, 32, 32}, {2048, 2048, 1024},
                               {2147483647, 32, 32}, {-5, 32, 32}};
    const double ext_rc[] = {9.0, 1e-300, 1e300, 5e-324};
    const double ext_b[] = {2.0, 1.012, 1.01, 1.0 + 1e-15, 1e300};
    for (const auto& bx : ext_box)
        for (const auto& gr : ext_grid)
            for (double rc : ext_rc)
                for (double bb : ext_b)
                    for (int ma : {0, 1 << 28, (1 << 28) + 1, 2147483647}) {
                        usr_params p = {};
                        usr_series_preset(1, &p.series);
                        p.series.b = bb;
                        p.series.n_terms = bb == 2.0 ? 0 : 3;
                        for (int a = 0; a < 3; ++a) { p.box[a] = bx[a]; p.grid[a] = gr[a]; }
                        p.r_c = rc;
                        p.max_atoms = ma;
                        usr::Plan plan;
                        if (usr::make_plan(&p, &plan) == USR_OK) ++ok; else ++rejected;
                    }
    printf("plans ok %d rejected %d tile violations %d\n", ok, rejected, tile_bad);
    return tile_bad == 0 ? 0 : 1;
}
// device-memory estimate lives in the CUDA translation unit; not exercised here
double usr::plan_device_bytes(const usr::Plan&) { return 0.0; }
