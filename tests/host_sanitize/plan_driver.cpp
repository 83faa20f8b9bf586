// Host-only driver for the set-up code (usr_setup.cpp): plans over boxes, grids, presets, cutoffs, forms,
// stencils, the multilevel option and the virial, then over extreme and out-of-range values, built with
// AddressSanitizer and UndefinedBehaviorSanitizer (float-to-int overflow included) by
// tests/test_host_sanitizers.py (no GPU).
#include <cstdio>
#include "usr_internal.h"
int main()
{
    int ok = 0, rejected = 0;
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
                                if (usr::make_plan(&p, &plan) == USR_OK) ++ok; else ++rejected;
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
    printf("plans ok %d rejected %d\n", ok, rejected);
    return 0;
}
// device-memory estimate lives in the CUDA translation unit; not exercised here
double usr::plan_device_bytes(const usr::Plan&) { return 0.0; }
