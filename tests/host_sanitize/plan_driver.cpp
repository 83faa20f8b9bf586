// Host-only driver for the set-up code (usr_setup.cpp): plans over boxes, grids, presets, cutoffs, forms,
// stencils, the multilevel option and the virial, built with AddressSanitizer and UndefinedBehaviorSanitizer
// by tests/test_host_sanitizers.py (no GPU).
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
    printf("plans ok %d rejected %d\n", ok, rejected);
    return 0;
}
// device-memory estimate lives in the CUDA translation unit; not exercised here
double usr::plan_device_bytes(const usr::Plan&) { return 0.0; }
