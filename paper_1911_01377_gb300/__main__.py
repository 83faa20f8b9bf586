"""Run u-series evaluations of a named synthetic workload on the current GPU.

    python -m paper_1911_01377_gb300 --workload membrane_slab --rc 10 --evals 3

Prints the energy breakdown and the per-stage times (CUDA events), averaged over
the evaluations after the first.  Useful for profiling a single evaluation under a tool such as ncu.
"""
from __future__ import annotations

import argparse

from . import build as B
from . import usr
from . import workloads as W


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="membrane_slab",
                    choices=["water_3k", "membrane_slab", "water_20k", "water_1m"])
    ap.add_argument("--rc", type=float, default=0.0, help="cutoff (default: the workload's first)")
    ap.add_argument("--series", default="C1_B2", choices=sorted(usr.PRESETS))
    ap.add_argument("--evals", type=int, default=1)
    ap.add_argument("--conv", type=int, default=0, choices=[0, 1, 2], help="0 FP32, 1 TF32x3, 2 BF16x3")
    ap.add_argument("--spread-points", type=int, default=0)
    ap.add_argument("--spread-sigma", type=float, default=0.0, help="spreading width / grid spacing")
    ap.add_argument("--virial", type=int, default=0, choices=[0, 1])
    ap.add_argument("--multilevel", type=int, default=0, choices=[0, 1], help="wide terms on the coarse grid")
    args = ap.parse_args(argv)

    import torch

    B.build()
    w = W.get(args.workload)
    r_c = args.rc or w.r_c[0]
    ctx = usr.USeries(w.box, w.grid, r_c, args.series, max_atoms=w.n, conv=args.conv,
                      spread_points=args.spread_points, spread_sigma_over_h=args.spread_sigma, virial=args.virial,
                      multilevel=args.multilevel)
    usr.usr_set_profiling(ctx.ctx, True)
    x = torch.from_numpy(w.xyzq).cuda()
    out = torch.empty((w.n, 4), dtype=torch.float32, device="cuda")
    en = torch.empty(4, dtype=torch.float64, device="cuda")
    acc = [0.0] * usr.USR_NSTAGES
    for k in range(args.evals):
        ctx.eval(x, out, en)
        if k > 0 or args.evals == 1:               # the first of several evaluations is a warm-up
            acc = [a + v for a, v in zip(acc, usr.usr_stage_times(ctx.ctx))]
    torch.cuda.synchronize()
    st = usr.usr_last_device_status(ctx.ctx)
    if st != 0:
        raise usr.UsrError(st, "usr_eval")
    e = en.cpu().tolist()
    info = ctx.info
    print(f"{w.name}: n={w.n} r_c={r_c:g} grid={w.grid} terms={info.n_terms} (coarse {info.n_terms_coarse}) "
          f"cells={tuple(info.cells)}")
    print(f"E={e[0]:.10f} E_near={e[1]:.10f} E_far={e[2]:.10f} E_self={e[3]:.10f}")
    if args.virial:
        print("virial:", ctx.virial().cpu().numpy().round(6).tolist())
    ms = [a / max(1, args.evals - 1) if args.evals > 1 else a for a in acc]
    print("stage ms (mean): " + " ".join(f"{k}={v:.4f}" for k, v in zip(usr.STAGES, ms)) + f" total={sum(ms):.4f}")
    ctx.close()


if __name__ == "__main__":
    main()
