"""Run one named workload through the library, for profilers (ncu) and timing.

    python -m paper_1009_1351_gb300.profile_run --case mid_a --k 1 [--m1 3 --m2 5] [--ops 10] [--mixed]
    python -m paper_1009_1351_gb300.profile_run --case large_a,large_b,large_c,large_d --k 2 --fbp

Builds the seeded inputs of each named workload, runs tnlm_reconstruct with
K outer iterations from the constant start image (or, with --fbp, from the
FBP of all views, as the benchmark does), then --ops projections and --ops
backprojections of a random image, and prints the CUDA-event time of each
part.  Everything runs in the library's kernels.
"""
from __future__ import annotations

import argparse

import torch

import paper_1009_1351_gb300 as tn
from paper_1009_1351_gb300 import synth


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="mid_a")
    ap.add_argument("--k", type=int, default=1)
    ap.add_argument("--m1", type=int, default=None)
    ap.add_argument("--m2", type=int, default=None)
    ap.add_argument("--ops", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--mixed", action="store_true", help="tensor-core patch distances")
    ap.add_argument("--fbp", action="store_true", help="start from the FBP of all views")
    args = ap.parse_args()
    for name in args.case.split(","):
        run_case(name, args)


def run_case(name: str, args) -> None:
    c = synth.case(name)
    d = synth.make_inputs(c)
    over = {"k_outer": args.k}
    if args.m1 is not None:
        over["m1"] = args.m1
    if args.m2 is not None:
        over["m2"] = args.m2
    if args.mixed:
        over["precision"] = tn.PREC_MIXED
    p = synth.Params(**{**c.params.__dict__, **over})
    geo = tn.tnlm_create_geometry(c.geom)
    dv = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    y, w = dv(d["y"]), dv(d["w"])
    f0 = torch.full(geo.img_shape, 0.01, device="cuda")
    if args.fbp:
        tn.tnlm_fbp(geo, y, f0)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for r in range(args.repeat):
        f = f0.clone()
        e0, e1 = ev(), ev()
        e0.record()
        tn.tnlm_reconstruct(geo, p, y, w, f, report=False)
        e1.record()
        torch.cuda.synchronize()
        print(f"{name} reconstruct K={args.k}: {e0.elapsed_time(e1):.3f} ms")
    if args.ops:
        img = dv(synth.random_images(geo.img_shape, 1))
        sino = torch.zeros(geo.sino_shape, device="cuda")
        for name, fn in (("project", lambda: tn.tnlm_project(geo, img, sino)),
                         ("backproject", lambda: tn.tnlm_backproject(geo, sino, img))):
            e0, e1 = ev(), ev()
            e0.record()
            for _ in range(args.ops):
                fn()
            e1.record()
            torch.cuda.synchronize()
            print(f"{name}: {e0.elapsed_time(e1) / args.ops:.3f} ms per call")


if __name__ == "__main__":
    main()
