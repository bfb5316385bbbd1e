"""The learned warm start at full scale, with the final images checked
against the FP64 oracle (test infrastructure: it runs the oracle).

    python tests/warmstart_report.py [--train 4000 --test 200 --epochs 6 --oracle-slices 4 \
        --out profiles/warmstart_256x256.json]

Runs the library's warm-start study (paper_1009_1351_gb300.warmstart.run:
pairs made by the plain method on the GPU, training by the library's own
kernels, held-out slices run cold and warm to the same stopping tolerance,
then the batched + warm form against the plain form), with nvidia-smi clocks
sampled during the evaluation.  Then, for --oracle-slices held-out slices
(the first of each dose scenario in turn), the FP64 oracle runs from the same cold
and warm start images for the same number of outer iterations as the GPU
took, and the relative L2 error of each GPU result against it is recorded.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)


def main():
    import torch

    import bench
    import oracle
    from paper_1009_1351_gb300 import synth, warmstart

    ap = warmstart.parser()
    ap.set_defaults(train=4000, test=200, epochs=6, target_tol=4e-3, tol=4e-3, kmax=300)
    ap.add_argument("--oracle-slices", type=int, default=4)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    oracle.build()
    out, test, maker, net = warmstart.run(args, clocks=bench.ClockSampler(0))
    t0 = time.perf_counter()
    rows = []
    # the first held-out slice of each dose scenario in turn
    order, seen = [], {}
    for i, sc in enumerate(test["scenario"]):
        seen.setdefault(sc, []).append(i)
    while len(order) < min(args.oracle_slices, len(test["seed"])):
        for sc in list(seen):
            if seen[sc] and len(order) < args.oracle_slices:
                order.append(seen[sc].pop(0))
    for i in order:
        c = maker.cases[test["scenario"][i]]
        G = oracle.Geom(c.geom)
        y = test["y"][i].double().cpu().numpy().astype(np.float32)
        w = test["lam"][i].double().cpu().numpy().astype(np.float32)
        row = {"scenario": test["scenario"][i], "seed": test["seed"][i]}
        for mode in ("cold", "warm"):
            f0 = test["start"][i][mode].cpu().numpy()
            got, k = test["result"][i][mode]
            p = synth.Params(**{**c.params.__dict__, "k_outer": k})
            ref, _, _ = oracle.reconstruct(G, y, w, f0, p)
            g = got.double().cpu().numpy()
            row[f"iters_{mode}"] = int(k)
            row[f"rel_l2_vs_fp64_oracle_{mode}"] = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
        rows.append(row)
    out["fp64_oracle"] = {"slices": rows, "threads": oracle.threads(0),
                          "seconds": round(time.perf_counter() - t0, 1),
                          "reading": "GPU FP32 result vs the FP64 oracle run from the same start image "
                                     "for the same number of outer iterations"}
    print(json.dumps({k: v for k, v in out.items() if k != "per_slice"}))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
