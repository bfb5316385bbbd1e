"""Learned warm start for the TNLM iteration.

A 2D U-Net over the 10 phases of a slice (phases as channels; include/
tnlm_unet.h) maps the per-phase FBP of a slice to the converged TNLM image.
Its output is only a start image: the plain TNLM iteration (Sec. 2.2) then
runs from it to the same stopping tolerance as from the usual start (the
FBP of all views, box step 1) and decides the result.

    python -m paper_1009_1351_gb300.warmstart --train 4000 --test 200 --epochs 4
    python -m paper_1009_1351_gb300.warmstart --time-net        (network timing only)

1. Data: the plain method makes its own training pairs on the GPU.  Each
   seeded slice is a phantom of the ellipse family (256 x 256 at 1.5 mm,
   anatomy shifted by up to 5 % of the side), its sinogram P f* (the
   library's projector) with Poisson noise in one of the three dose
   scenarios of the 256^2 workload, the per-phase FBP (input) and the TNLM
   result from the all-views FBP (target): run to the stopping tolerance
   (--target-tol) or for K = 50 outer iterations (slices of one scenario
   then run together with tnlm_reconstruct_batch).
2. Training: mean squared error, Adam, images scaled by 50 (unit order).
3. Evaluation on held-out seeds: iterations to the stopping tolerance
   (relative change of f below tol), device time and the error of the final
   image, from the usual start (cold) and from the network (warm); then the
   batched + warm-started form (network starts, one batched launch per
   chunk of slices, each slice stopping at the same rule) against the plain
   GPU form (one call per slice from the usual start).
"""
from __future__ import annotations

import argparse
import json
import math
import time
from typing import Dict, List

import numpy as np

from . import synth

SCALE = 50.0
SCENARIOS = ("mid_a", "mid_b", "mid_c")


def init_params(in_ch: int, out_ch: int, base: int, levels: int, seed: int) -> np.ndarray:
    """Flat initial parameters in the order of include/tnlm_unet.h: He-normal
    3x3 weights (std sqrt(2 / fan_in)), zero biases and a zero final 1x1
    layer, so that the untrained network returns its input."""
    rng = np.random.default_rng(seed)
    shapes = []
    cin = in_ch
    for l in range(levels):
        shapes += [(base << l, cin, 3), (base << l, base << l, 3)]
        cin = base << l
    for l in range(levels - 2, -1, -1):
        shapes += [(base << l, (base << (l + 1)) + (base << l), 3), (base << l, base << l, 3)]
    parts = []
    for co, ci, k in shapes:
        parts.append(rng.standard_normal(co * ci * k * k) * math.sqrt(2.0 / (ci * k * k)))
        parts.append(np.zeros(co))
    parts += [np.zeros(out_ch * base), np.zeros(out_ch)]
    return np.concatenate(parts).astype(np.float32)


def phantom_gpu(torch, c: synth.Case, offset, dev, ss: int = 4):
    """Area fractions of the phase ellipses on an ss x ss subgrid -> [N][L][L]."""
    g = c.geom
    L, s = g.nx, g.pixel_mm
    xs = (torch.arange(L * ss, device=dev, dtype=torch.float32) + 0.5) / ss - 0.5 - (L - 1) / 2.0
    X = (xs * s)[None, :].expand(L * ss, L * ss)
    Y = (xs * s)[:, None].expand(L * ss, L * ss)
    out = torch.zeros((g.n_phases, L, L), device=dev)
    for k in range(g.n_phases):
        img = torch.zeros((L * ss, L * ss), device=dev)
        for (cx, cy, ax, ay, mu, under) in synth.phantom_ellipses(L, s, k, g.n_phases,
                                                                   c.with_spine_diaphragm, offset):
            m = ((X - cx) / ax) ** 2 + ((Y - cy) / ay) ** 2 <= 1.0
            img = torch.where(m, torch.full_like(img, mu), img)
        out[k] = img.reshape(L, ss, L, ss).mean(dim=(1, 3))
    return out


class PairMaker:
    """Makes (per-phase FBP, all-views FBP, TNLM target, truth) on the GPU."""

    def __init__(self, torch, tn, slots: int = 16, k_outer: int = 50, tol: float = 0.0,
                 scenarios=SCENARIOS):
        self.torch, self.tn, self.k, self.tol = torch, tn, k_outer, tol
        self.dev = torch.device("cuda")
        self.scenarios = tuple(scenarios)
        self.cases = {s: synth.case(s) for s in self.scenarios}
        self.geos = {s: [tn.tnlm_create_geometry(self.cases[s].geom) for _ in range(slots)]
                     for s in self.scenarios}
        self.slots = slots

    def make(self, seeds: List[int], keep_all: bool = True) -> Dict[str, "object"]:
        torch, tn = self.torch, self.tn
        out = {"inp": [], "init": [], "target": [], "truth": [], "scenario": [], "seed": []}
        by_sc: Dict[str, List[int]] = {}
        for sd in seeds:
            by_sc.setdefault(self.scenarios[sd % len(self.scenarios)], []).append(sd)
        for sc, lst in by_sc.items():
            c = self.cases[sc]
            p = synth.Params(**{**c.params.__dict__, "k_outer": self.k})
            for j0 in range(0, len(lst), self.slots):
                chunk = lst[j0:j0 + self.slots]
                ys, ws, fs = [], [], []
                for j, sd in enumerate(chunk):
                    rng = np.random.default_rng(sd)
                    off = (float(rng.uniform(-0.05, 0.05) * c.geom.nx), float(rng.uniform(-0.05, 0.05) * c.geom.nx))
                    truth = phantom_gpu(torch, c, off, self.dev)
                    geo = self.geos[sc][j]
                    pbar = torch.empty(geo.sino_shape, device=self.dev)
                    tn.tnlm_project(geo, truth, pbar)
                    gen = torch.Generator(device=self.dev).manual_seed(sd)
                    lam = c.i0 * torch.exp(-pbar)
                    counts = torch.poisson(lam, generator=gen)
                    y = torch.log(c.i0 / torch.clamp(counts, min=1.0))
                    inp = torch.empty_like(truth)
                    tn.tnlm_fbp_phases(geo, y, inp)
                    f = torch.empty_like(truth)
                    tn.tnlm_fbp(geo, y, f)
                    out["inp"].append(inp)
                    if keep_all:
                        out["init"].append(f.clone())
                        out["truth"].append(truth)
                    out["scenario"].append(sc)
                    out["seed"].append(sd)
                    ys.append(y); ws.append(lam); fs.append(f)
                if self.tol > 0.0:
                    # targets converged to the stopping tolerance, one slice at a time
                    import types
                    pt = types.SimpleNamespace(**p.__dict__, tol=self.tol, tol_check_every=1)
                    for j in range(len(chunk)):
                        rep = tn.tnlm_reconstruct(self.geos[sc][j], pt, ys[j], ws[j], fs[j])
                        out.setdefault("target_iters", []).append(rep["iterations"])
                else:
                    tn.tnlm_reconstruct_batch(self.geos[sc][:len(chunk)], p, ys, ws, fs)
                out["target"].extend(fs)
        return out


def evaluate(torch, tn, net, maker: PairMaker, data, tol: float, kmax: int):
    """Cold vs warm start to the same tolerance on every held-out slice."""
    rows = []
    dev = maker.dev
    for i in range(len(data["seed"])):
        sc = data["scenario"][i]
        c = maker.cases[sc]
        geo = maker.geos[sc][0]
        truth = data["truth"][i]
        # the sinogram is rebuilt exactly as when the pair was made
        sd = data["seed"][i]
        pbar = torch.empty(geo.sino_shape, device=dev)
        tn.tnlm_project(geo, truth, pbar)
        gen = torch.Generator(device=dev).manual_seed(sd)
        lam = c.i0 * torch.exp(-pbar)
        y = torch.log(c.i0 / torch.clamp(torch.poisson(lam, generator=gen), min=1.0))
        p = synth.Params(**{**c.params.__dict__, "k_outer": kmax})
        import types
        pt = types.SimpleNamespace(**p.__dict__, tol=tol, tol_check_every=1)
        data.setdefault("y", {})[i] = y
        data.setdefault("lam", {})[i] = lam
        res = {}
        for mode in ("cold", "warm"):
            if mode == "cold":
                f = data["init"][i].clone()
            else:
                x = (data["inp"][i] * SCALE)[None].contiguous()
                o = torch.empty_like(x)
                net.forward(x, o)
                f = torch.clamp(o[0] / SCALE, min=0.0).contiguous()
            data.setdefault("start", {}).setdefault(i, {})[mode] = f.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            rep = tn.tnlm_reconstruct(geo, pt, y, lam, f)
            e1.record()
            e1.synchronize()
            res[mode] = (f, rep["iterations"], e0.elapsed_time(e1))
            data.setdefault("result", {}).setdefault(i, {})[mode] = (f, rep["iterations"])
        data.setdefault("cold_result", {})[i] = res["cold"][0]
        fc, fw = res["cold"][0].double(), res["warm"][0].double()
        t = truth.double()
        rows.append({"scenario": sc, "seed": sd,
                     "iters_cold": res["cold"][1], "iters_warm": res["warm"][1],
                     "ms_cold": res["cold"][2], "ms_warm": res["warm"][2],
                     "err_truth_cold": float((fc - t).norm() / t.norm()),
                     "err_truth_warm": float((fw - t).norm() / t.norm()),
                     "warm_vs_cold": float((fw - fc).norm() / fc.norm())})
    return rows


def warm_start(torch, net, inp, batch: int = 8):
    """Network start images for a list of per-phase FBP stacks."""
    out = []
    for b in range(0, len(inp), batch):
        x = torch.stack(inp[b:b + batch]) * SCALE
        o = torch.empty_like(x)
        net.forward(x, o)
        out.extend(torch.clamp(o / SCALE, min=0.0).unbind(0))
    return [t.contiguous() for t in out]


def evaluate_batched(torch, tn, net, maker: PairMaker, data, tol: float, kmax: int, chunk: int = 64):
    """The batched + warm-started form against the plain GPU form on the
    held-out slices (after evaluate(), which keeps their sinograms and cold
    results): chunks of slices of all scenarios, network start images, then
    ONE tnlm_reconstruct_batch launch per chunk in which every slice stops
    at the same rule as a single cold call (tol, checked every iteration).
    The plain form's time is the sum of the single cold calls' device
    times; the batched cold form (all-views FBP starts) separates the two
    gains."""
    import types
    n = len(data["seed"])
    pool: Dict[str, List[object]] = {s: [] for s in maker.scenarios}
    tot = {"batched_cold_ms": 0.0, "batched_warm_ms": 0.0}
    iters = {"batched_cold": [], "batched_warm": []}
    err_truth, vs_cold = [], []
    for c0 in range(0, n, chunk):
        idx = list(range(c0, min(n, c0 + chunk)))
        used = {s: 0 for s in maker.scenarios}
        geos, ps = [], []
        for i in idx:
            sc = data["scenario"][i]
            if used[sc] == len(pool[sc]):
                pool[sc].append(tn.tnlm_create_geometry(maker.cases[sc].geom))
            geos.append(pool[sc][used[sc]])
            used[sc] += 1
            p = synth.Params(**{**maker.cases[sc].params.__dict__, "k_outer": kmax})
            ps.append(types.SimpleNamespace(**p.__dict__, tol=tol, tol_check_every=1))
        ys = [data["y"][i] for i in idx]
        lams = [data["lam"][i] for i in idx]
        for mode in ("batched_cold", "batched_warm"):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if mode == "batched_cold":
                fs = [data["init"][i].clone() for i in idx]
            torch.cuda.synchronize()
            e0.record()
            if mode == "batched_warm":
                fs = warm_start(torch, net, [data["inp"][i] for i in idx])
            reps = tn.tnlm_reconstruct_batch(geos, ps, ys, lams, fs, autotune=False)
            e1.record()
            e1.synchronize()
            tot[mode + "_ms"] += e0.elapsed_time(e1)
            iters[mode] += [r["iterations"] for r in reps]
        for i, f in zip(idx, fs):
            t = data["truth"][i].double()
            fc = data["cold_result"][i].double()
            err_truth.append(float((f.double() - t).norm() / t.norm()))
            vs_cold.append(float((f.double() - fc).norm() / fc.norm()))
    return {"slices": n, "chunk": chunk, "loop_graph": tn.tnlm_batch_last_was_loop(),
            "batched_cold_ms": tot["batched_cold_ms"], "batched_warm_ms": tot["batched_warm_ms"],
            "iters_batched_cold": float(np.mean(iters["batched_cold"])),
            "iters_batched_warm": float(np.mean(iters["batched_warm"])),
            "err_truth_batched_warm": float(np.mean(err_truth)),
            "batched_warm_vs_single_cold": float(np.mean(vs_cold))}


def time_net(torch, tn, base: int, levels: int, batch: int, reps: int = 10) -> Dict[str, float]:
    """Device time of the network's forward pass and of one training step
    (gradients + Adam) on random 10-phase 256 x 256 inputs."""
    net = tn.UNet(10, 10, base, levels)
    net.set_params(init_params(10, 10, base, levels, 1))
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.rand((batch, 10, 256, 256), device="cuda", generator=g)
    t = torch.rand_like(x)
    o = torch.empty_like(x)
    for _ in range(2):
        net.forward(x, o)
        net.grads(x, t)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    for _ in range(reps):
        net.forward(x, o)
    e[1].record()
    for _ in range(reps):
        net.grads(x, t)
        net.adam_step(1e-3)
    e[2].record()
    torch.cuda.synchronize()
    return {"batch": batch, "forward_ms": e[0].elapsed_time(e[1]) / reps,
            "train_step_ms": e[1].elapsed_time(e[2]) / reps}


def parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--time-net", action="store_true", help="only time the network (random data)")
    ap.add_argument("--train", type=int, default=4000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--tol", type=float, default=1e-3, help="stopping tolerance of the evaluation")
    ap.add_argument("--target-tol", type=float, default=0.0,
                    help="> 0: targets are TNLM runs to this tolerance (else K = 50)")
    ap.add_argument("--kmax", type=int, default=300)
    ap.add_argument("--base", type=int, default=32)
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--seed", type=int, default=7000)
    ap.add_argument("--chunk", type=int, default=64, help="slices per batched launch in the evaluation")
    ap.add_argument("--out", default=None)
    return ap


def run(args, clocks=None):
    """Make the data, train, evaluate cold vs warm and batched + warm vs
    plain; returns (summary dict, held-out data, pair maker, network).
    clocks: optional object with start() / stop() -> dict, sampled around
    the evaluation."""
    import torch
    import paper_1009_1351_gb300 as tn
    maker = PairMaker(torch, tn, k_outer=args.kmax if args.target_tol > 0 else 50, tol=args.target_tol)
    t0 = time.perf_counter()
    train = maker.make(list(range(args.seed, args.seed + args.train)), keep_all=False)
    test = maker.make(list(range(args.seed + 100000, args.seed + 100000 + args.test)))
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    X = torch.stack(train["inp"]) * SCALE
    Y = torch.stack(train["target"]) * SCALE
    Xt = torch.stack(test["inp"]) * SCALE
    Yt = torch.stack(test["target"]) * SCALE

    net = tn.UNet(10, 10, args.base, args.levels)
    net.set_params(init_params(10, 10, args.base, args.levels, args.seed))
    rng = np.random.default_rng(args.seed)
    steps_per_epoch = args.train // args.batch
    total = steps_per_epoch * args.epochs
    hist = []
    t1 = time.perf_counter()
    step = 0
    for ep in range(args.epochs):
        order = rng.permutation(args.train)
        ls = []
        for s in range(steps_per_epoch):
            idx = torch.as_tensor(order[s * args.batch:(s + 1) * args.batch], device=X.device)
            lr = args.lr * 0.5 * (1 + math.cos(math.pi * step / total))
            ls.append(net.grads(X[idx].contiguous(), Y[idx].contiguous()))
            net.adam_step(lr)
            step += 1
        # held-out loss
        tl = []
        for s in range(0, args.test, args.batch):
            xb = Xt[s:s + args.batch].contiguous()
            ob = torch.empty_like(xb)
            net.forward(xb, ob)
            tl.append(float(((ob - Yt[s:s + args.batch]) ** 2).mean()))
        hist.append({"epoch": ep, "train_loss": float(np.mean(ls)), "test_loss": float(np.mean(tl))})
        print(json.dumps(hist[-1]), flush=True)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    # loss of the network's input itself (identity map) for reference
    base_loss = float(((Xt - Yt) ** 2).mean())
    if clocks is not None:
        clocks.start()
    rows = evaluate(torch, tn, net, maker, test, args.tol, args.kmax)
    summ = {k: float(np.mean([r[k] for r in rows])) for k in
            ("iters_cold", "iters_warm", "ms_cold", "ms_warm", "err_truth_cold", "err_truth_warm",
             "warm_vs_cold")}
    bat = evaluate_batched(torch, tn, net, maker, test, args.tol, args.kmax, args.chunk)
    bat["plain_ms"] = float(np.sum([r["ms_cold"] for r in rows]))
    bat["speedup_batched_warm_vs_plain"] = bat["plain_ms"] / bat["batched_warm_ms"]
    bat["speedup_batched_cold_vs_plain"] = bat["plain_ms"] / bat["batched_cold_ms"]
    clk = clocks.stop() if clocks is not None else None
    ti = train.get("target_iters", [])
    out = {"train": args.train, "test": args.test, "epochs": args.epochs, "batch": args.batch,
           "target": (f"TNLM to tol {args.target_tol} (mean {np.mean(ti):.1f} iterations)" if ti
                      else "TNLM after K = 50"),
           "net": {"base": args.base, "levels": args.levels, "params": net.param_count},
           "seconds": {"data": round(t_data, 1), "train": round(t_train, 1)},
           "loss": hist, "identity_test_loss": base_loss, "tol": args.tol,
           "mean": summ, "batched": bat, "clocks": clk, "per_slice": rows}
    return out, test, maker, net


def main() -> None:
    import torch
    import paper_1009_1351_gb300 as tn

    args = parser().parse_args()
    torch.cuda.set_device(0)
    if args.time_net:
        print(json.dumps(time_net(torch, tn, args.base, args.levels, args.batch)))
        return
    out, _, _, _ = run(args)
    print(json.dumps({k: v for k, v in out.items() if k != "per_slice"}))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(out, fh)


if __name__ == "__main__":
    main()
