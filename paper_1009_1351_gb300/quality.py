"""Image-quality measures of the paper's evaluation (Sec. 3) and a dose study.

cnr(f, roi, bg)  Eq. 10: |mu_s - mu_b| / sigma_b, mean over the ROI against
                 the mean and standard deviation of its background region.
snr_db(f, truth) Eq. 11: 10 log10( ||f - mean(f)||^2 / ||f - f*||^2 ).

ROIs on the synthetic phantom (the paper's Fig. 4 ROIs are on the NCAT
phantom, which is not available): ROI1 is the tumour disc against the
surrounding lung (a small high-contrast structure on dark lung, as in the
paper), ROI2 the spine disc against the surrounding soft tissue.  Both are
eroded / kept away from edges by two pixels.

    python -m paper_1009_1351_gb300.quality --case mid_a [--k 50] [--sweep]

reconstructs the slice by FBP and by the TNLM iteration on the GPU and
prints the mean CNR of both ROIs and the mean SNR over the phases; --sweep
adds the TNLM results over mu_hat in {0.25, 0.5, 1, 2} and h scaled by
{0.5, 1, 2}.
"""
from __future__ import annotations

import argparse
import json
import math
from typing import Dict, Tuple

import numpy as np

from . import synth


def cnr(f: np.ndarray, roi: np.ndarray, bg: np.ndarray) -> float:
    """Eq. 10 on one image."""
    s = f[roi]
    b = f[bg]
    return float(abs(s.mean() - b.mean()) / b.std())


def snr_db(f: np.ndarray, truth: np.ndarray) -> float:
    """Eq. 11 on one image (f-bar is the mean of the image f)."""
    num = float(np.sum((f - f.mean()) ** 2))
    den = float(np.sum((f - truth) ** 2))
    return 10.0 * math.log10(num / den)


def _disc_mask(L, pixel, cx, cy, r):
    xs = (np.arange(L) - (L - 1) / 2.0) * pixel
    X, Y = np.meshgrid(xs, xs)
    return np.hypot(X - cx, Y - cy) <= r


def _ellipse_mask(L, pixel, cx, cy, ax, ay):
    xs = (np.arange(L) - (L - 1) / 2.0) * pixel
    X, Y = np.meshgrid(xs, xs)
    return ((X - cx) / ax) ** 2 + ((Y - cy) / ay) ** 2 <= 1.0


def rois(c: synth.Case, phase: int) -> Dict[str, Tuple[np.ndarray, np.ndarray]]:
    """(roi, background) masks of ROI1 (tumour / lung) and, with a spine, ROI2
    (spine / soft tissue) for one phase of a workload's phantom."""
    g = c.geom
    L, s = g.nx, g.pixel_mm
    ells = synth.phantom_ellipses(L, s, phase, g.n_phases, c.with_spine_diaphragm)
    tum = ells[-1]
    lung = [e for e in ells if e[4] == 0.004 and e[0] > 0][0]
    out = {}
    tumour = _disc_mask(L, s, tum[0], tum[1], tum[2] - 2 * s)
    near = _disc_mask(L, s, tum[0], tum[1], tum[2] + 6 * s) & ~_disc_mask(L, s, tum[0], tum[1], tum[2] + 2 * s)
    lung_in = _ellipse_mask(L, s, lung[0], lung[1], lung[2] - 2 * s, lung[3] - 2 * s)
    out["roi1"] = (tumour, near & lung_in)
    spines = [e for e in ells if e[4] == 0.04]
    if spines:
        sp = spines[0]
        body = ells[0]
        spine = _disc_mask(L, s, sp[0], sp[1], sp[2] - 2 * s)
        ring = _disc_mask(L, s, sp[0], sp[1], sp[2] + 6 * s) & ~_disc_mask(L, s, sp[0], sp[1], sp[2] + 2 * s)
        body_in = _ellipse_mask(L, s, body[0], body[1], body[2] - 2 * s, body[3] - 2 * s)
        lungs = np.zeros_like(ring)
        for e in ells:
            if e[4] == 0.004:
                lungs |= _ellipse_mask(L, s, e[0], e[1], e[2] + 2 * s, e[3] + 2 * s)
        out["roi2"] = (spine, ring & body_in & ~lungs)
    return out


def evaluate(c: synth.Case, f: np.ndarray, truth: np.ndarray) -> Dict[str, float]:
    """Mean over phases of the CNRs and of the SNR of a reconstruction f[N][ny][nx]."""
    res: Dict[str, list] = {"snr_db": []}
    for i in range(c.geom.n_phases):
        res["snr_db"].append(snr_db(f[i], truth[i]))
        for name, (roi, bg) in rois(c, i).items():
            res.setdefault("cnr_" + name, []).append(cnr(f[i], roi, bg))
    return {k: float(np.mean(v)) for k, v in res.items()}


MU_SWEEP = (0.25, 0.5, 1.0, 2.0)
H_SCALE_SWEEP = (0.5, 1.0, 2.0)


def sweep(c: synth.Case, d, geo, y, w, f0, k_outer: int):
    """TNLM image quality over the grid mu_hat x h-scale (each from the FBP start)."""
    import torch
    import paper_1009_1351_gb300 as tn

    rows = []
    for mu in MU_SWEEP:
        for hs in H_SCALE_SWEEP:
            p = synth.Params(**{**c.params.__dict__, "k_outer": k_outer, "mu_hat": mu,
                                "h": c.params.h * hs})
            f = f0.clone()
            tn.tnlm_reconstruct(geo, p, y, w, f)
            torch.cuda.synchronize()
            rows.append({"mu_hat": mu, "h": p.h, **evaluate(c, f.double().cpu().numpy(), d["truth"])})
    return rows


def main() -> None:
    import torch
    import paper_1009_1351_gb300 as tn

    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="mid_a")
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--sweep", action="store_true", help="also run the mu_hat x h grid")
    args = ap.parse_args()
    c = synth.case(args.case)
    d = synth.make_inputs(c)
    p = c.params if args.k is None else synth.Params(**{**c.params.__dict__, "k_outer": args.k})
    geo = tn.tnlm_create_geometry(c.geom)
    y = torch.tensor(d["y"], dtype=torch.float32, device="cuda")
    w = torch.tensor(d["w"], dtype=torch.float32, device="cuda")
    f = torch.zeros((c.geom.n_phases, c.geom.ny, c.geom.nx), device="cuda")
    tn.tnlm_fbp(geo, y, f)
    torch.cuda.synchronize()
    fbp = f.double().cpu().numpy()
    f_init = f.clone()
    tn.tnlm_reconstruct(geo, p, y, w, f)
    torch.cuda.synchronize()
    tnlm = f.double().cpu().numpy()
    # the paper's FBP baseline reconstructs each phase from its own views only
    fbp_phase = np.zeros_like(fbp)
    for i in range(c.geom.n_phases):
        gi = synth.Geometry(**{**c.geom.__dict__})
        yi = np.zeros_like(d["y"])
        yi[:] = d["y"][i]
        ang = np.tile(c.geom.view_angles().reshape(c.geom.n_phases, -1)[i], c.geom.n_phases)
        geo_i = tn.tnlm_create_geometry(gi, angles=ang)
        yt = torch.tensor(yi, dtype=torch.float32, device="cuda")
        fi = torch.zeros_like(f)
        tn.tnlm_fbp(geo_i, yt, fi)
        torch.cuda.synchronize()
        # the N copies of phase i's views are weighted 2 pi / (N V) each: together
        # exactly the single-phase FBP with weight 2 pi / V
        fbp_phase[i] = fi[0].double().cpu().numpy()
    out = {"case": args.case, "k_outer": p.k_outer,
           "fbp_per_phase": evaluate(c, fbp_phase, d["truth"]),
           "fbp_all_views_init": evaluate(c, fbp, d["truth"]),
           "tnlm": evaluate(c, tnlm, d["truth"])}
    if args.sweep:
        out["sweep"] = sweep(c, d, geo, y, w, f_init, p.k_outer)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
