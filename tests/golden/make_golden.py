"""Writes the stored expected values under tests/golden/ from the FP64
oracle alone (test infrastructure: nothing here touches the CUDA path).

    python tests/golden/make_golden.py

tiny_k3.txt: the tiny workload (64 x 64 pixels of 1 mm, 10 phases, 60 views
per phase, 128 bins of 1.2 mm, SID 1000 / SDD 1500 mm, I0 = 1e4, d = 3,
W = 5, h = 0.006, mu_hat = 0.5, M1 = 3 CGLS steps, M2 = 5 Gauss-Jacobi
sweeps, clamp), three outer iterations of the TNLM algorithm box from the
constant start image 0.01: the relative change and data residual after
every iteration and 96 pixel values at seeded positions.

large_<s>_k100.txt: a 512 x 512 workload (0.8 mm pixels, 10 phases, 888
bins of 1 mm, d = 7, W = 15, h = 0.014, mu_hat = 0.5, M1 = 3, M2 = 5,
clamp; scenario a: 360 views per phase at I0 = 5e3, b: 90 views at
I0 = 1e5), the full K = 100 outer iterations of the TNLM algorithm box from
the oracle's own FBP of all views (box step 1): the relative change and data
residual after every iteration and 8192 pixel values at seeded positions
over the whole image.  At 8 host threads one file takes 30-60 minutes.

    python tests/golden/make_golden.py large_a large_b

batch<i>_k50.txt: the four slices sampled from the 64-slice batched
workload (the first of each side length 256 / 384 / 512 and the first other
60-view slice; d = 5, W = 11, h = 0.01, mu_hat = 0.5, M1 = 3, M2 = 5), the
full K = 50 outer iterations from the constant start 0.01: histories and
4096 pixel values at seeded positions.

    python tests/golden/make_golden.py batch
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

K = 3
SAMPLES = 96
SAMPLE_SEED = 3141


def sample_positions(shape, n=SAMPLES, seed=SAMPLE_SEED):
    """Seeded positions inside the body ellipse (central 60 % of each axis)."""
    rng = np.random.default_rng(seed)
    N, ny, nx = shape
    return np.stack([rng.integers(0, N, n), rng.integers(ny // 5, ny - ny // 5, n),
                     rng.integers(nx // 5, nx - nx // 5, n)], axis=1)


def tiny_k3():
    import oracle
    from paper_1009_1351_gb300 import synth
    c = synth.case("tiny")
    d = synth.make_inputs(c)
    p = synth.Params(**{**c.params.__dict__, "k_outer": K})
    f0 = np.full((c.geom.n_phases, c.geom.ny, c.geom.nx), 0.01, np.float32)
    f, rel, res = oracle.reconstruct(oracle.Geom(c.geom), d["y"].astype(np.float32),
                                     d["w"].astype(np.float32), f0, p)
    return f, np.asarray(rel), np.asarray(res)


def write_tiny_k3(path=os.path.join(HERE, "tiny_k3.txt")):
    f, rel, res = tiny_k3()
    pos = sample_positions(f.shape)
    with open(path, "w") as fh:
        fh.write("# TNLM algorithm box, tiny workload, K = 3 from f0 = 0.01 (FP64 oracle).\n")
        fh.write("# Written by tests/golden/make_golden.py; see its docstring for the workload.\n")
        fh.write("# iter <k> <relative change> <data residual>\n")
        fh.write("# pixel <phase> <row> <column> <value>\n")
        for k in range(len(rel)):
            fh.write(f"iter {k + 1} {float(rel[k])!r} {float(res[k])!r}\n")
        for i, y, x in pos:
            fh.write(f"pixel {i} {y} {x} {float(f[i, y, x])!r}\n")


LARGE_K = 100
LARGE_SAMPLES = 8192
LARGE_SEED = 2718


def large_positions(shape, n=LARGE_SAMPLES, seed=LARGE_SEED):
    """Seeded positions anywhere in the [N][ny][nx] image."""
    rng = np.random.default_rng(seed)
    N, ny, nx = shape
    return np.stack([rng.integers(0, N, n), rng.integers(0, ny, n), rng.integers(0, nx, n)], axis=1)


def large_path(name):
    return os.path.join(HERE, f"{name}_k{LARGE_K}.txt")


def write_large(name):
    """Full-length reconstruction of one 512^2 scenario from the oracle's FBP."""
    import oracle
    from paper_1009_1351_gb300 import synth
    c = synth.case(name)
    assert c.params.k_outer == LARGE_K
    d = synth.make_inputs(c)
    G = oracle.Geom(c.geom)
    y32, w32 = d["y"].astype(np.float32), d["w"].astype(np.float32)
    f0 = oracle.fbp(G, y32)
    f, rel, res = oracle.reconstruct(G, y32, w32, f0, c.params)
    pos = large_positions(f.shape)
    with open(large_path(name), "w") as fh:
        fh.write(f"# TNLM algorithm box, workload {name}, K = {LARGE_K} from the FBP of all views "
                 "(FP64 oracle).\n")
        fh.write("# Written by tests/golden/make_golden.py; see its docstring for the workload.\n")
        fh.write(f"# norm {float(np.linalg.norm(f))!r}\n")
        fh.write("# iter <k> <relative change> <data residual>\n")
        fh.write("# pixel <phase> <row> <column> <value>\n")
        for k in range(len(rel)):
            fh.write(f"iter {k + 1} {float(rel[k])!r} {float(res[k])!r}\n")
        for i, y, x in pos:
            fh.write(f"pixel {i} {y} {x} {float(f[i, y, x])!r}\n")


def read_large(name):
    """(iters, pixels) of a stored 512^2 file, or None when it is missing."""
    if not os.path.exists(large_path(name)):
        return None
    return read_tiny_k3(large_path(name))


BATCH_K = 50
BATCH_SAMPLES = 4096
BATCH_SEED = 1618


def batch_pick(items):
    """Indices of the four sampled slices of the batched workload: the first
    slice of each side length, then the first remaining 60-view slice."""
    pick, seen = [], set()
    for i, (c, _) in enumerate(items):
        if c.geom.nx not in seen:
            seen.add(c.geom.nx)
            pick.append(i)
    pick.append(next(i for i, (c, _) in enumerate(items) if c.geom.n_views == 60 and i not in pick))
    return pick


def batch_path(i):
    return os.path.join(HERE, f"batch{i:02d}_k{BATCH_K}.txt")


def write_batch(i):
    """Slice i of the 64-slice batched workload, K = 50 outer iterations from
    the constant start 0.01 (the oracle has no mixed precision: FP64 throughout)."""
    import oracle
    from paper_1009_1351_gb300 import synth
    c, off = synth.batch_cases(64)[i]
    assert c.params.k_outer == BATCH_K
    d = synth.make_inputs(c, off)
    G = oracle.Geom(c.geom)
    f0 = np.full((c.geom.n_phases, c.geom.ny, c.geom.nx), 0.01, np.float32)
    f, rel, res = oracle.reconstruct(G, d["y"].astype(np.float32), d["w"].astype(np.float32), f0, c.params)
    pos = large_positions(f.shape, BATCH_SAMPLES, BATCH_SEED)
    with open(batch_path(i), "w") as fh:
        fh.write(f"# TNLM algorithm box, slice {i} of the batched workload ({c.geom.nx}^2, "
                 f"{c.geom.n_views} views), K = {BATCH_K} from f0 = 0.01 (FP64 oracle).\n")
        fh.write("# Written by tests/golden/make_golden.py; see its docstring for the workload.\n")
        fh.write("# iter <k> <relative change> <data residual>\n")
        fh.write("# pixel <phase> <row> <column> <value>\n")
        for k in range(len(rel)):
            fh.write(f"iter {k + 1} {float(rel[k])!r} {float(res[k])!r}\n")
        for ph, y, x in pos:
            fh.write(f"pixel {ph} {y} {x} {float(f[ph, y, x])!r}\n")


def read_batch(i):
    if not os.path.exists(batch_path(i)):
        return None
    return read_tiny_k3(batch_path(i))


def read_tiny_k3(path=os.path.join(HERE, "tiny_k3.txt")):
    iters, pix = [], []
    for line in open(path):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "iter":
            iters.append((int(t[1]), float(t[2]), float(t[3])))
        elif t[0] == "pixel":
            pix.append((int(t[1]), int(t[2]), int(t[3]), float(t[4])))
    return iters, pix


if __name__ == "__main__":
    import oracle
    oracle.build()
    names = sys.argv[1:] or ["tiny"]
    for nm in names:
        if nm == "tiny":
            write_tiny_k3()
            print("wrote", os.path.join(HERE, "tiny_k3.txt"))
        elif nm == "batch":
            from paper_1009_1351_gb300 import synth
            for i in batch_pick(synth.batch_cases(64)):
                write_batch(i)
                print("wrote", batch_path(i), flush=True)
        else:
            write_large(nm)
            print("wrote", large_path(nm))
