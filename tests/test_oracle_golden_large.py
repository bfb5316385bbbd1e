"""The stored full-length oracle values belong to the current inputs (CPU).

tests/golden/large_<s>_k100.txt and batch<i>_k50.txt hold FP64-oracle
results after the full K of the 512^2 workload and of four slices of the
batched workload; writing them takes hours, so they are not regenerated
here.  What is checked is that each file still describes the workload the
GPU tests and the benchmark compare against: its iteration count is the
workload's K, its pixel positions are the seeded ones, its monitors are
finite and positive, and its first data-residual monitor -- the data term of the start image,
sum_i ||Sigma^{-1/2}(P_i f_i^(0) - y_i)||^2 (Eq. 1's first term), which
the oracle recomputes here in seconds from the seeded inputs (the FBP start
for the 512^2 files, the constant 0.01 start for the batch files) --
matches to 1e-12.  A change of the input generator, of the geometry or of
the start image that would leave a stale file in place fails here.
"""
import os
import sys

import numpy as np
import pytest

from paper_1009_1351_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_golden  # noqa: E402


@pytest.mark.parametrize("name", ["large_b", "large_a"])
def test_large_golden_matches_the_current_workload(oracle_mod, name):
    gold = make_golden.read_large(name)
    if gold is None:
        pytest.skip(f"no stored values for {name}")
    iters, pix = gold
    c = synth.case(name)
    assert c.params.k_outer == make_golden.LARGE_K
    assert [k for k, _, _ in iters] == list(range(1, make_golden.LARGE_K + 1))
    assert all(np.isfinite(r) and r > 0 and np.isfinite(d) and d > 0 for _, r, d in iters)
    pos = make_golden.large_positions((c.geom.n_phases, c.geom.ny, c.geom.nx))
    assert np.array_equal(np.array([p[:3] for p in pix]), pos)
    d = synth.make_inputs(c)
    G = oracle_mod.Geom(c.geom)
    y32, w32 = d["y"].astype(np.float32), d["w"].astype(np.float32)
    f0 = oracle_mod.fbp(G, y32)
    assert oracle_mod.data_term(G, y32, w32, f0) == pytest.approx(iters[0][2], rel=1e-12)


@pytest.mark.parametrize("slot", range(4))
def test_batch_golden_matches_the_current_workload(oracle_mod, slot):
    items = synth.batch_cases(64)
    i = make_golden.batch_pick(items)[slot]
    gold = make_golden.read_batch(i)
    if gold is None:
        pytest.skip(f"no stored values for batch slice {i}")
    iters, pix = gold
    c, off = items[i]
    assert c.params.k_outer == make_golden.BATCH_K
    assert [k for k, _, _ in iters] == list(range(1, make_golden.BATCH_K + 1))
    pos = make_golden.large_positions((c.geom.n_phases, c.geom.ny, c.geom.nx),
                                      make_golden.BATCH_SAMPLES, make_golden.BATCH_SEED)
    assert np.array_equal(np.array([p[:3] for p in pix]), pos)
    d = synth.make_inputs(c, off)
    G = oracle_mod.Geom(c.geom)
    f0 = np.full((c.geom.n_phases, c.geom.ny, c.geom.nx), 0.01, np.float32)
    got = oracle_mod.data_term(G, d["y"].astype(np.float32), d["w"].astype(np.float32), f0)
    assert got == pytest.approx(iters[0][2], rel=1e-12)
