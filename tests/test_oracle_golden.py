"""The stored expected values of tests/golden/ (written by
tests/golden/make_golden.py from the FP64 oracle) are reproduced by the
oracle as it stands: a change to the oracle's arithmetic shows up here
and has to be justified by the passage of the paper it follows."""
import numpy as np

from tests.golden import make_golden


def test_oracle_reproduces_the_tiny_k3_fixture(oracle_mod):
    iters, pix = make_golden.read_tiny_k3()
    assert [k for k, _, _ in iters] == [1, 2, 3] and len(pix) == make_golden.SAMPLES
    f, rel, res = make_golden.tiny_k3()
    np.testing.assert_allclose(rel, [r for _, r, _ in iters], rtol=1e-9)
    np.testing.assert_allclose(res, [r for _, _, r in iters], rtol=1e-9)
    got = np.array([f[i, y, x] for i, y, x, _ in pix])
    want = np.array([v for _, _, _, v in pix])
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-15)
    pos = make_golden.sample_positions(f.shape)
    assert [tuple(p) for p in pos] == [(i, y, x) for i, y, x, _ in pix]
