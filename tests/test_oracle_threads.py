"""The threaded oracle variants (used only to time the oracle on all host
cores) compute what the single-threaded oracle computes: the same images bit
for bit (pixels are independent) and the same gradients up to the order of
the FP64 partial sums."""
import numpy as np

from oracle import oracle as O
from paper_2509_25191_gb300 import synth


def test_threaded_oracle_equals_single_threaded():
    sc, vw = synth.orbit_views(2, 3000, 2, 96, 64, 1000.0 * 96 / 979.0)
    rng = np.random.default_rng(0)
    ups = [rng.standard_normal((3, int(vw.height[v]), int(vw.width[v]))) for v in range(vw.n)]
    f1 = O.forward(sc, vw)
    f4 = O.forward(sc, vw, threads=5)
    for a, b in zip(f1, f4):
        assert np.array_equal(a["image"], b["image"]) and np.array_equal(a["T"], b["T"])
        assert np.array_equal(a["n_contrib"], b["n_contrib"]) and np.array_equal(a["flags"], b["flags"])
        for k in ("xy", "conic", "rgb", "radius"):
            assert np.array_equal(a["proj"][k], b["proj"][k])
    g1, dRt1, tw1, _ = O.backward(sc, vw, f1, ups)
    g4, dRt4, tw4, _ = O.backward(sc, vw, f4, ups, threads=5)
    for k in g1:
        assert np.allclose(g4[k], g1[k], rtol=1e-12, atol=1e-15 * np.abs(g1[k]).max())
    assert np.allclose(dRt4, dRt1, rtol=1e-12, atol=1e-15 * np.abs(dRt1).max())
    assert np.abs(g1["means"]).max() > 0
