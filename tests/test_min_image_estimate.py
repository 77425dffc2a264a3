"""Host check of the image-index estimate used by the device minimum image (geom.cuh, min_image_k).

The kernels take n = rint(dk / L) from an FP32 estimate: dk truncated to its leading 20 mantissa bits
(the high word of the double), times (float) 1/L in FP32, used only when |estimate| <= 2 and it is
more than 1e-5 from a half-integer; otherwise they run the FP64 operations.  This test restates that
rule in numpy and checks, over random and adversarial differences (exact half-box distances, values
one ulp around them, tiny and signed-zero differences, unwrapped coordinates), that whenever the
estimate is used it gives the same index, so the minimum-image difference is bit-identical to the
FP64 formula of the oracle (dk - L rint(dk (1/L))).
"""
import numpy as np


def _estimate(dk, invLf):
    """(use, n) of the device rule for FP64 differences dk (array)."""
    bits = dk.view(np.uint64)
    hi = (bits >> np.uint64(32)).astype(np.uint32)
    e = ((hi >> 20) & 0x7FF).astype(np.int64) - 1023 + 127
    small = e < 140
    ef = np.clip(e, 0, 255).astype(np.uint32)
    fbits = (hi & np.uint32(0x80000000)) | (ef << np.uint32(23)) | ((hi & np.uint32(0xFFFFF)) << np.uint32(3))
    xf = np.where(e > 0, fbits.view(np.float32), np.float32(0)).astype(np.float32) * np.float32(invLf)
    xf = xf.astype(np.float32)
    nf = np.rint(xf)
    use = small & (np.abs(xf) <= 2) & (np.abs(np.abs(xf - nf) - np.float32(0.5)) > np.float32(1e-5)) & (np.abs(nf) <= 1)
    return use, nf.astype(np.float64)


def test_image_index_estimate_matches_fp64():
    rng = np.random.default_rng(3)
    for L in (12.42, 36.34, 109.02, 198.72, 3.634 * 10, 7.3):
        invL = 1.0 / L
        invLf = np.float32(invL)
        half = L / 2
        cases = [rng.uniform(-L, L, 200000), rng.uniform(-3 * L, 3 * L, 50000),
                 np.array([half, -half, 0.0, -0.0, 1e-300, -1e-300, L, -L, 1.5 * L, -1.5 * L]),
                 np.nextafter(np.full(1000, half), np.inf) + rng.integers(-3, 4, 1000) * np.spacing(half),
                 half + rng.normal(scale=1e-9, size=20000), -half + rng.normal(scale=1e-9, size=20000),
                 half * (1 + rng.normal(scale=1e-6, size=20000))]
        dk = np.concatenate(cases).astype(np.float64)
        n_exact = np.rint(dk * invL)
        use, n_est = _estimate(dk, invLf)
        assert use[:200000].mean() > 0.999   # differences within one box length: nearly always
        assert np.array_equal(n_est[use], n_exact[use]), L
        # the shortened forms give the FP64 formula's result bit for bit
        d_exact = dk - L * n_exact
        d0 = np.where(dk.view(np.uint64) == np.uint64(0x8000000000000000), 0.0, dk)   # -0 becomes +0
        d_short = np.where(n_est == 0, d0, np.where(n_est == 1, dk - L, dk + L))
        assert np.array_equal(d_short[use].view(np.uint64), d_exact[use].view(np.uint64))
