"""The FP64 kernels' tanh on the GPU against CUDA's tanh and the C library's.

The device routine (degree-10 Taylor table, see test_tanh_table.py; the
terms of degree 6-10, below 2^-31 of the result, summed in FP32) adds the
rounding of its Horner steps to the table's 0.77 ulp (about 1.1 ulp in all
in a CPU emulation); CUDA's and the C library's tanh carry their own errors
of about 1-2 ulp.  Agreement within
4 ulp of both on 4 million random arguments over the table's range and
beyond, odd symmetry, and exact special values pin the device evaluation
(wrong interval index, wrong coefficient stride or a lost sign fail by far
more).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2005_00223_gb300 as pkg
    pkg.load()
    return pkg


def _ulps(a, b):
    ia = a.view(np.int64).astype(np.int64)
    ib = b.view(np.int64).astype(np.int64)
    ia = np.where(ia < 0, np.int64(-2 ** 63) - ia, ia)    # monotone integer order across zero
    ib = np.where(ib < 0, np.int64(-2 ** 63) - ib, ib)
    return np.abs(ia - ib)


def test_tanh_f64_against_cuda_and_libm(dp):
    import torch
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-17, 17, 2_000_000), rng.normal(0, 1.5, 1_000_000),
                        rng.uniform(-0.05, 0.05, 500_000), np.arange(-4096, 4097) / 256.0,
                        10.0 ** rng.uniform(-300, 0, 500_000) * rng.choice([-1, 1], 500_000)])
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    dp.dp_tanh_f64_dev(xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    ycuda = torch.tanh(xd).cpu().numpy()
    ylib = np.tanh(x)
    assert _ulps(y, ycuda).max() <= 4, _ulps(y, ycuda).max()
    assert _ulps(y, ylib).max() <= 4, _ulps(y, ylib).max()
    # odd symmetry is exact
    ym = torch.empty_like(xd)
    dp.dp_tanh_f64_dev(-xd, ym)
    np.testing.assert_array_equal(ym.cpu().numpy(), -y)


def test_tanh_f64_special_values(dp):
    import torch
    x = np.array([0.0, -0.0, 16.0, -16.0, np.nextafter(16.0, 0), 30.0, -1e300, np.inf, -np.inf, 5e-324,
                  -5e-324, 1e-200])
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    dp.dp_tanh_f64_dev(xd, yd)
    y = yd.cpu().numpy()
    assert y[0] == 0 and not np.signbit(y[0])
    assert y[1] == 0 and np.signbit(y[1])
    big = [2, 3, 5, 6, 7, 8]                                 # |x| >= 16: CUDA's own tanh
    np.testing.assert_array_equal(y[big], torch.tanh(xd).cpu().numpy()[big])
    assert (np.abs(y[big]) <= 1).all() and (np.sign(y[big]) == np.sign(x[big])).all()
    assert _ulps(y[4:5], np.tanh(x[4:5])).max() <= 4
    np.testing.assert_array_equal(y[9:], x[9:])            # tanh(x) = x below 2^-26
    n = torch.tensor([np.nan], dtype=torch.float64, device="cuda")
    dp.dp_tanh_f64_dev(n, n)
    assert np.isnan(n.cpu().numpy()[0])
