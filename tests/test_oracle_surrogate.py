"""Pins of the FP64 reference of the warm-start network (CPU).

The reference's gradients come from autograd; they are pinned here by central
finite differences, and the convolution orientation (cross-correlation, taps
at offsets -1..1, padding 1) by a brute-force loop."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import surrogate as S  # noqa: E402
from paper_1801_04577_gb300 import inputs as I  # noqa: E402
from paper_1801_04577_gb300.net import bf16_round, layer_shapes  # noqa: E402


def _case(G=8, cin=2, cout=2, base=2, levels=2, N=2, seed=5):
    shapes = layer_shapes(G, cin, cout, base, levels)
    npar = sum(co * ci * k * k + co for ci, co, k in shapes)
    r = I.splitmix64_uniform(seed, npar + 2 * N * (cin + cout) * G * G + N * G * G)
    params = 0.6 * (2 * r[:npar] - 1)
    o = npar
    x = (2 * r[o:o + N * cin * G * G] - 1).reshape(N, cin, G, G); o += N * cin * G * G
    t = (2 * r[o:o + N * cout * G * G] - 1).reshape(N, cout, G, G); o += N * cout * G * G
    mask = (r[o:o + N * G * G] > 0.3).astype(np.float64).reshape(N, G, G)
    return shapes, params, x, t, mask, levels


def test_autograd_matches_finite_differences():
    shapes, params, x, t, mask, levels = _case()
    L0, g, _ = S.loss_and_grad(params, shapes, levels, x, t, mask)
    idx = np.unique((I.splitmix64_uniform(9, 60) * len(params)).astype(int))
    h = 1e-6
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        fd = (S.loss_and_grad(pp, shapes, levels, x, t, mask)[0] -
              S.loss_and_grad(pm, shapes, levels, x, t, mask)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9), i


def test_convolution_is_cross_correlation_with_unit_padding():
    r = I.splitmix64_uniform(3, 2 * 3 * 5 * 5 + 4 * 3 * 9 + 4)
    x = r[:150].reshape(2, 3, 5, 5)
    w = r[150:150 + 108].reshape(4, 3, 3, 3)
    b = r[258:262]
    y = S.F.conv2d(torch.tensor(x), torch.tensor(w), torch.tensor(b), padding=1).numpy()
    want = np.zeros((2, 4, 5, 5))
    for n in range(2):
        for co in range(4):
            for yy in range(5):
                for xx in range(5):
                    s = b[co]
                    for ci in range(3):
                        for ky in range(3):
                            for kx in range(3):
                                sy, sx = yy + ky - 1, xx + kx - 1
                                if 0 <= sy < 5 and 0 <= sx < 5:
                                    s += w[co, ci, ky, kx] * x[n, ci, sy, sx]
                    want[n, co, yy, xx] = s
    np.testing.assert_allclose(y, want, atol=1e-13)


def test_bf16_rounding_is_nearest_even():
    a = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 1e-30, 65504.0], np.float32)
    r = bf16_round(a)
    # bfloat16 keeps 8 significand bits: 1 + 1/128 spacing near 1
    assert r[0] == 1.0
    assert r[1] == 1.0            # exactly halfway between 1 and 1+2^-7: ties to even
    assert r[2] == np.float32(1.0078125)
    assert abs(r[3] - a[3]) <= 2.0 ** -7 * 4
    assert (r.view(np.uint32) & 0xFFFF == 0).all()


def test_rounded_convolution_backward_matches_autograd_when_rounding_is_identity():
    """The hand-written backward of the rounded convolution (input gradient by
    conv2d_input, weight gradient by conv2d_weight, bias by a sum) reduces to
    the finite-difference-pinned autograd network when nothing is rounded."""
    shapes, params, x, t, mask, levels = _case(G=8, cin=3, cout=2, base=3, levels=3)
    L0, g0, y0 = S.loss_and_grad(params, shapes, levels, x, t, mask)
    L1, g1, y1 = S.loss_and_grad(params, shapes, levels, x, t, mask, rnd=lambda a: a)
    assert L1 == pytest.approx(L0, rel=1e-13)
    np.testing.assert_allclose(y1, y0, rtol=0, atol=1e-13)
    np.testing.assert_allclose(g1, g0, rtol=0, atol=1e-12 * np.abs(g0).max())


def test_oracle_bf16_rounding_values():
    """bf16() rounds to float32 first, then to bfloat16 ties-to-even (spacing
    2^-7 just above 1)."""
    u = 2.0 ** -8
    v = torch.tensor([1 + u, 1 + 3 * u, 1 + u + 2.0 ** -20, -(1 + 3 * u), 3.0, 1 + u + 2.0 ** -40],
                     dtype=torch.float64)
    want = [1.0, 1 + 4 * u, 1 + 2 * u, -(1 + 4 * u), 3.0, 1.0]
    assert S.bf16(v).tolist() == want


def test_bf16_network_differs_from_fp64_by_bf16_rounding_only():
    """With rounding on, the loss moves by about the bf16 unit roundoff (2^-9
    relative per operand), not by O(1): the rounding is applied to the GEMM
    operands only."""
    shapes, params, x, t, mask, levels = _case(G=8, cin=3, cout=2, base=3, levels=3)
    L0, g0, y0 = S.loss_and_grad(params, shapes, levels, x, t, mask)
    L1, g1, y1 = S.loss_and_grad(params, shapes, levels, x, t, mask, rnd=S.bf16)
    assert 0 < abs(L1 - L0) / L0 < 2e-2
    assert np.abs(y1 - y0).max() < 5e-2 * np.abs(y0).max()
