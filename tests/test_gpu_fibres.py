"""Rows a1/a2 (mode-wise FFT and Fourier multipliers on fibres): CUDA path vs the oracle, FP64.

Tolerance: an FP64 radix-p FFT of length N has relative error ~ eps * log N; we allow 1e-12
(relative to the largest input magnitude) for every size used here (N <= 1215)."""
import numpy as np
import pytest
import torch

from oracle import fourier_galerkin as fg

pytestmark = pytest.mark.gpu

SIZES = [3, 5, 7, 9, 11, 13, 15, 21, 25, 27, 45, 63, 81, 135, 243, 405, 729, 1215]


def _dft_axis1(x, sign):
    # sum_n x[o,n,i] exp(sign 2 pi i f n / N): the oracle's F_N (sign -1) or F_N^-1 (sign +1) along axis 1
    N = x.shape[1]
    y = np.moveaxis(x, 1, -1)
    out = fg.dft(y, 1) * N if sign < 0 else fg.idft(y, 1)
    return np.moveaxis(out, -1, 1)


@pytest.mark.parametrize("N", SIZES)
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_fibres_matches_oracle(ctx, N, sign):
    rng = np.random.default_rng(N)
    for outer, inner in [(1, 1), (3, 7), (1, 33), (5, 1), (2, 64)]:
        x = rng.standard_normal((outer, N, inner)) + 1j * rng.standard_normal((outer, N, inner))
        ref = _dft_axis1(x, sign)
        got = ctx.fft_fibres(torch.as_tensor(x, device="cuda"), sign).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * N * np.abs(x).max(), (outer, inner)


@pytest.mark.parametrize("N", [3, 9, 27, 45, 81, 135, 243, 729])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_fibres_f32_matches_oracle(ctx, N, sign):
    # FP32 passes of the mixed full format (81 and 243 take the two-pass kernel: 32 fibres a block, so
    # inner sizes below, at and across 32 and batches whose tiles straddle two outer indices).  An FP32
    # transform errs by a few u_32 log2(N) of the fibre's norm, sqrt(N) max|x| for these inputs.
    rng = np.random.default_rng(3 * N)
    for outer, inner in [(1, 1), (3, 7), (1, 32), (2, 33), (5, 122), (1, 300)]:
        x = (rng.standard_normal((outer, N, inner)) + 1j * rng.standard_normal((outer, N, inner))).astype(np.complex64)
        ref = _dft_axis1(x.astype(np.complex128), sign)
        got = ctx.fft_fibres(torch.as_tensor(x, device="cuda"), sign).cpu().numpy()
        tol = 4 * 2.0 ** -24 * np.log2(N + 1) * np.sqrt(N) * np.abs(x).max()
        assert np.abs(got - ref).max() <= tol, (outer, inner, np.abs(got - ref).max() / tol)
        y = torch.as_tensor(x, device="cuda")
        ctx.fft_fibres(y, sign, out=y)
        assert torch.equal(y.cpu(), torch.as_tensor(got)), (outer, inner)


def test_fft_fibres_in_place_and_empty(ctx):
    x = torch.randn(4, 45, 9, dtype=torch.complex128, device="cuda")
    ref = ctx.fft_fibres(x.clone(), -1)
    y = x.clone()
    ctx.fft_fibres(y, -1, out=y)
    assert torch.allclose(y, ref, atol=1e-12, rtol=0)
    z = torch.empty(0, 45, 9, dtype=torch.complex128, device="cuda")
    assert ctx.fft_fibres(z, -1).shape == z.shape


@pytest.mark.parametrize("N", [3, 9, 15, 45, 63, 243, 1215])
@pytest.mark.parametrize("kind", ["deriv", "gauss", "identity"])
def test_fibre_operator_matches_oracle(ctx, N, kind):
    import paper_1902_07455_gb300 as lrfg
    rng = np.random.default_rng(7 * N)
    K = fg.frequencies(N).astype(np.float64)
    if kind == "deriv":
        m, code, param = 2j * np.pi * K, lrfg.MUL_DERIV, 0.0
    elif kind == "gauss":
        param = 0.37 / N
        m, code = np.exp(-param * K ** 2), lrfg.MUL_GAUSS
    else:
        m, code, param = np.ones(N), lrfg.MUL_IDENTITY, 0.0
    for outer, inner in [(1, 1), (2, 5), (1, 40), (7, 3)]:
        x = rng.standard_normal((outer, N, inner))
        # oracle: F^-1 diag(m) F along the mode
        y = np.moveaxis(x, 1, -1)
        ref = np.real(fg.idft(m * fg.dft(y, 1), 1))
        ref = -1.5 * np.moveaxis(ref, -1, 1)
        got = ctx.fibre_operator(torch.as_tensor(x, device="cuda"), code, param, -1.5).cpu().numpy()
        scale = np.abs(ref).max() + np.abs(x).max()
        assert np.abs(got - ref).max() <= 1e-12 * N * scale


def test_derivative_of_trig_polynomial_is_exact(ctx):
    import paper_1902_07455_gb300 as lrfg
    N = 81
    x = fg.grid_points(N)
    u = np.sin(2 * np.pi * 5 * x).reshape(1, N, 1)
    got = ctx.fibre_operator(torch.as_tensor(u, device="cuda"), lrfg.MUL_DERIV).cpu().numpy()[0, :, 0]
    assert np.allclose(got, 10 * np.pi * np.cos(2 * np.pi * 5 * x), atol=1e-11)
