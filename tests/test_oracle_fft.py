"""Pins for the oracle's radix-2 FFT against the dense DFT matrix and numpy.

The split-step method (Sec. IV) needs forward and inverse 3D DFTs; the oracle
writes its own radix-2 transform, so it is checked here against definitions
that share nothing with it.
"""
import numpy as np
import pytest


def dft_matrix(n, sign):
    j = np.arange(n)
    # reduce jk mod n first so the angle stays exact for large n
    return np.exp(sign * 2j * np.pi * (np.outer(j, j) % n) / n)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128, 256, 1024])
def test_fft1d_matches_dense_dft(orc, n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    fwd = orc.fft1d(a, -1)
    ref = a @ dft_matrix(n, -1).T
    assert rel(fwd, ref) < 1e-13
    inv = orc.fft1d(a, +1)
    ref_inv = a @ dft_matrix(n, +1).T / n
    assert rel(inv, ref_inv) < 1e-13


def test_fft3d_matches_dense_dft_8cubed(orc):
    rng = np.random.default_rng(8)
    a = rng.standard_normal((8, 8, 8)) + 1j * rng.standard_normal((8, 8, 8))
    F = dft_matrix(8, -1)
    ref = np.einsum("zc,yb,xa,cba->zyx", F, F, F, a)
    assert rel(orc.fft3d(a, -1), ref) < 1e-14
    Fi = dft_matrix(8, +1) / 8
    ref_i = np.einsum("zc,yb,xa,cba->zyx", Fi, Fi, Fi, a)
    assert rel(orc.fft3d(a, +1), ref_i) < 1e-14


@pytest.mark.parametrize("shape", [(32, 8, 16), (1, 16, 64), (4, 1, 2), (64, 32, 8)])
def test_fft3d_matches_numpy_anisotropic(orc, shape):
    rng = np.random.default_rng(sum(shape))
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    assert rel(orc.fft3d(a, -1), np.fft.fftn(a)) < 1e-13
    assert rel(orc.fft3d(a, +1), np.fft.ifftn(a)) < 1e-13


def test_fft_roundtrip_and_parseval(orc):
    rng = np.random.default_rng(1)
    a = rng.standard_normal((16, 32, 64)) + 1j * rng.standard_normal((16, 32, 64))
    A = orc.fft3d(a, -1)
    assert rel(orc.fft3d(A, +1), a) < 1e-14
    assert abs(np.sum(np.abs(A) ** 2) / a.size - np.sum(np.abs(a) ** 2)) \
        < 1e-12 * np.sum(np.abs(a) ** 2)


def test_fft_rejects_non_power_of_two(orc):
    with pytest.raises(ValueError):
        orc.fft1d(np.zeros(12, dtype=complex), -1)
