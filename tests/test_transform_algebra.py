"""The transform algebra the multi-pass uneven engine (uneven_big.cu) relies on, restated in numpy
and checked against numpy's FFT on the CPU: Bluestein's chirp z-transform with the phase reduced mod
2n and the kernel spectrum divided by M, the inverse as conj(DFT(conj x)), two real rows through one
complex transform in both directions (with the imaginary parts of the DC and Nyquist bins dropped
on the way back, as a real inverse transform does), and the filter spectra as direct DFTs over the
taps placed with their centre at the origin."""
import numpy as np
import pytest


def smooth7(n):
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def bluestein(x, inverse=False):
    n = len(x)
    M = 2 * n - 1
    while not smooth7(M):
        M += 1
    j = np.arange(n)
    w = np.exp(-1j * np.pi * ((j * j) % (2 * n)) / n)        # chirp, phase reduced mod 2n
    b = np.zeros(M, complex)
    b[:n] = np.conj(w)
    b[M - np.arange(1, n)] = np.conj(w[1:])
    bhat = np.fft.fft(b) / M                                   # kernel spectrum, 1/M folded in
    a = np.zeros(M, complex)
    a[:n] = (np.conj(x) if inverse else x) * w
    y = np.fft.ifft(np.fft.fft(a) * bhat) * M                  # unnormalised inverse of length M
    out = y[:n] * w
    return np.conj(out) if inverse else out


@pytest.mark.parametrize("n", [11, 13, 67, 97, 131, 181, 487, 509, 1021])
def test_bluestein_equals_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.fft(x)
    assert np.abs(bluestein(x) - ref).max() <= 1e-12 * np.abs(ref).max()
    inv = np.fft.ifft(x) * n                                   # unnormalised inverse
    assert np.abs(bluestein(x, inverse=True) - inv).max() <= 1e-12 * np.abs(inv).max()


@pytest.mark.parametrize("W", [8, 9, 76, 131, 512])
def test_two_real_rows_per_complex_transform(W):
    rng = np.random.default_rng(W)
    Wc = W // 2 + 1
    ua, ub = rng.standard_normal(W), rng.standard_normal(W)
    # forward: U_a(k) = (Z(k) + conj Z(-k)) / 2, U_b(k) = (Z(k) - conj Z(-k)) / 2i
    Z = np.fft.fft(ua + 1j * ub)
    Zm = np.conj(Z[(-np.arange(Wc)) % W])
    Ua, Ub = (Z[:Wc] + Zm) / 2, (Z[:Wc] - Zm) / 2j
    np.testing.assert_allclose(Ua, np.fft.rfft(ua), atol=1e-12)
    np.testing.assert_allclose(Ub, np.fft.rfft(ub), atol=1e-12)
    # inverse: each half spectrum completed by Hermitian symmetry, DC / Nyquist imaginary parts
    # dropped, z = IDFT(X_a + i X_b) = x_a + i x_b
    Xa = np.fft.rfft(ua) + 1j * rng.standard_normal(Wc) * 1e-3 * (np.arange(Wc) % W == 0)
    Xb = np.fft.rfft(ub)

    def complete(X):
        X = X.copy()
        X[0] = X[0].real
        if W % 2 == 0:
            X[-1] = X[-1].real
        full = np.zeros(W, complex)
        full[:Wc] = X
        full[Wc:] = np.conj(X[W - np.arange(Wc, W)])
        return full

    z = np.fft.ifft(complete(Xa) + 1j * complete(Xb))
    np.testing.assert_allclose(z.real, np.fft.irfft(Xa, n=W), atol=1e-12)
    np.testing.assert_allclose(z.imag, np.fft.irfft(Xb, n=W), atol=1e-12)


@pytest.mark.parametrize("H,W,fh,fw", [(67, 131, 11, 11), (9, 8, 5, 3), (200, 181, 7, 9)])
def test_direct_filter_dft_equals_placed_filter_transform(H, W, fh, fw):
    rng = np.random.default_rng(H * W)
    f = rng.standard_normal((fh, fw))
    ch, cw = (fh - 1) // 2, (fw - 1) // 2
    grid = np.zeros((H, W))
    for ta in range(fh):
        for tb in range(fw):
            grid[(ta - ch) % H, (tb - cw) % W] = f[ta, tb]
    ref = np.fft.rfft2(grid)
    Wc = W // 2 + 1
    kw, h = np.arange(Wc), np.arange(H)
    # row DFTs of the tap rows, then fh terms per output
    R = np.array([[np.sum(f[ta] * np.exp(-2j * np.pi * kw[c] * (np.arange(fw) - cw) / W)) for c in range(Wc)]
                  for ta in range(fh)])
    out = np.einsum("tc,ht->hc", R, np.exp(-2j * np.pi * np.outer(h, np.arange(fh) - ch) / H))
    assert np.abs(out - ref).max() <= 1e-10 * np.abs(ref).max()
