"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no step of the method: it only draws the initial fields and the
instance parameters. Every consumer (CUDA path, oracle, tests, bench) receives the
same host arrays from here.

Initial fields.  The paper starts from a random perturbation of the magnetic field
(Sec. 4, "Implementation"); here the perturbation is a seeded complex Gaussian
spectrum with amplitude |k3|^-2, made solenoidal (k3 . b = 0, i.e. the constraint
of Eq. 4c / 6c holds) and scaled to unit 2-norm, because the problem is linear and
only relative errors are reported.

Layout of a field: complex128 array [3][n][n] = [component][ky][kx] of spectral
coefficients b_hat(k) with b(x) = sum_k b_hat(k) exp(i k.x), indices in FFT order
(index i <-> wavenumber i for i < n/2, i - n otherwise). Modes outside the
dealiased square |kx|, |ky| <= n // 3 are zero.
"""
import numpy as np


def fft_wavenumbers(n):
    """Integer wavenumbers of an n-point periodic grid on [0, 2 pi), FFT order."""
    i = np.arange(n)
    return np.where(i < n // 2, i, i - n).astype(np.float64)


def initial_field(n, kz, seed):
    """Seeded solenoidal unit-norm field on the n x n grid (complex128 [3][n][n])."""
    return _solenoidal(n, kz, seed, decay=True)


def flat_field(n, kz, seed):
    """Seeded solenoidal unit-norm field whose kept modes all have the same expected
    amplitude (no |k3|^-2 decay): a test input that weighs the highest kept wavenumbers
    as much as the lowest (complex128 [3][n][n])."""
    return _solenoidal(n, kz, seed, decay=False)


def _solenoidal(n, kz, seed, decay):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((2, 3, n, n))
    k = fft_wavenumbers(n)
    kx = k[None, :]
    ky = k[:, None]
    K = n // 3
    keep = (np.abs(kx) <= K) & (np.abs(ky) <= K)
    k2 = kx * kx + ky * ky + kz * kz
    b = (g[0] + 1j * g[1]) / np.sqrt(2.0)
    if decay:
        b = b / k2
    b = np.where(keep, b, 0.0)
    kvec = (np.broadcast_to(kx, (n, n)), np.broadcast_to(ky, (n, n)),
            np.full((n, n), float(kz)))
    kdotb = kvec[0] * b[0] + kvec[1] * b[1] + kvec[2] * b[2]
    for c in range(3):
        b[c] = b[c] - kvec[c] * kdotb / k2
    b = np.where(keep, b, 0.0)
    return (b / np.sqrt(np.sum(np.abs(b) ** 2))).astype(np.complex128)


def initial_batch(n, kz, seeds):
    """Stack of initial_field for several seeds: complex128 [len(seeds)][3][n][n]."""
    return np.stack([initial_field(n, kz, s) for s in seeds])


def sweep_instance(seed):
    """Parameters of one instance of the batched Rm / kz sweep.

    Flow is Roberts for even seeds and Galloway-Proctor for odd ones; Rm is
    log-uniform in [50, 3200]; the grid side follows Rm^(1/2) as 64 * sqrt(Rm / 50),
    rounded in log2 to a power of two in [64, 512]; kz is uniform in [0.2, 1.5].
    """
    rng = np.random.default_rng(seed)
    Rm = float(np.exp(rng.uniform(np.log(50.0), np.log(3200.0))))
    kz = float(rng.uniform(0.2, 1.5))
    n_exact = 64.0 * np.sqrt(Rm / 50.0)
    n = int(2 ** int(np.clip(np.round(np.log2(n_exact)), 6, 9)))
    flow = 0 if seed % 2 == 0 else 1
    return {"flow": flow, "n": n, "Rm": Rm, "kz": kz}
