"""The seeded input generators against their recipe: solenoidal, unit-norm, |k|^-2
initial spectra on the dealiased square (the random initial perturbation of Sec. 4,
with the constraint of Eq. 4c / 6c), and the parameter mix of the batched Rm / kz sweep."""
import math

import numpy as np
import pytest

import kd_inputs as I


@pytest.mark.parametrize("n,kz", [(32, 1.0), (96, 0.57), (160, 2.87)])
def test_initial_field_is_solenoidal_unit_norm_and_dealiased(n, kz):
    b = I.initial_field(n, kz, 3)
    assert b.shape == (3, n, n) and b.dtype == np.complex128
    assert abs(np.linalg.norm(b.ravel()) - 1.0) < 1e-14
    k = I.fft_wavenumbers(n)
    kx, ky = k[None, :], k[:, None]
    div = kx * b[0] + ky * b[1] + kz * b[2]
    assert np.max(np.abs(div)) < 1e-15 * max(1.0, kz) * n
    K = n // 3
    outside = (np.abs(kx) > K) | (np.abs(ky) > K)
    assert np.all(b[:, outside] == 0)
    assert np.count_nonzero(b[0]) == (2 * K + 1) ** 2


def test_initial_field_depends_on_the_seed_only():
    a = I.initial_field(64, 0.57, 11)
    assert np.array_equal(a, I.initial_field(64, 0.57, 11))
    assert not np.allclose(a, I.initial_field(64, 0.57, 12))
    batch = I.initial_batch(64, 0.57, [11, 12])
    assert np.array_equal(batch[0], a)


def test_initial_spectrum_falls_as_k_to_the_minus_four():
    # E |b_hat(k)|^2 = 2 / |k3|^4 before normalisation (a complex Gaussian of unit
    # variance per component, scaled by |k3|^-2, projected onto the plane normal to k3):
    # the log of the shell-averaged energy falls with slope -4 in log |k3|
    n, kz = 192, 0.5
    b = sum(np.abs(I.initial_field(n, kz, s)) ** 2 for s in range(8)).sum(axis=0)
    k = I.fft_wavenumbers(n)
    k3 = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2 + kz * kz)
    edges = np.geomspace(2.0, n // 3, 12)
    xs, ys = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (k3 >= lo) & (k3 < hi) & (np.abs(k[None, :]) <= n // 3) & (np.abs(k[:, None]) <= n // 3)
        ys.append(np.log(np.mean(b[m] * k3[m] ** 4)))
        xs.append(np.log(np.sqrt(lo * hi)))
    # compensated by |k3|^4 the shell means are flat
    slope = np.polyfit(xs, ys, 1)[0]
    assert abs(slope) < 0.15, slope


def test_flat_field_is_solenoidal_unit_norm_and_flat():
    # same constraints as initial_field; E |b_hat(k)|^2 = 2 before normalisation for
    # every kept k, so the edge ring of the kept square carries its share of the energy
    n, kz = 96, 0.57
    b = I.flat_field(n, kz, 5)
    assert b.shape == (3, n, n) and abs(np.linalg.norm(b.ravel()) - 1.0) < 1e-14
    k = I.fft_wavenumbers(n)
    kx, ky = k[None, :], k[:, None]
    assert np.max(np.abs(kx * b[0] + ky * b[1] + kz * b[2])) < 1e-14
    K = n // 3
    keep = (np.abs(kx) <= K) & (np.abs(ky) <= K)
    assert np.all(b[:, ~keep] == 0)
    e = sum(np.abs(I.flat_field(n, kz, s)) ** 2 for s in range(8)).sum(axis=0)
    ring = keep & ((np.abs(kx) == K) | (np.abs(ky) == K))
    inner = keep & (np.abs(kx) <= K // 2) & (np.abs(ky) <= K // 2)
    assert abs(np.mean(e[ring]) / np.mean(e[inner]) - 1.0) < 0.1
    assert not np.allclose(b, I.flat_field(n, kz, 6))


def test_sweep_instances_follow_the_recipe():
    counts = {64: 0, 128: 0, 256: 0, 512: 0}
    seeds = range(1000, 1600)
    for seed in seeds:
        q = I.sweep_instance(seed)
        assert q["flow"] == (0 if seed % 2 == 0 else 1)
        assert 50.0 <= q["Rm"] <= 3200.0 and 0.2 <= q["kz"] <= 1.5
        assert abs(math.log2(q["n"]) - math.log2(64.0 * math.sqrt(q["Rm"] / 50.0))) <= 0.5 + 1e-12
        counts[q["n"]] += 1
    # log-uniform Rm gives log2 n uniform on [6, 9]: 1/6, 1/3, 1/3, 1/6 after rounding
    frac = {n: c / len(seeds) for n, c in counts.items()}
    for n, want in ((64, 1 / 6), (128, 1 / 3), (256, 1 / 3), (512, 1 / 6)):
        assert abs(frac[n] - want) < 0.06, (n, frac)
    assert I.sweep_instance(1234) == I.sweep_instance(1234)
