"""Direct growth rate on the GPU (kd_growth_power): power iteration of the fine
propagator against the oracle's Floquet power iteration (Galloway-Proctor, Table 1) and
the leading eigenvalue of the oracle's sparse linear operator (Roberts)."""
import math

import numpy as np
import pytest

import kd_inputs as I
from oracle import kd_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kd():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_00387_gb300 as kd
    kd.load()
    torch.cuda.init()
    return kd


def test_gp_floquet_rate_matches_oracle_and_table1(kd):
    # Table 1: GP, Rm = 3, kx = 0.57 (our kz), 16 modes -> 0.15; one period = 1257 steps
    n, kz, Rm, S = 16, 0.57, 3.0, 1257
    dt = 2 * math.pi / S
    b = I.initial_field(n, kz, 1)
    p = O.Problem(O.GALLOWAY_PROCTOR, n, kz, Rm)
    g = []
    x = b.copy()
    for _ in range(6):
        nx = O.propagate(x, p, 0.0, dt, S)
        g.append(math.log(O.l2(nx) / O.l2(x)) / (2 * math.pi))
        x = nx / O.l2(nx)
    ctx = kd.kd_create(kd.make_params(O.GALLOWAY_PROCTOR, n, kz, Rm, dt, kd.KD_C128))
    try:
        out = np.zeros_like(b)
        s, rate, its = kd.kd_growth_power(ctx, b, 0.0, 2 * math.pi, 6, 0.0, out)
    finally:
        kd.kd_destroy(ctx)
    assert its == 6
    assert abs(rate - g[-1]) < 1e-11, (rate, g[-1])
    assert float("%.2g" % rate) == 0.15
    assert np.linalg.norm(out - x) < 1e-10                 # same normalised vector


def test_roberts_rate_matches_leading_eigenvalue(kd):
    import scipy.sparse.linalg as sla
    n, kz, Rm = 32, 1.0, 8.0
    w = sla.eigs(O.linear_operator(O.Problem(O.ROBERTS, n, kz, Rm)).tocsc(), k=3, sigma=0.3,
                 return_eigenvectors=False, tol=1e-13)
    gamma = max(w.real)
    ctx = kd.kd_create(kd.make_params(O.ROBERTS, n, kz, Rm, 0.01, kd.KD_C64))
    try:
        s, rate, its = kd.kd_growth_power(ctx, I.initial_field(n, kz, 3), 0.0, 2.0, 60, 1e-8)
    finally:
        kd.kd_destroy(ctx)
    assert s == kd.KD_OK, (rate, its)
    assert abs(rate - gamma) < 1e-4, (rate, gamma)          # growth-rate tolerance


def test_table1_roberts_rate_at_the_papers_resolution(kd):
    """Table 1, Roberts row: Rm = 512, kz = 2.87, N_F = 160, delta t = 1e-2 -> growth
    rate 0.11.  N_F = 160 is not a power of two, so the fine operator is the exact
    spectral convolution; the rate matches the leading eigenvalue of the oracle's sparse
    operator at the same resolution (time-step error of RK443 at delta t = 1e-2 inside the
    1e-4 tolerance) and rounds to the printed 0.11."""
    import scipy.sparse.linalg as sla
    n, kz, Rm, dt = 160, 2.87, 512.0, 1e-2
    w = sla.eigs(O.linear_operator(O.Problem(O.ROBERTS, n, kz, Rm)).tocsc(), k=3, sigma=0.15,
                 return_eigenvectors=False, tol=1e-12)
    gamma = max(w.real)
    ctx = kd.kd_create(kd.make_params(O.ROBERTS, n, kz, Rm, dt, kd.KD_C128, n_coarse=80,
                                      fine_operator=kd.KD_FINE_CONV))
    try:
        s, rate, its = kd.kd_growth_power(ctx, I.initial_field(n, kz, 5), 0.0, 10.0, 60, 1e-10)
    finally:
        kd.kd_destroy(ctx)
    assert s == kd.KD_OK, (rate, its)
    assert abs(rate - gamma) < 1e-4, (rate, gamma)
    assert float("%.2g" % rate) == 0.11


def test_gp_fp32_rate_matches_fp64(kd):
    """The FP32 propagator gives the FP64 growth rate to 1e-4 (Rm = 100, 64^2)."""
    n, kz, Rm = 64, 0.57, 100.0
    dt = 2 * math.pi / 1257
    b = I.initial_field(n, kz, 9)
    rates = []
    for prec in (kd.KD_C64, kd.KD_C128):
        ctx = kd.kd_create(kd.make_params(O.GALLOWAY_PROCTOR, n, kz, Rm, dt, prec))
        try:
            s, r, its = kd.kd_growth_power(ctx, b, 0.0, 2 * math.pi, 30, 1e-9)
            rates.append(r)
        finally:
            kd.kd_destroy(ctx)
    assert abs(rates[0] - rates[1]) < 1e-4, rates


def test_growth_argument_errors(kd):
    ctx = kd.kd_create(kd.make_params(O.ROBERTS, 16, 1.0, 8.0, 0.01, kd.KD_C64))
    try:
        b = I.initial_field(16, 1.0, 1)
        with pytest.raises(kd.KdError):
            kd.kd_growth_power(ctx, b, 0.0, 0.0, 5, 1e-6)
        with pytest.raises(kd.KdError):
            kd.kd_growth_power(ctx, b, 0.0, 1.0, 0, 1e-6)
    finally:
        kd.kd_destroy(ctx)


def test_arnoldi_finds_the_leading_spectrum_with_a_complex_pair(kd):
    """Restarted Arnoldi on the fine propagator: the 4 leading eigenvalues of the Roberts
    operator at kz = 0.3, Rm = 16 include a complex pair (-0.0321 +- 0.2788 i), where the
    power iteration cannot converge.  lambda = log(mu) / tau against the leading
    eigenvalues of the oracle's sparse operator (RK443 time error inside 1e-4)."""
    import scipy.sparse.linalg as sla
    n, kz, Rm, tau = 32, 0.3, 16.0, 10.0
    w = sla.eigs(O.linear_operator(O.Problem(O.ROBERTS, n, kz, Rm)).tocsc(), k=10, sigma=0.5,
                 return_eigenvectors=False, tol=1e-12)
    ref = sorted(w, key=lambda z: -z.real)[:4]
    ctx = kd.kd_create(kd.make_params(O.ROBERTS, n, kz, Rm, 1e-2, kd.KD_C128))
    try:
        s, mu, rate, its = kd.kd_growth_arnoldi(ctx, I.initial_field(n, kz, 11), 0.0, tau, 30, 4, 20, 1e-10)
    finally:
        kd.kd_destroy(ctx)
    assert s == kd.KD_OK, (mu, its)
    lam = np.log(mu) / tau
    assert np.all(np.diff(np.abs(mu)) <= 1e-12)                 # by decreasing modulus
    for z in ref:
        assert np.min(np.abs(lam - z)) < 1e-4, (z, lam)
    assert np.allclose(rate, lam.real, atol=1e-14)


def test_arnoldi_equals_power_iteration_on_a_real_leading_mode(kd):
    """Same discrete propagator, two methods: Roberts kz = 1, Rm = 8 (real leading
    eigenvalue) and the GP Floquet multiplier of Table 1 (Rm = 3, one period)."""
    for flow, n, kz, Rm, dt, tau in [(O.ROBERTS, 32, 1.0, 8.0, 0.01, 2.0),
                                     (O.GALLOWAY_PROCTOR, 16, 0.57, 3.0, 2 * math.pi / 1257, 2 * math.pi)]:
        b = I.initial_field(n, kz, 4)
        ctx = kd.kd_create(kd.make_params(flow, n, kz, Rm, dt, kd.KD_C128))
        try:
            s1, r_pow, _ = kd.kd_growth_power(ctx, b, 0.0, tau, 400, 1e-13)
            s2, mu, rate, its = kd.kd_growth_arnoldi(ctx, b, 0.0, tau, 20, 1, 10, 1e-12)
        finally:
            kd.kd_destroy(ctx)
        assert s2 == kd.KD_OK
        assert abs(rate[0] - r_pow) < 1e-9, (flow, rate[0], r_pow)
        if flow == O.GALLOWAY_PROCTOR:
            assert float("%.2g" % rate[0]) == 0.15


def test_arnoldi_table1_roberts_at_nf160_with_the_convolution_operator(kd):
    import scipy.sparse.linalg as sla
    n, kz, Rm = 160, 2.87, 512.0
    w = sla.eigs(O.linear_operator(O.Problem(O.ROBERTS, n, kz, Rm)).tocsc(), k=3, sigma=0.15,
                 return_eigenvectors=False, tol=1e-12)
    gamma = max(w.real)
    ctx = kd.kd_create(kd.make_params(O.ROBERTS, n, kz, Rm, 1e-2, kd.KD_C128, n_coarse=80,
                                      fine_operator=kd.KD_FINE_CONV))
    try:
        out = np.zeros((3, n, n), np.complex128)
        s, mu, rate, its = kd.kd_growth_arnoldi(ctx, I.initial_field(n, kz, 6), 0.0, 5.0, 16, 1, 10, 1e-9, out)
    finally:
        kd.kd_destroy(ctx)
    assert s == kd.KD_OK
    assert abs(rate[0] - gamma) < 1e-4 and float("%.2g" % rate[0]) == 0.11
    assert abs(np.linalg.norm(out) - 1.0) < 1e-9               # orthonormal basis to round-off


def test_arnoldi_argument_errors(kd):
    ctx = kd.kd_create(kd.make_params(O.ROBERTS, 16, 1.0, 8.0, 0.01, kd.KD_C64))
    try:
        b = I.initial_field(16, 1.0, 1)
        for args in [(0.0, 0.0, 10, 1, 2, 1e-6), (0.0, 1.0, 1, 1, 2, 1e-6), (0.0, 1.0, 10, 10, 2, 1e-6),
                     (0.0, 1.0, 65, 1, 2, 1e-6), (0.0, 1.0, 10, 1, 0, 1e-6)]:
            with pytest.raises(kd.KdError):
                kd.kd_growth_arnoldi(ctx, b, *args)
    finally:
        kd.kd_destroy(ctx)
