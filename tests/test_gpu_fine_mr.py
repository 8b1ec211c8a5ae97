"""Parity of the mixed-radix FFT fine kernels (grid sides n = 32 R: 96, 160, 192; Table 1's
N_F = 160), and of the other even sides that run on the next alias-free transform side,
with the CPU FP64 oracle, through the C ABI.  The oracle's transforms are
numpy's FFTs of the same length, so an error anywhere in the radix-R / radix-2 warp
transform, its twiddles or its bit-reversed lane order shows up against it."""
import numpy as np
import pytest

import kd_inputs as I
from oracle import kd_oracle as O

pytestmark = pytest.mark.gpu

TOL32 = 1e-5      # relative L2 per field state, complex64 (as for the other grids)
TOL64 = 1e-12


@pytest.fixture(scope="module")
def kd():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_00387_gb300 as kd
    kd.load()
    torch.cuda.init()
    return kd


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def run_fine(kd, params, b, t0, nsteps):
    import torch
    prec = params.prec_fine
    ctx = kd.kd_create(params)
    try:
        dtype = torch.complex128 if prec == kd.KD_C128 else torch.complex64
        x = torch.tensor(b, dtype=dtype, device="cuda")
        y = torch.empty_like(x)
        tt = torch.tensor(np.asarray(t0, np.float64), device="cuda")
        kd.kd_fine_batched(ctx, x, y, tt, nsteps, b.shape[0], prec)
        torch.cuda.synchronize()
        return y.cpu().numpy().astype(np.complex128)
    finally:
        kd.kd_destroy(ctx)


@pytest.mark.parametrize("n", [96, 160, 192])
@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("flow", [O.ROBERTS, O.GALLOWAY_PROCTOR])
def test_mixed_radix_fine_matches_oracle(kd, n, prec, flow):
    """Five fields (a ragged last block of 4 warps) with their own start times."""
    P = kd.KD_C64 if prec == "c64" else kd.KD_C128
    kz, Rm, dt = 0.57, 100.0, 5e-3
    b = I.initial_batch(n, kz, [31, 32, 33, 34, 35])
    t0 = [0.0, 0.3, 1.1, 2.2, 5.0]
    out = run_fine(kd, kd.make_params(flow, n, kz, Rm, dt, P), b, t0, 4)
    p = O.Problem(flow, n, kz, Rm)
    for i in range(len(t0)):
        assert rel(out[i], O.propagate(b[i], p, t0[i], dt, 4)) < (TOL32 if P == kd.KD_C64 else TOL64), i


@pytest.mark.parametrize("n,m", [(18, 96), (120, 96), (200, 160), (240, 192), (286, 192)])
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_other_even_sides_on_the_next_alias_free_transform(kd, n, m, prec):
    """A side n with no kernels of its own runs on the smallest mixed-radix side m >= 2 (n/3) + 2
    (fine_fft_grid): the oracle steps on the n-point grid itself, so equality pins that
    u x b (wavenumbers +-1 times |k| <= n/3) is alias-free on the kept set on both grids.
    n = 240 is the 3/2-padded grid of 160 kept modes a side."""
    P = kd.KD_C64 if prec == "c64" else kd.KD_C128
    assert m >= 2 * (n // 3) + 2
    kz, Rm, dt = 0.57, 100.0, 5e-3
    b = I.initial_batch(n, kz, [91, 92])
    t0 = [0.0, 1.3]
    out = run_fine(kd, kd.make_params(O.GALLOWAY_PROCTOR, n, kz, Rm, dt, P), b, t0, 4)
    p = O.Problem(O.GALLOWAY_PROCTOR, n, kz, Rm)
    for i in range(2):
        assert rel(out[i], O.propagate(b[i], p, t0[i], dt, 4)) < (TOL32 if P == kd.KD_C64 else TOL64), i


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_table1_roberts_row_with_160_kept_modes(kd, prec):
    """The other reading of Table 1's N_F = 160: 160 kept modes a side on a 3/2-padded grid
    of 240 points (kept |k| <= 80), run on the 192-point transform; against the oracle's
    240-point steps, 20 steps at delta t = 1e-2."""
    P = kd.KD_C64 if prec == "c64" else kd.KD_C128
    n, kz, Rm, dt = 240, 2.87, 512.0, 1e-2
    b = I.initial_batch(n, kz, [95])
    out = run_fine(kd, kd.make_params(O.ROBERTS, n, kz, Rm, dt, P), b, [0.5], 20)
    ref = O.propagate(b[0], O.Problem(O.ROBERTS, n, kz, Rm), 0.5, dt, 20)
    assert rel(out[0], ref) < (TOL32 if P == kd.KD_C64 else 1e-11)


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_table1_roberts_fine_slice_at_nf160(kd, prec):
    """Table 1's Roberts row on the FFT path: Rm = 512, kz = 2.87, N_F = 160,
    delta t = 1e-2, 50 steps (half a unit of time) from two start times."""
    P = kd.KD_C64 if prec == "c64" else kd.KD_C128
    n, kz, Rm, dt = 160, 2.87, 512.0, 1e-2
    b = I.initial_batch(n, kz, [51, 52])
    t0 = [0.0, 3.0]
    out = run_fine(kd, kd.make_params(O.ROBERTS, n, kz, Rm, dt, P), b, t0, 50)
    p = O.Problem(O.ROBERTS, n, kz, Rm)
    for i in range(2):
        assert rel(out[i], O.propagate(b[i], p, t0[i], dt, 50)) < (TOL32 if P == kd.KD_C64 else 1e-11), i


def test_flat_spectrum_edge_ring_nf160(kd):
    """A flat-spectrum divergence-free input puts as much weight on the edge ring
    |kx| = K or |ky| = K as on the low modes; its max-abs error there stays at the
    complex64 bound."""
    n, kz, Rm, dt, S = 160, 2.87, 512.0, 1e-2, 10
    b = I.flat_field(n, kz, 7)[None]
    out = run_fine(kd, kd.make_params(O.ROBERTS, n, kz, Rm, dt, kd.KD_C64), b, [0.7], S)[0]
    ref = O.propagate(b[0], O.Problem(O.ROBERTS, n, kz, Rm), 0.7, dt, S)
    K = n // 3
    k = np.fft.fftfreq(n, 1.0 / n).astype(int)
    ring = ((np.abs(k)[None, :] == K) & (np.abs(k)[:, None] <= K)) | \
           ((np.abs(k)[:, None] == K) & (np.abs(k)[None, :] <= K))
    scale = np.abs(ref).max()
    assert np.abs(out[:, ring] - ref[:, ring]).max() < 2e-6 * scale
    assert rel(out, ref) < TOL32


@pytest.mark.parametrize("scheme", ["RK222", "RK111"])
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_lower_order_schemes_at_nf160(kd, scheme, prec):
    P = kd.KD_C64 if prec == "c64" else kd.KD_C128
    sch = {"RK222": kd.KD_RK222, "RK111": kd.KD_RK111}[scheme]
    tab = {"RK222": O.RK222, "RK111": O.RK111}[scheme]
    n, kz, Rm, dt = 160, 0.57, 100.0, 2e-3
    b = I.initial_batch(n, kz, [61, 62, 63])
    t0 = [0.0, 0.9, 1.6]
    out = run_fine(kd, kd.make_params(O.GALLOWAY_PROCTOR, n, kz, Rm, dt, P, fine_scheme=sch), b, t0, 5)
    p = O.Problem(O.GALLOWAY_PROCTOR, n, kz, Rm)
    for i in range(3):
        assert rel(out[i], O.propagate(b[i], p, t0[i], dt, 5, tab=tab)) < (TOL32 if P == kd.KD_C64 else TOL64), i


def test_fft_and_convolution_operators_agree_at_nf160(kd):
    """The two fine operators compute the same discrete operator (the flow has only the
    wavenumbers +-1, so the grid product of the FFT route is alias-free on the kept set);
    in complex128 they agree to round-off over a 20-step slice."""
    n, kz, Rm, dt = 160, 2.87, 512.0, 1e-2
    b = I.initial_batch(n, kz, [71])
    outs = [run_fine(kd, kd.make_params(O.ROBERTS, n, kz, Rm, dt, kd.KD_C128, fine_operator=op), b, [0.4], 20)
            for op in (kd.KD_FINE_FFT, kd.KD_FINE_CONV)]
    assert rel(outs[0][0], outs[1][0]) < 1e-13


def test_static_entry_on_the_mixed_radix_grid(kd):
    """kd_fine_batched_static takes the same kernels at n = 160."""
    import torch
    n, kz, Rm, dt = 160, 2.87, 512.0, 1e-2
    p = kd.make_params(O.ROBERTS, n, kz, Rm, dt, kd.KD_C64)
    b = I.initial_batch(n, kz, [81, 82])
    x = torch.tensor(b, dtype=torch.complex64, device="cuda")
    y = torch.full_like(x, float("nan"))
    tt = torch.tensor([0.0, 1.0], dtype=torch.float64, device="cuda")
    assert kd.kd_fine_batched_static(p, x, y, tt, 6, 2) == kd.KD_OK
    torch.cuda.synchronize()
    out = y.cpu().numpy().astype(np.complex128)
    prob = O.Problem(O.ROBERTS, n, kz, Rm)
    for i, t in enumerate((0.0, 1.0)):
        assert rel(out[i], O.propagate(b[i], prob, t, dt, 6)) < TOL32, i


def test_table1_roberts_parareal_on_the_fft_path(kd):
    """Parareal on Table 1's Roberts grids (N_F = 160 on the mixed-radix FFT, N_C = 80
    on the cluster solver), FP64, iterates equal to the oracle's Parareal."""
    import math
    n, nc, kz, Rm, T, N, kmax = 160, 80, 2.87, 512.0, 0.8, 4, 2
    b0 = I.initial_field(n, kz, 23)
    p = kd.make_params(O.ROBERTS, n, kz, Rm, 1e-2, kd.KD_C128, n_coarse=nc, dt_coarse=2e-2,
                       prec_coarse=kd.KD_C128, fine_operator=kd.KD_FINE_FFT)
    ctx = kd.kd_create(p)
    try:
        out = np.zeros((N + 1, 3, n, n), np.complex128)
        status, st = kd.kd_parareal_run(ctx, b0, T, N, kmax, 0.0, out)
    finally:
        kd.kd_destroy(ctx)
    assert status == kd.KD_ENOTCONV and st.k_con == kmax
    prob = O.Problem(O.ROBERTS, n, kz, Rm)
    dT = T / N
    S, Sc = math.ceil(dT / 1e-2 - 1e-9), math.ceil(dT / 2e-2 - 1e-9)
    assert (st.n_fine_steps, st.n_coarse_steps) == (S, Sc) == (20, 10)
    fine = lambda u, i: O.propagate(u, prob, i * dT, dT / S, S)
    coarse = lambda u, i: O.coarse_propagate(u, prob, nc, i * dT, dT / Sc, Sc)
    ref = O.parareal(b0, fine, coarse, N, kmax, 0.0)
    for i in range(N + 1):
        assert rel(out[i], ref["U"][i]) < 1e-11, i
    for k in range(kmax):
        assert abs(st.sigma[k] - ref["sigma"][k]) <= 1e-8 * ref["sigma"][k]


def test_table1_roberts_growth_rate_on_the_fft_path(kd):
    """Table 1, Roberts row: the growth rate 0.11 at N_F = 160 from the FFT fine operator,
    equal to the leading eigenvalue of the oracle's operator within 1e-4."""
    import scipy.sparse.linalg as sla
    n, kz, Rm, dt = 160, 2.87, 512.0, 1e-2
    w = sla.eigs(O.linear_operator(O.Problem(O.ROBERTS, n, kz, Rm)).tocsc(), k=3, sigma=0.15,
                 return_eigenvectors=False, tol=1e-12)
    gamma = max(w.real)
    ctx = kd.kd_create(kd.make_params(O.ROBERTS, n, kz, Rm, dt, kd.KD_C128, n_coarse=80))
    try:
        s, rate, its = kd.kd_growth_power(ctx, I.initial_field(n, kz, 5), 0.0, 10.0, 60, 1e-10)
    finally:
        kd.kd_destroy(ctx)
    assert s == kd.KD_OK, (rate, its)
    assert abs(rate - gamma) < 1e-4, (rate, gamma)
    assert float("%.2g" % rate) == 0.11


@pytest.mark.parametrize("n", [32, 64, 128, 256])
def test_mixed_radix_plan_on_power_of_two_sides(kd, n):
    """The warp-owned kernels as a launch-plan variant of the complex64 sides 32 R (R = 1,
    2, 4, 8: the in-lane transform is radix 2, the cross-lane one unchanged), against the
    oracle, RK443 and RK222."""
    import torch
    P = kd.KD_C64
    kz, Rm, dt = 0.57, 100.0, 5e-3
    b = I.initial_batch(n, kz, [41, 42, 43])
    t0 = [0.0, 0.7, 2.4]
    for sch, tab in ((kd.KD_RK443, O.RK443), (kd.KD_RK222, O.RK222)):
        ctx = kd.kd_create(kd.make_params(O.GALLOWAY_PROCTOR, n, kz, Rm, dt, P, fine_scheme=sch))
        try:
            ncol, nrow = kd.kd_plan_variants(ctx, kd.KD_GRID_FINE)
            mr = 5 if n == 128 else (3 if n <= 64 else 4)          # the mixed-radix variant's index
            kd.kd_set_plan(ctx, kd.KD_GRID_FINE, mr, 8 if n >= 128 else 6)
            dtype = torch.complex128 if P == kd.KD_C128 else torch.complex64
            x = torch.tensor(b, dtype=dtype, device="cuda")
            y = torch.empty_like(x)
            kd.kd_fine_batched(ctx, x, y, torch.tensor(t0, dtype=torch.float64, device="cuda"), 3, 3, P)
            torch.cuda.synchronize()
            out = y.cpu().numpy().astype(np.complex128)
        finally:
            kd.kd_destroy(ctx)
        p = O.Problem(O.GALLOWAY_PROCTOR, n, kz, Rm)
        for i in range(3):
            assert rel(out[i], O.propagate(b[i], p, t0[i], dt, 3, tab=tab)) < (TOL32 if P == kd.KD_C64 else TOL64), i
