"""Pins of the CPU FP64 oracle against facts that do not come from the oracle itself:
closed forms, the paper's printed component equations, textbook properties of the
IMEX schemes, Parareal's finite termination and the growth rates of Table 1."""
import math
import os

import numpy as np
import pytest

import kd_inputs as I
from oracle import kd_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return float(np.sqrt(np.sum(np.abs(a - b) ** 2)) / max(np.sqrt(np.sum(np.abs(b) ** 2)), 1e-300))


# ------------------------------------------------------------------ transforms
def test_transform_convention_single_mode():
    n = 16
    x = O.grid_points(n)
    for kx, ky in [(0, 0), (3, -2), (-5, 5), (1, 4)]:
        bh = np.zeros((n, n), complex)
        bh[ky % n, kx % n] = 1.0
        expect = np.exp(1j * (kx * x[None, :] + ky * x[:, None]))
        assert np.abs(O.to_physical(bh) - expect).max() < 1e-13
        assert np.abs(O.to_spectral(expect) - bh).max() < 1e-13


def test_transform_against_naive_dft():
    n = 8
    rng = np.random.default_rng(1)
    b = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    x = O.grid_points(n)
    k = I.fft_wavenumbers(n)
    naive = np.zeros((n, n), complex)
    for iy in range(n):
        for ix in range(n):
            naive[iy, ix] = np.sum(b * np.exp(-1j * (k[ix] * x[None, :] + k[iy] * x[:, None]))) / n ** 2
    assert np.abs(O.to_spectral(b) - naive).max() < 1e-14
    # Parseval in this normalisation: sum |b|^2 = n^2 sum |b_hat|^2
    assert abs(np.sum(np.abs(b) ** 2) - n * n * np.sum(np.abs(naive) ** 2)) < 1e-10


@pytest.mark.parametrize("flow", [O.ROBERTS, O.GALLOWAY_PROCTOR])
def test_velocity_modes_match_grid_flow(flow):
    n = 16
    t = 0.731
    uh = O.to_spectral(O.velocity(flow, n, t).astype(complex))
    expect = np.zeros_like(uh)
    for (qx, qy), v in O.velocity_modes(flow, t).items():
        expect[:, qy % n, qx % n] = v
    assert np.abs(uh - expect).max() < 1e-14


def test_roberts_flow_matches_abc_form():
    # Sec. 2.1: A = B = 1, C = 0 in the ABC flow gives u = (cos y, sin x, sin y + cos x)
    n = 12
    x = O.grid_points(n)[None, :]
    y = O.grid_points(n)[:, None]
    u = O.velocity(O.ROBERTS, n, 0.0)
    assert np.abs(u[0] - np.cos(y)).max() < 1e-15
    assert np.abs(u[1] - np.sin(x)).max() < 1e-15
    assert np.abs(u[2] - (np.sin(y) + np.cos(x))).max() < 1e-15


def test_gp_flow_is_relabelled_paper_flow():
    # Sec. 2.2 in the paper's coordinates (invariant x, plane (y, z)), C = B = sqrt(3/2):
    # u = (C sin(z + sin t) + B cos(y + cos t), C cos(z + sin t), B sin(y + cos t)).
    # Relabelling (paper y, z, x) -> (x, y, z) must give our velocity field.
    n, t = 12, 1.3
    C = B = math.sqrt(1.5)
    X = O.grid_points(n)[None, :]
    Y = O.grid_points(n)[:, None]
    py, pz = X, Y           # paper's y and z at our grid point (x=X, y=Y)
    paper_ux = C * np.sin(pz + np.sin(t)) + B * np.cos(py + np.cos(t))
    paper_uy = C * np.cos(pz + np.sin(t)) + 0 * py
    paper_uz = B * np.sin(py + np.cos(t)) + 0 * pz
    u = O.velocity(O.GALLOWAY_PROCTOR, n, t)
    assert np.abs(u[0] - paper_uy).max() < 1e-14
    assert np.abs(u[1] - paper_uz).max() < 1e-14
    assert np.abs(u[2] - paper_ux).max() < 1e-14


# ------------------------------------------------------------------------ RHS
@pytest.mark.parametrize("flow", [O.ROBERTS, O.GALLOWAY_PROCTOR])
@pytest.mark.parametrize("n", [16, 32, 48])
def test_rhs_fft_equals_convolution(flow, n):
    p = O.Problem(flow, n, 0.57, 50.0)
    b = I.initial_field(n, 0.57, 5)
    for t in (0.0, 0.4, 2.9):
        a = O.rhs_fft(b, p, t)
        c = O.rhs_conv(b, p, t)
        assert rel(a, c) < 1e-13


def test_rhs_closed_form_uniform_field():
    # Roberts flow, b = e_x (the k = 0 mode): u x b = (0, u_z, -u_y) and
    # nabla_k x (u x b) = (-i kz (cos x + sin y), cos x, -sin x).
    n, kz = 16, 1.7
    p = O.Problem(O.ROBERTS, n, kz, 10.0)
    bh = np.zeros((3, n, n), complex)
    bh[0, 0, 0] = 1.0
    F = O.to_physical(O.rhs_fft(bh, p, 0.0))
    x = O.grid_points(n)[None, :]
    y = O.grid_points(n)[:, None]
    assert np.abs(F[0] - (-1j * kz * (np.cos(x) + np.sin(y)))).max() < 1e-13
    assert np.abs(F[1] - np.cos(x) * np.ones_like(y)).max() < 1e-13
    assert np.abs(F[2] - (-np.sin(x)) * np.ones_like(y)).max() < 1e-13


def test_rhs_solenoidal_and_zero_without_flow():
    n = 32
    b = I.initial_field(n, 0.9, 2)
    p = O.Problem(O.GALLOWAY_PROCTOR, n, 0.9, 30.0)
    F = O.rhs_fft(b, p, 1.1)
    assert np.abs(O.divergence_k(F, 0.9)).max() < 1e-15 * n * n
    assert np.abs(O.rhs_fft(b, O.Problem(O.NO_FLOW, n, 0.9, 30.0), 0.0)).max() == 0.0


def _deriv(b, axis_k):
    return O.to_physical(1j * axis_k * O.to_spectral(b))


def test_roberts_advective_equations_match_curl_form():
    # Eqs. 4a-4b (Sec. 2.1) hold for divergence-free b.
    n, kz = 32, 2.87
    p = O.Problem(O.ROBERTS, n, kz, 512.0)
    bh = I.initial_field(n, kz, 7)
    kx, ky, _ = O.wavevector(n, kz)
    bx, by = O.to_physical(bh[0]), O.to_physical(bh[1])
    x = O.grid_points(n)[None, :]
    y = O.grid_points(n)[:, None]
    dxb = lambda f: _deriv(f, kx)
    dyb = lambda f: _deriv(f, ky)
    adv_x = -by * np.sin(y) - np.cos(y) * dxb(bx) - np.sin(x) * dyb(bx) - (np.sin(y) + np.cos(x)) * 1j * kz * bx
    adv_y = bx * np.cos(x) - np.cos(y) * dxb(by) - np.sin(x) * dyb(by) - (np.sin(y) + np.cos(x)) * 1j * kz * by
    mask = O.kept_mask(n)
    F = O.rhs_fft(bh, p, 0.0)
    assert rel(O.to_spectral(adv_x) * mask, F[0]) < 1e-12
    assert rel(O.to_spectral(adv_y) * mask, F[1]) < 1e-12


def test_gp_advective_equations_match_curl_form():
    # Eqs. 6a-6b (Sec. 2.2) after relabelling (paper y, z, x) -> (x, y, z), so that
    # paper (b_y, b_z) = our (b_x, b_y), paper (u, v, w) = our (u_z, u_x, u_y) and the
    # paper's kx is our kz.  (The diffusion of Eq. 6a is printed with kz^2; with
    # b ~ exp(i kx x) it is kx^2, as in Eq. 6b; diffusion is not part of this check.)
    n, kz, t = 32, 0.57, 0.83
    p = O.Problem(O.GALLOWAY_PROCTOR, n, kz, 300.0)
    bh = I.initial_field(n, kz, 8)
    kx, ky, _ = O.wavevector(n, kz)
    u = O.velocity(O.GALLOWAY_PROCTOR, n, t)
    pu, pv, pw = u[2], u[0], u[1]
    by_, bz_ = O.to_physical(bh[0]), O.to_physical(bh[1])
    d_py = lambda f: _deriv(f, kx)     # paper d/dy = our d/dx
    d_pz = lambda f: _deriv(f, ky)     # paper d/dz = our d/dy
    rhs_by = bz_ * d_pz(pv.astype(complex)) - pu * 1j * kz * by_ - pv * d_py(by_) - pw * d_pz(by_)
    rhs_bz = by_ * d_py(pw.astype(complex)) - pu * 1j * kz * bz_ - pv * d_py(bz_) - pw * d_pz(bz_)
    mask = O.kept_mask(n)
    F = O.rhs_fft(bh, p, t)
    assert rel(O.to_spectral(rhs_by) * mask, F[0]) < 1e-12
    assert rel(O.to_spectral(rhs_bz) * mask, F[1]) < 1e-12


# ---------------------------------------------------------------- timesteppers
@pytest.mark.parametrize("tab", [O.RK111, O.RK222, O.RK443])
def test_tableau_row_sums(tab):
    c, A, H = tab["c"], tab["A"], tab["H"]
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)
    assert np.allclose(H.sum(axis=1), c, atol=1e-15)
    assert np.allclose(np.triu(H), 0.0)            # explicit part strictly lower
    assert np.allclose(np.triu(A, 1), 0.0)         # diagonally implicit
    assert np.allclose(A[:, 0], 0.0)


def _stability_function(tab, z):
    # R(z) = e_s^T (I - z A)^-1 e_0 for the implicit tableau with explicit first stage;
    # the stage vector solves X = X0 1 + z A X.
    A = tab["A"]
    m = A.shape[0]
    X = np.linalg.solve(np.eye(m) - z * A, np.ones(m))
    return X[-1]


def test_pure_diffusion_exact_stability_function():
    # u = 0: every mode decays by exactly R(-lambda dt) per step.
    n, kz, Rm, dt, S = 16, 1.3, 7.0, 0.05, 40
    p = O.Problem(O.NO_FLOW, n, kz, Rm)
    b = I.initial_field(n, kz, 3)
    out = O.propagate(b, p, 0.0, dt, S)
    lam = O.diffusion_rate(p)
    R = np.vectorize(lambda l: _stability_function(O.RK443, -l * dt))(lam)
    assert rel(out, b * R ** S) < 1e-13


def test_pure_diffusion_decay_order_three():
    # u = 0: b_hat(t) = exp(-(|k|^2 + kz^2) t / Rm) b_hat(0); RK443 error drops ~8x per halving.
    n, kz, Rm, T = 16, 1.0, 2.0, 1.0
    p = O.Problem(O.NO_FLOW, n, kz, Rm)
    b = I.initial_field(n, kz, 4)
    exact = b * np.exp(-O.diffusion_rate(p) * T)
    errs = []
    for S in (20, 40, 80):
        errs.append(rel(O.propagate(b, p, 0.0, T / S, S), exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 6.5 < r1 < 10.0 and 6.5 < r2 < 10.0, errs


@pytest.mark.parametrize("tab,order", [(O.RK111, 1), (O.RK222, 2), (O.RK443, 3)])
def test_imex_order_on_forced_scalar_problem(tab, order):
    # y' = (i w) y + sin t  (explicit)  - lam y  (implicit), exact solution in closed form.
    lam, w, y0, T = 1.5, 2.0, 1.0 + 0.5j, 1.0
    a = -lam + 1j * w
    beta = -1.0 / (1.0 + a * a)
    alpha = -a / (1.0 + a * a)
    exact = np.exp(a * T) * (y0 - beta) + alpha * np.sin(T) + beta * np.cos(T)
    errs = []
    for S in (40, 80, 160):
        y = np.array(y0)
        dt = T / S
        for s in range(S):
            y = O.imex_step(y, s * dt, dt, lambda v, t: 1j * w * v + np.sin(t), lam, tab)
        errs.append(abs(y - exact))
    rate = math.log2(errs[1] / errs[2])
    assert abs(rate - order) < 0.25, (errs, rate)


def test_fine_propagator_linear():
    n, kz = 32, 0.57
    p = O.Problem(O.GALLOWAY_PROCTOR, n, kz, 100.0)
    a = I.initial_field(n, kz, 1)
    b = I.initial_field(n, kz, 2)
    al, be = 0.3 - 1.1j, -2.0 + 0.25j
    fa = O.propagate(a, p, 0.4, 5e-3, 25)
    fb = O.propagate(b, p, 0.4, 5e-3, 25)
    fab = O.propagate(al * a + be * b, p, 0.4, 5e-3, 25)
    assert rel(fab, al * fa + be * fb) < 1e-13


@pytest.mark.parametrize("flow", [O.ROBERTS, O.GALLOWAY_PROCTOR])
def test_fine_propagator_keeps_divergence_free(flow):
    n, kz = 32, 0.8
    p = O.Problem(flow, n, kz, 60.0)
    b = I.initial_field(n, kz, 9)
    out = O.propagate(b, p, 0.0, 1e-2, 100)
    k3 = np.sqrt(O.diffusion_rate(p) * p.Rm)
    assert np.abs(O.divergence_k(out, kz)).max() / (k3 * np.abs(out)).max() < 1e-13
    assert np.abs(out[:, ~O.kept_mask(n)]).max() == 0.0


# ---------------------------------------------------- restriction / prolongation
def test_restrict_prolong_are_fourier_resampling():
    n, nc = 32, 16
    b = I.initial_field(n, 1.0, 11)
    bc = O.restrict(b, nc)
    assert np.abs(O.restrict(O.prolong(bc, n), nc) - bc).max() == 0.0
    # a field supported on the coarse set survives the round trip unchanged
    low = O.prolong(bc, n)
    assert np.abs(O.prolong(O.restrict(low, nc), n) - low).max() == 0.0
    # the same function values at the shared grid points (coarse points = every 2nd fine point)
    assert np.abs(O.to_physical(low)[:, ::2, ::2] - O.to_physical(bc)).max() < 1e-13


# --------------------------------------------------------------------- parareal
def _small_parareal_problem():
    p = O.Problem(O.ROBERTS, 16, 1.0, 8.0)
    N, S, dt = 6, 10, 0.02
    Sc, dtc = 2, 0.1
    fine = lambda u, n: O.propagate(u, p, n * S * dt, dt, S)
    coarse = lambda u, n: O.coarse_propagate(u, p, 8, n * S * dt, dtc, Sc)
    return p, N, fine, coarse


def test_parareal_finite_termination_bitwise():
    p, N, fine, coarse = _small_parareal_problem()
    u0 = I.initial_field(16, 1.0, 0)
    ref = O.serial_fine(u0, fine, N)
    res = O.parareal(u0, fine, coarse, N, N, 0.0, keep_iterates=True)
    assert len(res["iterates"]) == N + 1
    for k, Uk in enumerate(res["iterates"]):
        for n in range(k + 1):            # slices 0..k are exact after k iterations
            assert np.array_equal(Uk[n], ref[n]), (k, n)
    for n in range(N + 1):
        assert np.array_equal(res["U"][n], ref[n])


def test_parareal_with_fine_as_coarse_converges_in_one_iteration():
    p, N, fine, _ = _small_parareal_problem()
    u0 = I.initial_field(16, 1.0, 1)
    res = O.parareal(u0, fine, fine, N, N, 1e-14)
    assert res["k_con"] == 1 and res["sigma"][0] == 0.0


def test_parareal_defect_decreases():
    p, N, fine, coarse = _small_parareal_problem()
    u0 = I.initial_field(16, 1.0, 2)
    res = O.parareal(u0, fine, coarse, N, N, 0.0)
    s = res["sigma"]
    assert len(s) == N
    # sigma_k is the change of the last slice; it shrinks as slices become exact
    assert s[1] < s[0] and s[2] < s[1] and s[-1] < s[0]
    ref = O.serial_fine(u0, fine, N)
    assert np.array_equal(res["U"][N], ref[N])


def test_speedup_model_and_bounds():
    # Eq. 10 and its bound Eq. 11: s <= min(N_p / k, R_f / R_c); efficiency <= 1 / k.
    for N, k, r in [(10, 3, 0.01), (64, 3, 0.05), (1600, 3, 1e-4), (8, 2, 0.2)]:
        s = O.speedup_model(k, N, r)
        assert s <= min(N / k, 1.0 / r) + 1e-12
        assert s / N <= 1.0 / k + 1e-12
    assert abs(O.speedup_model(3, 10, 0.0) - 10 / 3) < 1e-12


def test_speedup_model_hand_values():
    # Eq. 10 evaluated by hand in fractions, with a coarse/fine cost ratio that is not 0:
    #   k = 3, N_p = 16, R_c/R_f = 1/16: (1 + 3/16)(1/16) + 3/16 = 19/256 + 48/256 = 67/256
    #   k = 2, N_p = 64, R_c/R_f = 1/4:  (1 + 2/64)(1/4) + 2/64 = 33/128 + 4/128 = 37/128
    # (dropping the (1 + k/N_p) factor would give 4 and 128/36 instead)
    assert abs(O.speedup_model(3, 16, 1.0 / 16) - 256.0 / 67.0) < 1e-14
    assert abs(O.speedup_model(2, 64, 0.25) - 128.0 / 37.0) < 1e-14


@pytest.mark.parametrize("flow", [O.GALLOWAY_PROCTOR, O.ROBERTS])
def test_coarse_propagator_is_the_fine_one_on_the_coarse_mode_set(flow):
    # G of Sec. 3.2 restricts to the N_C grid and steps the same equations there.  On the
    # same grid and step it is F itself; on a smaller grid it equals F on the fine grid
    # with the state and the explicit term kept on the coarse square (no aliasing: the
    # flow has |q| = 1 modes only).  The slice start time t0 != 0 enters both through the
    # time-dependent GP flow.
    n, n_c, kz, Rm = 48, 24, 0.57, 30.0
    prob = O.Problem(flow, n, kz, Rm)
    b = I.initial_field(n, kz, 4)
    t0, dt, S = 1.3, 0.02, 12
    assert np.array_equal(O.coarse_propagate(b, prob, n, t0, dt, S), O.propagate(b, prob, t0, dt, S))
    k = I.fft_wavenumbers(n)
    Kc = n_c // 3
    mask = (np.abs(k[None, :]) <= Kc) & (np.abs(k[:, None]) <= Kc)
    ref = O.propagate(b, prob, t0, dt, S, mask=mask)
    got = O.coarse_propagate(b, prob, n_c, t0, dt, S)
    assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref)
    if flow == O.GALLOWAY_PROCTOR:
        later = O.coarse_propagate(b, prob, n_c, t0 + 0.5, dt, S)
        assert np.linalg.norm(later - got) > 1e-4 * np.linalg.norm(got)


# ------------------------------------------------------------------ growth rates
def test_growth_fit_exact_exponential():
    t = np.linspace(0, 10, 21)
    E = 3.0 * np.exp(2 * 0.137 * t)
    assert abs(O.growth_rate(t, E, 5.0) - 0.137) < 1e-14


def test_roberts_growth_rate_eigenvalue_equals_time_fit():
    # Steady flow: the leading eigenvalue of the truncated spectral operator (built from
    # the convolution form) equals the late-time slope of (1/2) ln E of the FFT-based
    # time integration (Sec. 1: steady u gives an eigenvalue problem).
    import scipy.sparse.linalg as sla
    p = O.Problem(O.ROBERTS, 32, 1.0, 8.0)
    w = sla.eigs(O.linear_operator(p).tocsc(), k=3, sigma=0.3, return_eigenvectors=False, tol=1e-13)
    gamma_eig = max(w.real)
    b = I.initial_field(32, 1.0, 0)
    ts, Es = [0.0], [O.energy(b)]
    for i in range(40):
        b = O.propagate(b, p, i * 1.0, 0.02, 50)
        ts.append(i + 1.0)
        Es.append(O.energy(b))
    gamma_fit = O.growth_rate(ts, Es, 25.0)
    assert abs(gamma_fit - gamma_eig) < 2e-4, (gamma_fit, gamma_eig)


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_growth_rates.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = line.split()
                rows.append({"flow": v[0], "Rm": float(v[1]), "k": float(v[2]), "rate": float(v[7])})
    return rows


def _round2(x):
    return float(f"{x:.2g}")


@pytest.mark.slow
def test_table1_roberts_growth_rate_and_refinement():
    import scipy.sparse.linalg as sla
    row = [r for r in _table1() if r["flow"] == "roberts" and r["Rm"] == 512][0]
    gam = []
    # up to the paper's own N_F = 160
    for n in (96, 128, 160):
        L = O.linear_operator(O.Problem(O.ROBERTS, n, row["k"], row["Rm"])).tocsc()
        w = sla.eigs(L, k=3, sigma=0.3, return_eigenvectors=False, tol=1e-12)
        gam.append(max(w.real))
    assert _round2(gam[-1]) == row["rate"], gam
    # converging under refinement
    assert abs(gam[2] - gam[1]) < 0.25 * abs(gam[1] - gam[0]), gam


def test_table1_gp_growth_rate_floquet():
    # Time-periodic flow: Floquet multiplier of the one-period map by power iteration,
    # gamma = ln|mu| / 2 pi (Sec. 1).  Table 1: GP, Rm = 3, kx = 0.57, N_F = 16 -> 0.15.
    row = [r for r in _table1() if r["flow"] == "gp" and r["Rm"] == 3][0]
    n = 16
    p = O.Problem(O.GALLOWAY_PROCTOR, n, row["k"], row["Rm"])
    S = 1257
    dt = 2 * np.pi / S
    b = I.initial_field(n, row["k"], 1)
    g = []
    for _ in range(6):
        nb = O.propagate(b, p, 0.0, dt, S)
        g.append(math.log(O.l2(nb) / O.l2(b)) / (2 * np.pi))
        b = nb / O.l2(nb)
    assert abs(g[-1] - g[-2]) < 1e-7
    assert _round2(g[-1]) == row["rate"], g


# ------------------------------------------------------ learned coarse propagator
def test_learned_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    nc, m, wd = 4, 6, 0.3
    c = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    W, W0, X, Y = c(nc, nc), c(nc, nc), c(m, nc), c(m, nc)
    _, G = O.learned_loss_grad(W, X, Y, W0, wd)
    h = 1e-6
    for i in range(nc):
        for j in range(nc):
            for part, unit in ((0, 1.0), (1, 1j)):
                Wp, Wm = W.copy(), W.copy()
                Wp[i, j] += h * unit
                Wm[i, j] -= h * unit
                fd = (O.learned_loss_grad(Wp, X, Y, W0, wd)[0] - O.learned_loss_grad(Wm, X, Y, W0, wd)[0]) / (2 * h)
                g = G[i, j].real if part == 0 else G[i, j].imag
                assert abs(fd - g) < 1e-6 * max(1.0, abs(g)), (i, j, part, fd, g)


def test_learned_ridge_solution_zeroes_gradient_and_recovers_exact_map():
    rng = np.random.default_rng(4)
    nc = 5
    c = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    Wstar, W0 = c(nc, nc), c(nc, nc)
    X = c(3, nc)                      # underdetermined: 3 pairs, 5 unknowns per row
    Y = X @ Wstar.T
    Wr = O.learned_ridge(X, Y, W0, 0.1)
    assert np.abs(O.learned_loss_grad(Wr, X, Y, W0, 0.1)[1]).max() < 1e-12
    X = c(12, nc)                     # overdetermined, no regularisation: exact recovery
    Wr = O.learned_ridge(X, X @ Wstar.T, W0, 0.0)
    assert np.abs(Wr - Wstar).max() < 1e-10


def test_learned_minnorm_interpolates_and_changes_nothing_off_the_inputs():
    # the defining properties: W x_i = y_i, and (W - W0) v = 0 for every v orthogonal to
    # the inputs (complex inner product); learned_ridge tends to it as wd -> 0
    rng = np.random.default_rng(6)
    nc, m = 7, 3
    c = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    W0, X, Y = c(nc, nc), c(m, nc), c(m, nc)
    W = O.learned_minnorm(X, Y, W0)
    assert np.abs(X @ W.T - Y).max() < 1e-12
    Q, _ = np.linalg.qr(X.T, mode="complete")                 # last nc - m columns: x_i^H v = 0
    V = Q[:, m:]
    assert np.abs(np.conj(X) @ V).max() < 1e-12
    assert np.abs((W - W0) @ V).max() < 1e-12
    assert np.abs(O.learned_ridge(X, Y, W0, 1e-7) - W).max() < 1e-5


def test_learned_exact_map_reproduces_fine_pairs():
    # R F P is the fine propagator restricted to the set: zero loss on its own pairs
    prob = O.Problem(O.GALLOWAY_PROCTOR, 16, 0.57, 30.0)
    m, dt, S, t0 = 4, 0.01, 6, 0.35
    Wex = O.learned_exact_map(prob, m, t0, dt, S)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3, 3 * m * m)) + 1j * rng.standard_normal((3, 3 * m * m))
    Y = O.learned_restrict(O.propagate(O.learned_prolong(X, m, 16), prob, t0, dt, S), m)
    loss, _ = O.learned_loss_grad(Wex, X, Y, Wex, 0.0)
    assert loss < 1e-26 * np.sum(np.abs(Y) ** 2)
    # restriction and prolongation are inverse on the set
    assert np.abs(O.learned_restrict(O.learned_prolong(X, m, 16), m) - X).max() == 0.0
