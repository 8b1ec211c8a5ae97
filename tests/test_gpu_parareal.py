"""Parity of the one-GPU Parareal driver (kd_parareal_run, kd_fine_serial) and the
growth-rate path (kd_energy, kd_growth_rate) with the CPU FP64 oracle."""
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


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def oracle_ops(prob, n_c, T, N, dt_f, dt_c):
    dT = T / N
    S = math.ceil(dT / dt_f - 1e-9)
    Sc = math.ceil(dT / dt_c - 1e-9)
    fine = lambda u, i: O.propagate(u, prob, i * dT, dT / S, S)
    coarse = lambda u, i: O.coarse_propagate(u, prob, n_c, i * dT, dT / Sc, Sc)
    return fine, coarse, S, Sc


# Roberts 32^2 complex128, kz = 1, Rm = 8, dt = 1e-2, T = 10, 8 slices, Delta t = 0.1, N_C = 16
C1 = dict(flow=O.ROBERTS, n=32, kz=1.0, Rm=8.0, dt=1e-2, T=10.0, N=8, dtc=0.1, nc=16)


def c1_ctx(kd):
    p = kd.make_params(C1["flow"], C1["n"], C1["kz"], C1["Rm"], C1["dt"], kd.KD_C128, n_coarse=C1["nc"],
                       dt_coarse=C1["dtc"], prec_coarse=kd.KD_C128)
    return kd.kd_create(p)


def test_parareal_roberts32_iterates_match_oracle(kd):
    # Same number of iterations on both sides (tol = 0), FP64 everywhere.
    b0 = I.initial_field(C1["n"], C1["kz"], 0)
    kmax = 3
    ctx = c1_ctx(kd)
    try:
        out = np.zeros((C1["N"] + 1, 3, C1["n"], C1["n"]), np.complex128)
        status, st = kd.kd_parareal_run(ctx, b0, C1["T"], C1["N"], kmax, 0.0, out)
    finally:
        kd.kd_destroy(ctx)
    assert status == kd.KD_ENOTCONV and st.k_con == kmax
    prob = O.Problem(C1["flow"], C1["n"], C1["kz"], C1["Rm"])
    fine, coarse, S, Sc = oracle_ops(prob, C1["nc"], C1["T"], C1["N"], C1["dt"], C1["dtc"])
    assert (st.n_fine_steps, st.n_coarse_steps) == (S, Sc) == (125, 13)
    ref = O.parareal(b0, fine, coarse, C1["N"], kmax, 0.0)
    for i in range(C1["N"] + 1):
        assert rel(out[i], ref["U"][i]) < 1e-11, i
    for k in range(kmax):
        assert abs(st.sigma[k] - ref["sigma"][k]) <= 1e-8 * ref["sigma"][k]


def test_parareal_k_equals_n_is_serial_fine_bitwise(kd):
    b0 = I.initial_field(C1["n"], C1["kz"], 1)
    ctx = c1_ctx(kd)
    try:
        par = np.zeros((C1["N"] + 1, 3, C1["n"], C1["n"]), np.complex128)
        ser = np.zeros_like(par)
        kd.kd_parareal_run(ctx, b0, C1["T"], C1["N"], C1["N"], 0.0, par)
        kd.kd_fine_serial(ctx, b0, C1["T"], C1["N"], ser)
    finally:
        kd.kd_destroy(ctx)
    assert np.array_equal(par, ser)
    prob = O.Problem(C1["flow"], C1["n"], C1["kz"], C1["Rm"])
    fine, _, _, _ = oracle_ops(prob, C1["nc"], C1["T"], C1["N"], C1["dt"], C1["dtc"])
    ref = O.serial_fine(b0, fine, C1["N"])
    assert rel(ser[-1], ref[-1]) < 1e-11


def test_parareal_gp_fp32_converges_to_serial_fine(kd):
    # GP flow, complex64 fine / complex64 coarse on N/2, FP64 update.  The coarse step
    # 0.05 is inside the explicit stability limit on the 32^2 grid; tol 1e-5 sits above
    # the FP32 round-off floor of the defect (about sqrt(N) x 2e-7 per slice).
    n, kz, Rm, T, N = 64, 0.57, 100.0, 2 * np.pi, 16
    dt, dtc = 5e-3, 0.05
    p = kd.make_params(O.GALLOWAY_PROCTOR, n, kz, Rm, dt, kd.KD_C64, n_coarse=32, dt_coarse=dtc,
                       prec_coarse=kd.KD_C64)
    b0 = I.initial_field(n, kz, 2)
    ctx = kd.kd_create(p)
    try:
        par = np.zeros((N + 1, 3, n, n), np.complex128)
        ser = np.zeros_like(par)
        status, st = kd.kd_parareal_run(ctx, b0, T, N, N, 1e-5, par)
        kd.kd_fine_serial(ctx, b0, T, N, ser)
    finally:
        kd.kd_destroy(ctx)
    assert status == kd.KD_OK and st.converged and st.k_con < N
    # Parareal reproduces the serial fine solution (same FP32 kernels) to its tolerance
    assert rel(par[-1], ser[-1]) < 1e-5
    # and every serial fine slice state matches the FP64 oracle propagated from the same
    # input state (per-slice tolerance 1e-5; sampled slices)
    prob = O.Problem(O.GALLOWAY_PROCTOR, n, kz, Rm)
    S = st.n_fine_steps
    dT = T / N
    for i in (0, 7, N - 1):
        x = O.propagate(ser[i], prob, i * dT, dT / S, S)
        assert rel(ser[i + 1], x) < 1e-5, i


def test_parareal_increment_form_passes_fp32_floor(kd):
    # GP flow, complex64 fine and coarse (coarse: same 64^2 grid, step 0.025).  In the
    # direct form the FP32 round-off of every F and G evaluation keeps the defect near
    # 1e-6; in the increment form F(U^k) = F(U^{k-1}) + F(U^k - U^{k-1}) and
    # G(U^{k+1}) - G(U^k) = G(U^{k+1} - U^k) the defect keeps falling.
    n, kz, Rm, T, N = 64, 0.57, 100.0, 2 * np.pi, 16
    res = {}
    for form in (kd.KD_FINE_DIRECT, kd.KD_FINE_INCREMENT):
        p = kd.make_params(O.GALLOWAY_PROCTOR, n, kz, Rm, 5e-3, kd.KD_C64, n_coarse=64, dt_coarse=0.025,
                           prec_coarse=kd.KD_C64, fine_form=form)
        ctx = kd.kd_create(p)
        try:
            par = np.zeros((N + 1, 3, n, n), np.complex128)
            status, st = kd.kd_parareal_run(ctx, I.initial_field(n, kz, 2), T, N, 8, 0.0, par)
        finally:
            kd.kd_destroy(ctx)
        res[form] = (list(st.sigma[:st.k_con]), par)
    s_dir, _ = res[kd.KD_FINE_DIRECT]
    s_inc, par = res[kd.KD_FINE_INCREMENT]
    assert min(s_dir) > 1e-8                  # round-off floor of the direct form
    assert s_inc[-1] < 1e-9 and s_inc[-1] < 1e-2 * min(s_dir)
    # the converged iterate is a fine solution to FP32 accuracy: each slice matches the
    # FP64 oracle propagated from the iterate's previous slice state
    prob = O.Problem(O.GALLOWAY_PROCTOR, n, kz, Rm)
    S = math.ceil(T / N / 5e-3 - 1e-9)
    dT = T / N
    for i in (0, 5, N - 1):
        x = O.propagate(par[i], prob, i * dT, dT / S, S)
        assert rel(par[i + 1], x) < 1e-5, i


def test_energy_and_growth_fit_match_oracle(kd):
    import torch
    n = 32
    ctx = c1_ctx(kd)
    try:
        fields = np.stack([I.initial_field(n, 1.0, s) * math.exp(0.3 * s) for s in range(9)])
        x = torch.tensor(fields, device="cuda")
        E = torch.zeros(9, dtype=torch.float64, device="cuda")
        kd.kd_energy(ctx, x, 9, E)
        torch.cuda.synchronize()
        e = E.cpu().numpy()
        for i in range(9):
            assert abs(e[i] - O.energy(fields[i])) <= 1e-14 * O.energy(fields[i])
        rate = kd.kd_growth_rate(ctx, x, 9, 4.0, 2.0)
    finally:
        kd.kd_destroy(ctx)
    ts = np.linspace(0, 4.0, 9)
    assert abs(rate - O.growth_rate(ts, [O.energy(f) for f in fields], 2.0)) < 1e-13


def test_parareal_stats_growth_rate_matches_oracle(kd):
    # Roberts Rm = 8, kz = 1: the leading eigenvalue of the spectral operator is ~0.04994
    b0 = I.initial_field(C1["n"], C1["kz"], 3)
    ctx = c1_ctx(kd)
    try:
        status, st = kd.kd_parareal_run(ctx, b0, 40.0, 32, 32, 1e-10, None)
    finally:
        kd.kd_destroy(ctx)
    prob = O.Problem(C1["flow"], C1["n"], C1["kz"], C1["Rm"])
    E = list(st.energy[:33])
    fit = O.growth_rate(np.arange(33) * 40.0 / 32, E, 20.0)
    assert abs(st.growth_rate - fit) < 1e-12
    import scipy.sparse.linalg as sla
    lam = sla.eigs(O.linear_operator(prob).tocsc(), k=3, sigma=0.3, return_eigenvectors=False)
    assert abs(st.growth_rate - max(lam.real)) < 1e-3


def test_invalid_arguments_are_rejected(kd):
    ctx = c1_ctx(kd)
    try:
        with pytest.raises(kd.KdError) as e:
            kd.kd_parareal_run(ctx, I.initial_field(32, 1.0, 0), 1.0, 0, 3, 1e-6)
        assert e.value.status == kd.KD_EINVAL
        with pytest.raises(kd.KdError):
            kd.kd_parareal_run(ctx, I.initial_field(32, 1.0, 0), -1.0, 4, 3, 1e-6)
    finally:
        kd.kd_destroy(ctx)


def test_parareal_with_convolution_fine_operator(kd):
    """The whole Parareal run with KD_FINE_CONV agrees with the FFT fine operator to FP32
    accuracy, takes the same iterations, and reproduces its own serial fine run."""
    n, kz, Rm, T, N = 32, 0.57, 100.0, 2.0, 8
    b0 = I.initial_field(n, kz, 19)
    outs, ks = [], []
    for op in (kd.KD_FINE_FFT, kd.KD_FINE_CONV):
        p = kd.make_params(O.GALLOWAY_PROCTOR, n, kz, Rm, 5e-3, kd.KD_C64, n_coarse=32, dt_coarse=0.025,
                           prec_coarse=kd.KD_C64, fine_form=kd.KD_FINE_INCREMENT, fine_operator=op)
        ctx = kd.kd_create(p)
        try:
            u = np.zeros((N + 1, 3, n, n), np.complex128)
            s, st = kd.kd_parareal_run(ctx, b0, T, N, N, 1e-6, u)
            ser = np.zeros_like(u)
            kd.kd_fine_serial(ctx, b0, T, N, ser)
        finally:
            kd.kd_destroy(ctx)
        assert s == kd.KD_OK
        assert np.linalg.norm(u[-1] - ser[-1]) / np.linalg.norm(ser[-1]) < 1e-5
        outs.append(u)
        ks.append(st.k_con)
    assert ks[0] == ks[1]
    assert np.linalg.norm(outs[1][-1] - outs[0][-1]) / np.linalg.norm(outs[0][-1]) < 2e-5


def test_parareal_table1_roberts_grids_match_oracle(kd):
    """Parareal on Table 1's Roberts grids (N_F = 160, N_C = 80, delta t = 1e-2,
    Delta t = 2e-2; neither side a power of two), FP64 on both sides, iterates equal to
    the oracle's Parareal."""
    n, nc, kz, Rm, T, N, kmax = 160, 80, 2.87, 512.0, 0.8, 4, 2
    b0 = I.initial_field(n, kz, 23)
    p = kd.make_params(O.ROBERTS, n, kz, Rm, 1e-2, kd.KD_C128, n_coarse=nc, dt_coarse=2e-2,
                       prec_coarse=kd.KD_C128, fine_operator=kd.KD_FINE_CONV)
    ctx = kd.kd_create(p)
    try:
        out = np.zeros((N + 1, 3, n, n), np.complex128)
        status, st = kd.kd_parareal_run(ctx, b0, T, N, kmax, 0.0, out)
    finally:
        kd.kd_destroy(ctx)
    assert status == kd.KD_ENOTCONV and st.k_con == kmax
    prob = O.Problem(O.ROBERTS, n, kz, Rm)
    fine, coarse, S, Sc = oracle_ops(prob, nc, T, N, 1e-2, 2e-2)
    assert (st.n_fine_steps, st.n_coarse_steps) == (S, Sc) == (20, 10)
    ref = O.parareal(b0, fine, coarse, N, kmax, 0.0)
    for i in range(N + 1):
        assert rel(out[i], ref["U"][i]) < 1e-11, i
    for k in range(kmax):
        assert abs(st.sigma[k] - ref["sigma"][k]) <= 1e-8 * ref["sigma"][k]


@pytest.mark.parametrize("form", ["direct", "increment"])
@pytest.mark.parametrize("chunks", [1, 3, 16])
def test_pipelined_iterations_equal_unpipelined(kd, form, chunks):
    """The fine sweep of iteration k + 1 overlapping the serial sweep of iteration k gives
    the same slice states and defects bit for bit as the unpipelined order."""
    n, kz, Rm, T, N = 32, 0.57, 100.0, 3.0, 13
    b0 = I.initial_field(n, kz, 23)
    res = []
    for ov in (0, chunks):
        p = kd.make_params(O.GALLOWAY_PROCTOR, n, kz, Rm, 5e-3, kd.KD_C64, n_coarse=32, dt_coarse=0.025,
                           prec_coarse=kd.KD_C64,
                           fine_form=kd.KD_FINE_INCREMENT if form == "increment" else kd.KD_FINE_DIRECT)
        ctx = kd.kd_create(p)
        try:
            kd.kd_set_overlap(ctx, ov)
            u = np.zeros((N + 1, 3, n, n), np.complex128)
            s, st = kd.kd_parareal_run(ctx, b0, T, N, 5, 0.0, u)
            res.append((u, list(st.sigma[:st.k_con]), st.k_con))
        finally:
            kd.kd_destroy(ctx)
    assert res[0][2] == res[1][2] == 5
    assert res[0][1] == res[1][1]
    assert np.array_equal(res[0][0], res[1][0])


def c1_increment_ctx(kd):
    p = kd.make_params(C1["flow"], C1["n"], C1["kz"], C1["Rm"], C1["dt"], kd.KD_C128, n_coarse=C1["nc"],
                       dt_coarse=C1["dtc"], prec_coarse=kd.KD_C128, fine_form=kd.KD_FINE_INCREMENT)
    return kd.kd_create(p)


def test_resume_from_a_checkpointed_iterate(kd):
    """kd_parareal_resume continues from the iterate an earlier run returned: iterations 3
    and 4 resumed from U^2 equal those of the uninterrupted run (FP64; the first resumed
    fine sweep is direct instead of incremental, so equal to round-off)."""
    b0 = I.initial_field(C1["n"], C1["kz"], 2)
    N, T = C1["N"], C1["T"]
    ctx = c1_increment_ctx(kd)
    try:
        u2 = np.zeros((N + 1, 3, C1["n"], C1["n"]), np.complex128)
        s, st2 = kd.kd_parareal_run(ctx, b0, T, N, 2, 0.0, u2)
        u4 = np.zeros_like(u2)
        s, st4 = kd.kd_parareal_run(ctx, b0, T, N, 4, 0.0, u4)
        ur = np.zeros_like(u2)
        s, str_ = kd.kd_parareal_resume(ctx, u2, 2, T, N, 4, 0.0, ur)
    finally:
        kd.kd_destroy(ctx)
    assert str_.k_con == 4 and list(str_.sigma[:2]) == [0.0, 0.0]
    for k in (2, 3):
        assert abs(str_.sigma[k] - st4.sigma[k]) <= 1e-8 * st4.sigma[k], k
    for i in range(N + 1):
        assert rel(ur[i], u4[i]) < 1e-12, i


def test_resume_from_the_fine_solution_is_converged(kd):
    """An initial iterate that is already the serial fine solution is a fixed point: the
    first defect is round-off."""
    b0 = I.initial_field(C1["n"], C1["kz"], 3)
    N, T = C1["N"], C1["T"]
    ctx = c1_increment_ctx(kd)
    try:
        ser = np.zeros((N + 1, 3, C1["n"], C1["n"]), np.complex128)
        kd.kd_fine_serial(ctx, b0, T, N, ser)
        s, st = kd.kd_parareal_resume(ctx, ser, 0, T, N, 3, 1e-12)
    finally:
        kd.kd_destroy(ctx)
    assert s == kd.KD_OK and st.k_con == 1 and st.sigma[0] < 1e-12


def test_resume_needs_the_increment_form(kd):
    ctx = c1_ctx(kd)                                 # KD_FINE_DIRECT
    try:
        u = np.zeros((C1["N"] + 1, 3, C1["n"], C1["n"]), np.complex128)
        u[0] = I.initial_field(C1["n"], C1["kz"], 0)
        with pytest.raises(kd.KdError):
            kd.kd_parareal_resume(ctx, u, 0, C1["T"], C1["N"], 2, 0.0)
    finally:
        kd.kd_destroy(ctx)


@pytest.mark.parametrize("overlap", [0])
def test_captured_graphs_give_the_direct_launch_values(kd, overlap):
    """The fine sweeps replayed from captured CUDA graphs give the iterates and defects
    of the direct launches bit for bit, also when the same graphs are replayed by a
    second solve."""
    n, N, T = 64, 16, 4.0
    b0 = I.initial_field(n, 0.57, 31)
    outs = []
    for graphs in (False, True, True):
        p = kd.make_params(O.GALLOWAY_PROCTOR, n, 0.57, 100.0, 5e-3, kd.KD_C64, n_coarse=64, dt_coarse=2.0 / 64,
                           prec_coarse=kd.KD_C64, fine_form=kd.KD_FINE_INCREMENT)
        ctx = kd.kd_create(p)
        try:
            kd.kd_set_graphs(ctx, graphs)
            kd.kd_set_overlap(ctx, overlap)
            u = np.zeros((N + 1, 3, n, n), np.complex128)
            kd.kd_parareal_run(ctx, b0, T, N, 6, 0.0, u)
            u2 = np.zeros_like(u)
            s, st = kd.kd_parareal_run(ctx, b0, T, N, 6, 0.0, u2)      # the cached graphs again
            assert np.array_equal(u, u2)
            outs.append((u2, [st.sigma[k] for k in range(6)]))
        finally:
            kd.kd_destroy(ctx)
    for u, sig in outs[1:]:
        assert np.array_equal(u, outs[0][0])
        assert sig == outs[0][1]


def test_true_error_against_a_reference(kd):
    """stats.true_err[k - 1] is the relative distance of the k-th iterate's last slice to
    the reference set by kd_set_reference (here the serial fine solution): every entry
    equals the distance of the final slice of a run stopped after k iterations, it is 0
    at k = N (Parareal is then the serial fine run), and -1 without a reference."""
    b0 = I.initial_field(C1["n"], C1["kz"], 4)
    N = C1["N"]
    ctx = c1_ctx(kd)
    try:
        ser = np.zeros((N + 1, 3, C1["n"], C1["n"]), np.complex128)
        kd.kd_fine_serial(ctx, b0, C1["T"], N, ser)
        kd.kd_set_reference(ctx, ser[-1])
        dist = []
        for k in (1, 2, 3):
            par = np.zeros_like(ser)
            kd.kd_parareal_run(ctx, b0, C1["T"], N, k, 0.0, par)
            dist.append(rel(par[-1], ser[-1]))
        _, st = kd.kd_parareal_run(ctx, b0, C1["T"], N, 3, 0.0)
        te = [st.true_err[i] for i in range(kd.KD_MAX_ITERS)]
        assert all(e == -1.0 for e in te[3:])
        for k in range(3):
            assert dist[k] > 0 and abs(te[k] - dist[k]) <= 1e-9 * dist[k], k
        _, st = kd.kd_parareal_run(ctx, b0, C1["T"], N, N, 0.0)
        assert st.true_err[N - 1] == 0.0
        kd.kd_set_reference(ctx, None)
        _, st = kd.kd_parareal_run(ctx, b0, C1["T"], N, 2, 0.0)
        assert st.true_err[0] == -1.0 and st.true_err[1] == -1.0
    finally:
        kd.kd_destroy(ctx)


def test_benched_gp128_solve_matches_oracle(kd):
    """The 128^2 GP Parareal solve exactly as bench.py times it (64 slices, coarse step
    2/128 on the fine grid, increment form, sigma <= 1e-6): sampled slices of the returned
    iterate each propagated by the oracle over one slice, and the growth rate of the solve
    against the oracle's serial FP64 run (Eq. 8, Eq. 9, Table 1 "Growth Rate")."""
    import bench
    W = bench.WL
    n, N, T = W["n"], W["slices"], W["T"]
    p = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, n, W["kz"], W["Rm"], W["dt_fine_max"], kd.KD_C64,
                       n_coarse=W["n_coarse"], dt_coarse=W["dt_coarse_max"], prec_coarse=kd.KD_C64,
                       fine_form=kd.KD_FINE_INCREMENT)
    ctx = kd.kd_create(p)
    b0 = I.initial_field(n, W["kz"], 1000)
    out = np.zeros((N + 1, 3, n, n), np.complex128)
    try:
        status, st = kd.kd_parareal_run(ctx, b0, T, N, W["k_max"], W["tol"], out)
    finally:
        kd.kd_destroy(ctx)
    assert status == kd.KD_OK and st.sigma[st.k_con - 1] <= W["tol"]
    dT = T / N
    S = st.n_fine_steps
    assert S == bench.fine_steps_per_slice()
    prob = O.Problem(O.GALLOWAY_PROCTOR, n, W["kz"], W["Rm"])
    for i in (0, 21, 42, 63):
        ref = O.propagate(out[i], prob, i * dT, dT / S, S)
        assert rel(out[i + 1], ref) < 1e-5, i
    U = O.serial_fine(b0, lambda u, i: O.propagate(u, prob, i * dT, dT / S, S), N)
    g_ref = O.growth_rate(np.arange(N + 1) * dT, [O.energy(u) for u in U], 0.5 * T)
    assert abs(st.growth_rate - g_ref) < 1e-4 * abs(g_ref), (st.growth_rate, g_ref)
