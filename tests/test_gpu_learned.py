"""Learned coarse propagator: its forward and backward kernels against the CPU oracle,
the training pairs against the oracle's fine propagator, the classical initialisation
against the oracle's coarse propagator, and what the trained operator gains in
Parareal over the classical coarse propagator."""
import math

import numpy as np
import pytest

import kd_inputs as I
from oracle import kd_oracle as O

pytestmark = pytest.mark.gpu

N_FINE, KZ, RM = 32, 0.57, 100.0
M_SET = 8                      # learned set kx, ky in [-4, 4)
NC = 3 * M_SET * M_SET
SLICE = 2 * np.pi / 16
N_PHASE = 16
DT_F, DT_C = 5e-3, 0.04


@pytest.fixture(scope="module")
def kd():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_00387_gb300 as kd
    kd.load()
    torch.cuda.init()
    return kd


def bf16(a):
    """Round float32 values to bfloat16 (nearest even), returned as float64."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def make_ctx(kd, coarse_kind=0):
    p = kd.make_params(O.GALLOWAY_PROCTOR, N_FINE, KZ, RM, DT_F, kd.KD_C64, n_coarse=16, dt_coarse=DT_C,
                       prec_coarse=kd.KD_C64, fine_form=kd.KD_FINE_INCREMENT, learned_modes=M_SET,
                       coarse_kind=coarse_kind)
    return kd.kd_create(p)


def learned_inputs(seeds):
    """Seeded |k|^-2 fields restricted to the learned set, as learned vectors."""
    return np.stack([O.learned_restrict(I.initial_field(N_FINE, KZ, s), M_SET) for s in seeds])


def test_loss_and_gradient_match_oracle(kd):
    import torch
    rng = np.random.default_rng(0)
    m, wd = 12, 0.05
    W = (0.1 * rng.standard_normal((2 * NC, NC))).astype(np.float32)
    W0 = (0.1 * rng.standard_normal((2 * NC, NC))).astype(np.float32)
    X = (rng.standard_normal((m, NC)) + 1j * rng.standard_normal((m, NC))).astype(np.complex64)
    Y = (rng.standard_normal((m, NC)) + 1j * rng.standard_normal((m, NC))).astype(np.complex64)
    ctx = make_ctx(kd)
    try:
        g = torch.zeros((2 * NC, NC), dtype=torch.float32, device="cuda")
        loss = kd.kd_learned_loss_grad(ctx, torch.tensor(W, device="cuda"), torch.tensor(W0, device="cuda"), wd,
                                       torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"), m, g)
        grad = g.cpu().numpy()
    finally:
        kd.kd_destroy(ctx)
    # the same arithmetic in FP64 with the kernels' BF16 operands: W and X rounded for
    # the forward product, the residual rounded for the gradient product
    Wb = bf16(W[:NC]) + 1j * bf16(W[NC:])
    Xb = bf16(X.real) + 1j * bf16(X.imag)
    R = Xb @ Wb.T - Y.astype(np.complex128)
    Rb = bf16(R.real) + 1j * bf16(R.imag)
    Wc = W[:NC].astype(np.float64) + 1j * W[NC:]
    W0c = W0[:NC].astype(np.float64) + 1j * W0[NC:]
    G = (2.0 / m) * (Rb.T @ np.conj(Xb)) + 2.0 * wd * (Wc - W0c)
    assert rel(grad[:NC], G.real) < 1e-4 and rel(grad[NC:], G.imag) < 1e-4
    ref_loss = float(np.sum(np.abs(R) ** 2) / m + wd * np.sum(np.abs(Wc - W0c) ** 2))
    assert abs(loss - ref_loss) < 1e-5 * ref_loss
    # and the oracle's exact objective (no rounding) agrees to BF16 accuracy
    ex_loss, ex_grad = O.learned_loss_grad(Wc, X.astype(np.complex128), Y.astype(np.complex128), W0c, wd)
    assert abs(loss - ex_loss) < 2e-2 * ex_loss
    assert rel(grad[:NC] + 1j * grad[NC:], ex_grad) < 2e-2


def test_pairs_match_oracle_fine_propagator(kd):
    import torch
    x = learned_inputs([1, 2, 3])
    phase = [0, 5, 11]
    ctx = make_ctx(kd)
    try:
        kd.kd_learned_init(ctx, N_PHASE, SLICE)
        xt = torch.tensor(x.astype(np.complex64), device="cuda")
        yt = torch.zeros_like(xt)
        kd.kd_learned_pairs(ctx, xt, 3, phase, yt)
        y = yt.cpu().numpy()
    finally:
        kd.kd_destroy(ctx)
    prob = O.Problem(O.GALLOWAY_PROCTOR, N_FINE, KZ, RM)
    S = math.ceil(SLICE / DT_F - 1e-9)
    for i in range(3):
        ref = O.learned_restrict(O.propagate(O.learned_prolong(x[i], M_SET, N_FINE), prob, phase[i] * SLICE,
                                             SLICE / S, S), M_SET)
        assert rel(y[i], ref) < 1e-5


def test_initial_operator_is_the_classical_coarse_propagator(kd):
    import torch
    x = learned_inputs([4, 5])
    ctx = make_ctx(kd)
    try:
        kd.kd_learned_init(ctx, N_PHASE, SLICE)
        xt = torch.tensor(x.astype(np.complex64), device="cuda")
        yt = torch.zeros_like(xt)
        kd.kd_learned_apply(ctx, xt, yt, 3, 2)
        torch.cuda.synchronize()
        y = yt.cpu().numpy()
    finally:
        kd.kd_destroy(ctx)
    ng = 16                                          # grid with no aliasing for |k| <= 4
    prob = O.Problem(O.GALLOWAY_PROCTOR, ng, KZ, RM)
    Sc = math.ceil(SLICE / DT_C - 1e-9)
    mask = O.learned_mask(ng, M_SET)
    for i in range(2):
        ref = O.learned_restrict(O.propagate(O.learned_prolong(x[i], M_SET, ng), prob, 3 * SLICE, SLICE / Sc, Sc,
                                             mask=mask), M_SET)
        assert rel(y[i], ref) < 2e-2                 # BF16 operator


def _train(kd, ctx, n_per_phase, seed0, epochs=300, lr=1e-2, wd=0.0, m_set=M_SET):
    import torch
    n = n_per_phase * N_PHASE
    x = np.stack([O.learned_restrict(I.initial_field(N_FINE, KZ, s), m_set)
                  for s in range(seed0, seed0 + n)]).astype(np.complex64)
    phase = np.arange(n) % N_PHASE
    xt = torch.tensor(x, device="cuda")
    yt = torch.zeros_like(xt)
    kd.kd_learned_pairs(ctx, xt, n, phase, yt)
    loss = kd.kd_learned_train(ctx, xt, yt, phase, n, epochs, lr, wd, N_PHASE, kd.KD_TRAIN_ADAM)
    return loss


def test_training_reduces_error_below_classical(kd):
    import torch
    ctx = make_ctx(kd)
    try:
        kd.kd_learned_init(ctx, N_PHASE, SLICE)
        loss = _train(kd, ctx, 256, 10_000)
        assert np.all(loss[:, -1] < 0.1 * loss[:, 0])
        # held-out pairs from the same distribution: the fine solution decides
        n = 8 * N_PHASE
        xv = learned_inputs(range(50_000, 50_000 + n)).astype(np.complex64)
        ph = np.arange(n) % N_PHASE
        xt = torch.tensor(xv, device="cuda")
        yt = torch.zeros_like(xt)
        kd.kd_learned_pairs(ctx, xt, n, ph, yt)
        el, ec = kd.kd_learned_eval(ctx, xt, yt, ph, n, N_PHASE)
    finally:
        kd.kd_destroy(ctx)
    assert np.all(el < ec), (el, ec)
    assert np.median(el) < 0.3 * np.median(ec), (el, ec)


def test_parareal_gain_of_learned_coarse_propagator(kd):
    # Coarse set = the whole dealiased square |k| <= 10 of the 32^2 grid (m = 21), so
    # that the coarse propagators differ only in how they advance it: the classical one
    # with 5 RK443 steps of pi/40 per slice (cheap and crude), the learned one as a single
    # BF16 matrix fitted to fine-propagator pairs (1400 per phase, more than the 1323
    # unknowns per row) and started from that classical matrix.  The fine solution is
    # the measure: the learned operator is more accurate on held-out pairs, Parareal needs
    # fewer iterations with it, and both reproduce the fine solution.
    import torch
    T, N, m21, dtc = 2 * np.pi, 16, 21, 0.08
    b0 = I.initial_field(N_FINE, KZ, 7)
    res = {}
    for kind in (kd.KD_COARSE_CLASSICAL, kd.KD_COARSE_LEARNED):
        p = kd.make_params(O.GALLOWAY_PROCTOR, N_FINE, KZ, RM, DT_F, kd.KD_C64, n_coarse=16, dt_coarse=dtc,
                           prec_coarse=kd.KD_C64, fine_form=kd.KD_FINE_INCREMENT, learned_modes=m21,
                           coarse_kind=kind)
        ctx = kd.kd_create(p)
        try:
            if kind == kd.KD_COARSE_LEARNED:
                kd.kd_learned_init(ctx, N_PHASE, SLICE)
                _train(kd, ctx, 1400, 20_000, m_set=m21)
                nv = 4 * N_PHASE
                xv = np.stack([O.learned_restrict(I.initial_field(N_FINE, KZ, s), m21)
                               for s in range(90_000, 90_000 + nv)]).astype(np.complex64)
                ph = np.arange(nv) % N_PHASE
                xt = torch.tensor(xv, device="cuda")
                yt = torch.zeros_like(xt)
                kd.kd_learned_pairs(ctx, xt, nv, ph, yt)
                el, ec = kd.kd_learned_eval(ctx, xt, yt, ph, nv, N_PHASE)
                assert np.all(el < ec), (el, ec)
            out = np.zeros((N + 1, 3, N_FINE, N_FINE), np.complex128)
            status, st = kd.kd_parareal_run(ctx, b0, T, N, N, 1e-8, out)
            res[kind] = (st.k_con, bool(st.converged), bool(st.fallback_used), out, list(st.sigma[:st.k_con]))
        finally:
            kd.kd_destroy(ctx)
    kc, cc, _, uc, sc = res[kd.KD_COARSE_CLASSICAL]
    kl, cl, fl, ul, sl = res[kd.KD_COARSE_LEARNED]
    print("classical k_con", kc, sc)
    print("learned   k_con", kl, sl)
    # the learned run converges without falling back, in fewer iterations; the classical
    # one may need all N iterations (after which it is exact by construction)
    assert cl and not fl and sl[-1] <= 1e-8, sl
    assert kl < kc and (not cc or sl[-1] <= sc[-1]), (kl, kc, sc, sl)
    assert rel(ul[-1], uc[-1]) < 1e-5


def test_operator_checkpoint_round_trip(kd):
    """kd_learned_get / kd_learned_set: an operator copied out of one context and loaded
    into another gives the same products bit for bit, with its usability flag; a loaded
    zero operator gives zero."""
    import torch
    x = learned_inputs([6, 7, 8])
    xt = torch.tensor(x.astype(np.complex64), device="cuda")
    a, b = make_ctx(kd), make_ctx(kd)
    try:
        kd.kd_learned_init(a, N_PHASE, SLICE)
        kd.kd_learned_init(b, N_PHASE, SLICE)
        nc = 3 * M_SET * M_SET
        W = np.zeros((2 * nc, nc), np.uint16)                     # BF16 bit patterns on the host
        valid = kd.kd_learned_get(a, 5, W)
        assert W.any()
        Wz = torch.zeros((2 * nc, nc), dtype=torch.bfloat16, device="cuda")
        kd.kd_learned_set(b, 2, Wz, False)
        kd.kd_learned_set(b, 5, W, valid)
        assert kd.kd_learned_get(b, 5, np.zeros_like(W)) == valid
        ya, yb, y0 = (torch.zeros_like(xt) for _ in range(3))
        kd.kd_learned_apply(a, xt, ya, 5, 3)
        kd.kd_learned_apply(b, xt, yb, 5, 3)
        kd.kd_learned_apply(b, xt, y0, 2, 3)
        torch.cuda.synchronize()
        assert torch.equal(ya, yb)
        assert not y0.any()
        W2 = np.zeros_like(W)
        kd.kd_learned_get(b, 5, W2)
        assert np.array_equal(W, W2)
        with pytest.raises(kd.KdError):
            kd.kd_learned_get(a, N_PHASE, W)
    finally:
        kd.kd_destroy(a)
        kd.kd_destroy(b)


def _bf16_bits_to_complex(Wb):
    """BF16 bit patterns of a stacked operator [2 nc][nc] -> complex [nc][nc]."""
    f = (Wb.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    nc = Wb.shape[1]
    return f[:nc] + 1j * f[nc:]


@pytest.mark.parametrize("wd", [0.0, 1e-2])
def test_minimum_norm_correction_matches_oracle_ridge(kd, wd):
    """KD_TRAIN_MINNORM against the oracle's closed-form minimisers (learned_minnorm for
    wd = 0, learned_ridge for wd > 0), with
    the centre W0 the oracle's coarse propagator on the learned set (columns from unit
    vectors) and 48 pairs for 192 unknowns a row.  The outputs are y = (W0 + D) x for a
    fixed perturbation D of 20% of W0, so that the correction (D projected on the span of
    the inputs) is far above the BF16 resolution of the stored operator.  With wd = 0 the
    operator maps every training input onto its output."""
    import torch
    ph, m = 3, 48
    X = learned_inputs(range(70_000, 70_000 + m))               # learned vectors [m][NC]
    ng = 16                                                     # grid with no aliasing for |k| <= 4
    probc = O.Problem(O.GALLOWAY_PROCTOR, ng, KZ, RM)
    Sc = math.ceil(SLICE / DT_C - 1e-9)
    mask = O.learned_mask(ng, M_SET)
    W0 = np.zeros((NC, NC), np.complex128)
    for j in range(NC):
        e = np.zeros(NC, np.complex128)
        e[j] = 1.0
        W0[:, j] = O.learned_restrict(O.propagate(O.learned_prolong(e, M_SET, ng), probc, ph * SLICE, SLICE / Sc, Sc,
                                                  mask=mask), M_SET)
    rng = np.random.default_rng(5)
    D = rng.standard_normal((NC, NC)) + 1j * rng.standard_normal((NC, NC))
    D *= 0.2 * np.linalg.norm(W0) / np.linalg.norm(D)
    Y = X @ (W0 + D).T
    ref = O.learned_ridge(X, Y, W0, wd) if wd > 0 else O.learned_minnorm(X, Y, W0)
    ctx = make_ctx(kd)
    try:
        kd.kd_learned_init(ctx, N_PHASE, SLICE)
        xt = torch.tensor(X.astype(np.complex64), device="cuda")
        yt = torch.tensor(Y.astype(np.complex64), device="cuda")
        kd.kd_learned_train(ctx, xt, yt, [ph] * m, m, 0, 0.0, wd, N_PHASE, kd.KD_TRAIN_MINNORM)
        Wb = np.zeros((2 * NC, NC), np.uint16)
        kd.kd_learned_get(ctx, ph, Wb)
    finally:
        kd.kd_destroy(ctx)
    W = _bf16_bits_to_complex(Wb)
    assert rel(W, ref) < 4e-3                                  # BF16 storage of the operator
    assert rel(W - W0, ref - W0) < 0.05                        # the correction itself
    err, err0 = rel(X @ W.T, Y), rel(X @ W0.T, Y)
    if wd == 0.0:
        assert err < 0.02 * err0, (err, err0)                  # interpolation
    else:
        assert err < err0, (err, err0)
