"""The halo exchanges of the coarse-solver cluster kernel (kd_set_coarse_sync): halo
stores with a cluster barrier per stage, point-to-point st.async + mbarrier pushes, and
reads of the neighbours' rows after a split barrier give the same results bit for bit, for every modes-per-thread variant, cluster sizes whose last blocks
own no rows, both precisions, the convolution fine operator and the fused Parareal
update; and both match the CPU FP64 oracle."""
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


def conv_fine(kd, n, prec, cluster, sync, b, t0, nsteps, flow=O.GALLOWAY_PROCTOR):
    import torch
    kz, Rm, dt = 0.57, 100.0, 5e-3
    ctx = kd.kd_create(kd.make_params(flow, n, kz, Rm, dt, prec, n_coarse=n, fine_operator=kd.KD_FINE_CONV))
    try:
        if cluster:
            kd.kd_set_coarse_cluster(ctx, cluster)
        kd.kd_set_coarse_sync(ctx, sync)
        dtype = torch.complex64 if prec == kd.KD_C64 else torch.complex128
        x = torch.tensor(b, dtype=dtype, device="cuda")
        y = torch.empty_like(x)
        kd.kd_fine_batched(ctx, x, y, torch.tensor(t0, dtype=torch.float64, device="cuda"), nsteps, b.shape[0], prec)
        torch.cuda.synchronize()
        return y.cpu().numpy().astype(np.complex128)
    finally:
        kd.kd_destroy(ctx)


# (n, blocks per cluster): P = 2 (n // 3) + 1 kept modes a side
#   32 / 0: P 21, default 4 blocks of 6 rows, 2 modes per thread (256 threads)
#   128 / 8: P 85, 11 rows a block, 4 modes per thread
#   128 / 16: P 85, 6 rows, 1 mode per thread (512 threads), the last block 5 rows
#   150 / 16: P 101, 7 rows a block, the 16th block owns no row
#   160 / 12: P 107, 9 rows, the last block 8 rows
#   190 / 16: P 127, 8 rows, 4 modes per thread
CASES = [(32, 0), (128, 8), (128, 16), (150, 16), (160, 12), (190, 16)]


@pytest.mark.parametrize("n,cluster", CASES)
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_point_to_point_equals_cluster_barrier_and_oracle(kd, n, cluster, prec):
    P = kd.KD_C64 if prec == "c64" else kd.KD_C128
    b = I.initial_batch(n, 0.57, [81, 82])
    t0 = [0.0, 0.9]
    out_c = conv_fine(kd, n, P, cluster, kd.KD_SYNC_CLUSTER, b, t0, 5)
    for mode in (kd.KD_SYNC_P2P, kd.KD_SYNC_PULL):
        assert np.array_equal(conv_fine(kd, n, P, cluster, mode, b, t0, 5), out_c), mode
    out_p = out_c
    p = O.Problem(O.GALLOWAY_PROCTOR, n, 0.57, 100.0)
    for i in range(2):
        assert rel(out_p[i], O.propagate(b[i], p, t0[i], 5e-3, 5)) < (1e-5 if P == kd.KD_C64 else 1e-12)


@pytest.mark.parametrize("nsteps", [0, 1])
def test_zero_and_one_step(kd, nsteps):
    b = I.initial_batch(64, 0.57, [83])
    out_p = conv_fine(kd, 64, kd.KD_C128, 16, kd.KD_SYNC_P2P, b, [0.3], nsteps)
    out_c = conv_fine(kd, 64, kd.KD_C128, 16, kd.KD_SYNC_CLUSTER, b, [0.3], nsteps)
    out_l = conv_fine(kd, 64, kd.KD_C128, 16, kd.KD_SYNC_PULL, b, [0.3], nsteps)
    assert np.array_equal(out_p, out_c) and np.array_equal(out_l, out_c)
    ref = O.propagate(b[0], O.Problem(O.GALLOWAY_PROCTOR, 64, 0.57, 100.0), 0.3, 5e-3, nsteps)
    assert rel(out_p[0], ref) < 1e-12


def test_parareal_update_and_defects_identical(kd):
    """The fused Parareal update and defect (Eq. 8, 9) through both exchanges: the same
    iterates and defects bit for bit (GP 128^2 c64 fine, N_C = 128 coarse)."""
    n, T, N = 128, 1.0, 8
    b0 = I.initial_field(n, 0.57, 84)
    res = []
    for sync in (kd.KD_SYNC_CLUSTER, kd.KD_SYNC_P2P, kd.KD_SYNC_PULL):
        p = kd.make_params(O.GALLOWAY_PROCTOR, n, 0.57, 300.0, 1e-3, kd.KD_C64, n_coarse=128, dt_coarse=2.0 / 128,
                           prec_coarse=kd.KD_C64, fine_form=kd.KD_FINE_INCREMENT)
        ctx = kd.kd_create(p)
        try:
            kd.kd_set_coarse_sync(ctx, sync)
            u = np.zeros((N + 1, 3, n, n), np.complex128)
            s, st = kd.kd_parareal_run(ctx, b0, T, N, 4, 0.0, u)
            res.append((u, [st.sigma[k] for k in range(4)]))
        finally:
            kd.kd_destroy(ctx)
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0])
        assert r[1] == res[0][1]


def test_sync_mode_validation(kd):
    ctx = kd.kd_create(kd.make_params(O.ROBERTS, 32, 1.0, 8.0, 1e-2, kd.KD_C64))
    try:
        with pytest.raises(kd.KdError):
            kd.kd_set_coarse_sync(ctx, 3)
    finally:
        kd.kd_destroy(ctx)
