"""The allocation limit of a context (kd_set_alloc_limit): device out-of-memory made on the
host, without exhausting the GPU.  A call that needs a buffer beyond the limit returns
KD_ENOMEM with a message naming the limit, keeps no new buffer, and the same context then
runs the call normally once the limit allows it, with the values of a context that never
failed."""
import numpy as np
import pytest

import kd_inputs as I

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


def fine_once(kd, ctx, x, t0, nsteps):
    import torch
    out = torch.full_like(x, float("nan"))
    kd.kd_fine_batched(ctx, x, out, t0, nsteps, x.shape[0], kd.KD_C64)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def expect_enomem(kd, fn):
    with pytest.raises(kd.KdError) as e:
        fn()
    assert e.value.status == kd.KD_ENOMEM
    assert "allocation limit" in str(e.value)


def test_fine_call_beyond_the_limit_fails_and_the_context_recovers(kd):
    import torch
    p = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, 64, 0.57, 100.0, 5e-3, kd.KD_C64)
    b = I.initial_batch(64, 0.57, [3, 4, 5, 6, 7, 8, 9, 10])
    x8 = torch.tensor(b, dtype=torch.complex64, device="cuda")
    x4 = x8[:4].contiguous()
    t8 = torch.linspace(0.0, 1.4, 8, dtype=torch.float64, device="cuda")
    t4 = t8[:4].contiguous()
    fresh = kd.kd_create(p)
    try:
        want = fine_once(kd, fresh, x4, t4, 3)
    finally:
        kd.kd_destroy(fresh)
    ctx = kd.kd_create(p)
    try:
        held0, lim = kd.kd_get_alloc_bytes(ctx)
        assert held0 > 0 and lim == 0          # the grid tables, no limit by default
        # no room for the workspace: refused, nothing new kept
        kd.kd_set_alloc_limit(ctx, held0)
        assert kd.kd_get_alloc_bytes(ctx) == (held0, held0)
        expect_enomem(kd, lambda: fine_once(kd, ctx, x4, t4, 3))
        assert kd.kd_get_alloc_bytes(ctx)[0] == held0
        # limit lifted: the same call runs, with a fresh context's values
        kd.kd_set_alloc_limit(ctx, 0)
        assert np.array_equal(fine_once(kd, ctx, x4, t4, 3), want)
        held1 = kd.kd_get_alloc_bytes(ctx)[0]
        assert held1 > held0
        # a limit at what is held lets calls that need no new buffer run
        kd.kd_set_alloc_limit(ctx, held1)
        assert np.array_equal(fine_once(kd, ctx, x4, t4, 3), want)
        # a larger batch needs a larger workspace: refused (the old one was released first)
        expect_enomem(kd, lambda: fine_once(kd, ctx, x8, t8, 3))
        assert kd.kd_get_alloc_bytes(ctx)[0] <= held1
        # the smaller batch again: its workspace is made anew within the limit
        assert np.array_equal(fine_once(kd, ctx, x4, t4, 3), want)
        assert kd.kd_get_alloc_bytes(ctx)[0] == held1
    finally:
        kd.kd_destroy(ctx)


def test_parareal_beyond_the_limit_fails_then_converges(kd):
    # Roberts 32^2 complex128; the limit admits the first Parareal array (U, 9 slice
    # states) but not the second, so the failure comes in the middle of the set-up
    n, kz, Rm, dt, T, N = 32, 1.0, 8.0, 1e-2, 10.0, 8
    p = kd.make_params(kd.KD_FLOW_ROBERTS, n, kz, Rm, dt, kd.KD_C128, n_coarse=16, dt_coarse=0.1,
                       prec_coarse=kd.KD_C128)
    b0 = I.initial_field(n, kz, 2)
    P = 2 * (n // 3) + 1
    u_bytes = (N + 1) * 3 * P * P * 16

    def run(ctx):
        out = np.zeros((N + 1, 3, n, n), np.complex128)
        status, st = kd.kd_parareal_run(ctx, b0, T, N, 8, 1e-10, out)
        return status, st, out

    fresh = kd.kd_create(p)
    try:
        s_ref, st_ref, want = run(fresh)
    finally:
        kd.kd_destroy(fresh)
    assert s_ref == kd.KD_OK
    ctx = kd.kd_create(p)
    try:
        held0 = kd.kd_get_alloc_bytes(ctx)[0]
        kd.kd_set_alloc_limit(ctx, held0 + u_bytes + 1024)
        expect_enomem(kd, lambda: run(ctx))
        assert kd.kd_get_alloc_bytes(ctx)[0] <= held0 + u_bytes + 1024
        kd.kd_set_alloc_limit(ctx, 0)
        s, st, got = run(ctx)
        assert s == kd.KD_OK and st.k_con == st_ref.k_con
        assert np.array_equal(got, want)
        assert [st.sigma[k] for k in range(st.k_con)] == [st_ref.sigma[k] for k in range(st.k_con)]
    finally:
        kd.kd_destroy(ctx)
