"""The fine propagator on fields in the kept-mode layout [batch][3][P][P] (the |kx|, |ky| <=
n/3 square the 2/3 rule keeps): kd_fine_batched_kept on device buffers and
kd_fine_batched_host_kept on host buffers, against the full-layout call and the oracle."""
import ctypes

import numpy as np
import pytest

import kd_inputs as I
from oracle import kd_oracle as O

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-11


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


def kept_index(n):
    K = n // 3
    return np.arange(-K, K + 1) % n


def to_kept(full):
    """[..., n, n] (FFT order) -> [..., P, P] (row iy: ky = iy - K; column ix: kx = ix - K)."""
    idx = kept_index(full.shape[-1])
    return np.ascontiguousarray(full[..., idx[:, None], idx[None, :]])


def to_full(kept, n):
    out = np.zeros(kept.shape[:-2] + (n, n), dtype=kept.dtype)
    idx = kept_index(n)
    out[..., idx[:, None], idx[None, :]] = kept
    return out


@pytest.mark.parametrize("n,prec", [(64, "c64"), (64, "c128"), (128, "c64"), (160, "c64"), (1024, "c64")])
def test_kept_layout_equals_full_layout_and_oracle(kd, n, prec):
    """The same steps on the kept-mode array give the full-layout call's kept entries bit
    for bit (at 1024^2 the full-layout call keeps the state in the caller's layout, the
    kept-mode call in its own array), and the oracle's values."""
    import torch
    P = kd.KD_C128 if prec == "c128" else kd.KD_C64
    dtype = torch.complex128 if P == kd.KD_C128 else torch.complex64
    kz, Rm, dt, S = 0.57, 1e3, 2e-3, 3
    B = 1 if n == 1024 else 3
    b = I.initial_batch(n, kz, range(20, 20 + B))
    t0 = np.arange(B, dtype=np.float64) * 0.41
    ctx = kd.kd_create(kd.make_params(O.GALLOWAY_PROCTOR, n, kz, Rm, dt, P))
    try:
        tt = torch.tensor(t0, device="cuda")
        xf = torch.tensor(b, dtype=dtype, device="cuda")
        yf = torch.empty_like(xf)
        kd.kd_fine_batched(ctx, xf, yf, tt, S, B, P)
        xk = torch.tensor(to_kept(b), dtype=dtype, device="cuda")
        yk = torch.full_like(xk, float("nan"))
        kd.kd_fine_batched_kept(ctx, xk, yk, tt, S, B, P)
        torch.cuda.synchronize()
        full = yf.cpu().numpy()
        out = yk.cpu().numpy()
        assert np.array_equal(out, to_kept(full))
        # in place gives the same values
        kd.kd_fine_batched_kept(ctx, xk, xk, tt, S, B, P)
        torch.cuda.synchronize()
        assert torch.equal(xk, yk)
    finally:
        kd.kd_destroy(ctx)
    if n <= 160:
        p = O.Problem(O.GALLOWAY_PROCTOR, n, kz, Rm)
        for i in range(B):
            ref = O.propagate(b[i], p, t0[i], dt, S)
            assert rel(to_full(out[i].astype(np.complex128), n), ref) < (TOL64 if prec == "c128" else TOL32), i


@pytest.mark.parametrize("n,chunk,pinned", [(128, 0, True), (128, 2, False), (128, 3, True), (1024, 1, True)])
def test_host_kept_call_equals_device_kept_call(kd, n, chunk, pinned):
    """kd_fine_batched_host_kept (chunks through four device slots, stepped in place there,
    the last chunk ragged) gives kd_fine_batched_kept's values bit for bit, in place too."""
    import torch
    kz, Rm, dt, S = 0.57, 1e4, 1e-3, 2
    B = 7 if n == 128 else 3
    b = to_kept(I.initial_batch(n, kz, range(60, 60 + B)))
    t0 = np.arange(B, dtype=np.float64) * 0.29
    ctx = kd.kd_create(kd.make_params(O.GALLOWAY_PROCTOR, n, kz, Rm, dt, kd.KD_C64))
    try:
        x = torch.tensor(b, dtype=torch.complex64)
        y = torch.full_like(x, float("nan"))
        if pinned:
            x, y = x.pin_memory(), y.pin_memory()
        kd.kd_fine_batched_host_kept(ctx, x, y, t0, S, B, chunk)
        xd = x.cuda()
        yd = torch.empty_like(xd)
        kd.kd_fine_batched_kept(ctx, xd, yd, torch.tensor(t0, device="cuda"), S, B)
        torch.cuda.synchronize()
        assert torch.equal(y, yd.cpu())
        kd.kd_fine_batched_host_kept(ctx, x, x, t0, S, B, chunk)
        assert torch.equal(x, y)
        with pytest.raises(TypeError):
            kd.kd_fine_batched_host_kept(ctx, xd, y, t0, S, B, chunk)      # a device buffer is refused
        # the full-layout host call on the same context afterwards (shared slots and streams)
        xf = torch.tensor(to_full(b, n), dtype=torch.complex64).pin_memory()
        yf = torch.empty_like(xf).pin_memory()
        kd.kd_fine_batched_host(ctx, xf, yf, t0, S, B, chunk)
        assert np.array_equal(to_kept(yf.numpy()), y.numpy())
    finally:
        kd.kd_destroy(ctx)


def test_kept_call_edge_cases(kd):
    """No fields is a no-op; zero steps copies the input; a buffer that is not aligned to
    the complex element, a NULL buffer, a negative count and a short buffer are refused
    before anything is enqueued."""
    import torch
    n = 64
    P = kd.kept_side(n)
    ctx = kd.kd_create(kd.make_params(O.ROBERTS, n, 1.0, 8.0, 1e-2, kd.KD_C64))
    try:
        x = torch.tensor(to_kept(I.initial_batch(n, 1.0, [5, 6])), dtype=torch.complex64, device="cuda")
        y = torch.full_like(x, float("nan"))
        t0 = torch.zeros(2, dtype=torch.float64, device="cuda")
        kd.kd_fine_batched_kept(ctx, x, y, t0, 3, 0)
        torch.cuda.synchronize()
        assert torch.isnan(y).all()
        kd.kd_fine_batched_kept(ctx, x, y, t0, 0, 2)
        torch.cuda.synchronize()
        assert torch.equal(x, y)
        lib = kd.load()
        bad = ctypes.c_void_p(x.data_ptr() + 4)
        assert lib.kd_fine_batched_kept(ctx, bad, ctypes.c_void_p(y.data_ptr()),
                                        ctypes.c_void_p(t0.data_ptr()), 1, 1) == kd.KD_EINVAL
        assert lib.kd_fine_batched_kept(ctx, None, ctypes.c_void_p(y.data_ptr()),
                                        ctypes.c_void_p(t0.data_ptr()), 1, 1) == kd.KD_EINVAL
        assert lib.kd_fine_batched_kept(ctx, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                        ctypes.c_void_p(t0.data_ptr()), -1, 1) == kd.KD_EINVAL
        h = np.zeros((1, 3, P, P), np.complex64)
        assert lib.kd_fine_batched_host_kept(ctx, h.ctypes.data, h.ctypes.data, np.zeros(1).ctypes.data,
                                             1, 1, -1) == kd.KD_EINVAL
        with pytest.raises(ValueError):
            kd.kd_fine_batched_kept(ctx, x[:1], y, t0, 1, 2)
        torch.cuda.synchronize()
        assert torch.equal(x, y)
    finally:
        kd.kd_destroy(ctx)


def test_kept_layout_with_convolution_operator(kd):
    """KD_FINE_CONV through the kept-mode call: the full-layout call's kept entries."""
    import torch
    n, kz, Rm, dt, S, B = 96, 0.57, 1e3, 2e-3, 2, 2
    b = I.initial_batch(n, kz, [8, 9])
    ctx = kd.kd_create(kd.make_params(O.GALLOWAY_PROCTOR, n, kz, Rm, dt, kd.KD_C64, fine_operator=kd.KD_FINE_CONV))
    try:
        tt = torch.tensor([0.2, 1.3], dtype=torch.float64, device="cuda")
        xf = torch.tensor(b, dtype=torch.complex64, device="cuda")
        yf = torch.empty_like(xf)
        kd.kd_fine_batched(ctx, xf, yf, tt, S, B)
        xk = torch.tensor(to_kept(b), dtype=torch.complex64, device="cuda")
        yk = torch.empty_like(xk)
        kd.kd_fine_batched_kept(ctx, xk, yk, tt, S, B)
        torch.cuda.synchronize()
        assert np.array_equal(yk.cpu().numpy(), to_kept(yf.cpu().numpy()))
    finally:
        kd.kd_destroy(ctx)


def test_graded_chunk_plan_equals_device_call(kd):
    """chunk = 0 on 40 fields: the graded plan (2, 4, 8, 6, 6, 8, 4, 2 fields: chunks of
    unequal size rotating through the device slots) gives the device call's values bit for
    bit, in the kept-mode and in the full layout."""
    import torch
    n, kz, Rm, dt, S, B = 64, 0.57, 1e3, 2e-3, 2, 40
    b = I.initial_batch(n, kz, range(100, 100 + B))
    t0 = np.arange(B, dtype=np.float64) * 0.05
    ctx = kd.kd_create(kd.make_params(O.GALLOWAY_PROCTOR, n, kz, Rm, dt, kd.KD_C64))
    try:
        xd = torch.tensor(to_kept(b), dtype=torch.complex64, device="cuda")
        yd = torch.empty_like(xd)
        kd.kd_fine_batched_kept(ctx, xd, yd, torch.tensor(t0, device="cuda"), S, B)
        torch.cuda.synchronize()
        xk = xd.cpu().pin_memory()
        yk = torch.full_like(xk, float("nan")).pin_memory()
        kd.kd_fine_batched_host_kept(ctx, xk, yk, t0, S, B, 0)
        assert torch.equal(yk, yd.cpu())
        xf = torch.tensor(b, dtype=torch.complex64).pin_memory()
        yf = torch.full_like(xf, float("nan")).pin_memory()
        kd.kd_fine_batched_host(ctx, xf, yf, t0, S, B, 0)
        assert np.array_equal(to_kept(yf.numpy()), yk.numpy())
    finally:
        kd.kd_destroy(ctx)
