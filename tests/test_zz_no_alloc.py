"""kd_fine_batched_static, the allocation-free variant of the fine propagator, against
kd_fine_batched through the C ABI.  The static variant serves callers that cannot
allocate device memory (a host application's pool owns the GPU memory, or a loop
that cannot pay for cudaMalloc's device synchronisation); its workspace is a fixed
device array inside the library.

The file name puts it last in collection order, so that a run stopping at its first
failure has already run every other GPU test; it passes alone in a fresh process as
well as after the others (every call writes the parts of the array it reads)."""
import numpy as np
import pytest

import kd_inputs as I

pytestmark = pytest.mark.gpu

TOL32 = 1e-5     # the fine-propagator tolerance used by the other GPU tests
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


def run_both(kd, params, b, t0, nsteps):
    import torch
    dtype = torch.complex64 if params.prec_fine == kd.KD_C64 else torch.complex128
    x = torch.tensor(b, dtype=dtype, device="cuda")
    tt = torch.tensor(np.asarray(t0, np.float64), device="cuda")
    ref = torch.empty_like(x)
    ctx = kd.kd_create(params)
    try:
        kd.kd_fine_batched(ctx, x, ref, tt, nsteps, b.shape[0], params.prec_fine)
        torch.cuda.synchronize()
    finally:
        kd.kd_destroy(ctx)
    out = torch.full_like(x, float("nan"))
    assert kd.kd_fine_batched_static(params, x, out, tt, nsteps, b.shape[0]) == kd.KD_OK
    torch.cuda.synchronize()
    return out.cpu().numpy(), ref.cpu().numpy()


def test_static_matches_fine_batched_on_two_calls_in_a_row(kd):
    # call 1: Galloway-Proctor 128^2, complex64, 3 fields (time-dependent flow phases)
    p1 = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, 128, 0.57, 100.0, 5e-3, kd.KD_C64)
    b1 = I.initial_batch(128, 0.57, [1, 2, 3])
    o1, r1 = run_both(kd, p1, b1, [0.0, 0.4, 2.2], 6)
    for i in range(3):
        assert rel(o1[i], r1[i]) < TOL32
    # call 2 right after, reusing the same scratch: Roberts 32^2, complex128, 2 fields
    p2 = kd.make_params(kd.KD_FLOW_ROBERTS, 32, 1.0, 8.0, 1e-2, kd.KD_C128)
    b2 = I.initial_batch(32, 1.0, [4, 5])
    o2, r2 = run_both(kd, p2, b2, [0.0, 1.0], 9)
    for i in range(2):
        assert rel(o2[i], r2[i]) < TOL64


def test_static_call_allocates_no_device_memory(kd):
    # the property the entry point exists for: once a first call has set the kernels up
    # on this device, calls leave the device's free memory exactly as it was
    import torch
    p = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, 64, 0.57, 100.0, 5e-3, kd.KD_C64)
    x = torch.tensor(I.initial_batch(64, 0.57, [7, 8]), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    tt = torch.tensor([0.0, 0.6], dtype=torch.float64, device="cuda")
    assert kd.kd_fine_batched_static(p, x, y, tt, 4, 2) == kd.KD_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert kd.kd_fine_batched_static(p, x, y, tt, 4, 2) == kd.KD_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_rejects_requests_beyond_the_scratch(kd):
    import torch
    p = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, 1024, 0.57, 1e4, 1e-3, kd.KD_C64)
    x = torch.zeros((8, 3, 1024, 1024), dtype=torch.complex64, device="cuda")
    t0 = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(kd.KdError) as err:
        kd.kd_fine_batched_static(p, x, x, t0, 2, 8)
    assert err.value.status == kd.KD_EINVAL
    assert not torch.isnan(x).any()
