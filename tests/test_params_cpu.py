"""Host-side argument checks of the C ABI: kd_create rejects every invalid parameter set
with KD_EINVAL before it makes any CUDA call, so these run without a GPU."""
import math

import pytest


@pytest.fixture(scope="module")
def kd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_00387_gb300 as kd
    kd.load()
    return kd


BASE = dict(flow=1, n=64, kz=0.57, Rm=100.0, dt_fine=5e-3, prec_fine=0, n_coarse=32, dt_coarse=0.02,
            prec_coarse=0, coarse_kind=0, learned_modes=0, fine_form=0, fine_operator=0, fine_scheme=0)

BAD = [
    ("flow", 3), ("flow", -1),
    ("n", 8), ("n", 15), ("n", 2048), ("n", 97), ("n", 1026), ("n", 288), ("n", 1000),
    ("n_coarse", 17), ("n_coarse", 128), ("n_coarse", 8),
    ("Rm", 0.0), ("Rm", -1.0), ("Rm", math.inf), ("Rm", math.nan), ("kz", math.nan),
    ("dt_fine", 0.0), ("dt_coarse", -0.1), ("dt_fine", math.nan),
    ("prec_fine", 2), ("prec_coarse", -1),
    ("coarse_kind", 5),
    ("learned_modes", 1), ("learned_modes", 65), ("learned_modes", 48),   # 48 / 2 > 64 / 3
    ("fine_form", 7), ("fine_operator", 9), ("fine_scheme", 9),
]


def params(kd, **over):
    d = dict(BASE, **over)
    return kd.kd_params(*(d[name] for name, _ in kd.kd_params._fields_))


@pytest.mark.parametrize("field,value", BAD)
def test_invalid_parameters_are_rejected_on_the_host(kd, field, value):
    with pytest.raises(kd.KdError) as e:
        kd.kd_create(params(kd, **{field: value}), stream=0)
    assert e.value.status == kd.KD_EINVAL


@pytest.mark.parametrize("over", [
    dict(coarse_kind=1, learned_modes=16, fine_form=0),   # learned coarse needs the increment form
    dict(coarse_kind=1, learned_modes=0, fine_form=1),    # ... and a mode set
    dict(fine_operator=1, fine_scheme=1),                 # the convolution operator steps with RK443
])
def test_inconsistent_combinations_are_rejected_on_the_host(kd, over):
    with pytest.raises(kd.KdError) as e:
        kd.kd_create(params(kd, **over), stream=0)
    assert e.value.status == kd.KD_EINVAL


def test_null_arguments(kd):
    lib = kd.load()
    import ctypes
    out = ctypes.c_void_p()
    assert lib.kd_create(None, None, ctypes.byref(out)) == kd.KD_EINVAL
    assert lib.kd_create(ctypes.byref(params(kd)), None, None) == kd.KD_EINVAL
    assert lib.kd_destroy(None) == kd.KD_OK
    assert kd.kd_last_error(None) == "NULL context"
    assert kd.kd_version().startswith("kd ")


def test_static_entry_refuses_oversized_requests_on_the_host(kd):
    """kd_fine_batched_static bounds every workspace term before summing them, so sizes
    whose byte counts would wrap a 64-bit sum are refused with KD_EINVAL before any CUDA
    call (the pointers here are never dereferenced)."""
    import ctypes
    lib = kd.load()
    fake = ctypes.c_void_p(256)
    gp = params(kd)
    gp.n = 16
    # 2^30 fields x 2^30 steps: the phase table alone is 2^66 bytes (0 modulo 2^64);
    # 2^31 - 1 fields x 1879047834 steps at n = 16: the six terms sum to 1536 modulo 2^64
    for batch, nsteps in [(1 << 30, 1 << 30), (2**31 - 1, 1879047834), (2**31 - 1, 2**31 - 1), (1, 2**31 - 1),
                          (11556, 1)]:
        assert lib.kd_fine_batched_static(ctypes.byref(gp), fake, fake, fake, nsteps, batch, None) == kd.KD_EINVAL


def test_allocation_limit_calls_need_a_context(kd):
    """kd_set_alloc_limit / kd_get_alloc_bytes are host-only; without a context they
    return KD_EINVAL, and the binding refuses a negative limit before the library."""
    import ctypes
    lib = kd.load()
    held = ctypes.c_size_t(7)
    assert lib.kd_set_alloc_limit(None, 1 << 20) == kd.KD_EINVAL
    assert lib.kd_get_alloc_bytes(None, ctypes.byref(held), None) == kd.KD_EINVAL
    assert held.value == 7
    with pytest.raises(ValueError):
        kd.kd_set_alloc_limit(ctypes.c_void_p(16), -1)


def test_binding_rejects_short_buffers_before_the_library(kd, monkeypatch):
    """The binding knows each context's grid side and refuses buffers smaller than the
    fields the call will touch (the library takes plain pointers); nothing reaches the
    library here (a fake context address is registered, no CUDA call is made)."""
    import ctypes
    import numpy as np
    n = 16
    fake = ctypes.c_void_p(0x1000)
    monkeypatch.setitem(kd.kd._CTX_N, fake.value, n)

    class Trap:
        def __getattr__(self, name):
            raise AssertionError("library called: " + name)
    monkeypatch.setattr(kd.kd, "load", lambda: Trap())
    field = np.zeros((3, n, n), np.complex128)
    short = np.zeros((3, n, n - 1), np.complex128)
    slices = np.zeros((5, 3, n, n), np.complex128)
    t0 = np.zeros(4)
    cases = [
        lambda: kd.kd_parareal_run(fake, short, 1.0, 4, 4, 0.0),
        lambda: kd.kd_parareal_run(fake, field, 1.0, 5, 4, 0.0, slices),        # needs 6 slices
        lambda: kd.kd_parareal_resume(fake, slices, 1, 1.0, 5, 4, 0.0),
        lambda: kd.kd_fine_serial(fake, field, 1.0, 5, slices),
        lambda: kd.kd_set_reference(fake, short),
        lambda: kd.kd_energy(fake, slices, 6, np.zeros(6)),
        lambda: kd.kd_energy(fake, slices, 5, np.zeros(4)),
        lambda: kd.kd_growth_rate(fake, slices, 6, 1.0, 0.5),
        lambda: kd.kd_growth_power(fake, short, 0.0, 1.0, 10, 1e-6),
        lambda: kd.kd_growth_arnoldi(fake, field, 0.0, 1.0, 8, 2, 2, 1e-6, b_out=short),
        lambda: kd.kd_coarse(fake, slices, slices, t0, 2, 6),
        lambda: kd.kd_coarse(fake, slices, slices, t0, 2, 5),                   # t0 holds 4 times
    ]
    for i, call in enumerate(cases):
        with pytest.raises(ValueError):
            call()
    # the right sizes pass the checks and reach the library
    with pytest.raises(AssertionError, match="library called"):
        kd.kd_parareal_run(fake, field, 1.0, 4, 4, 0.0, slices)
