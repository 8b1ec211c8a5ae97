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
    ("n", 8), ("n", 15), ("n", 2048),
    ("n", 96),                                  # not a power of two with the FFT operator
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
