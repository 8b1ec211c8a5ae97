"""Batched sweep of independent Parareal instances (kd_sweep_run): per-instance parity
with the CPU oracle's Parareal and serial fine solutions, with instances of different
grids, flows, kz, Rm and step counts in one call."""
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


# (flow, n, kz, Rm, dt_fine, n_coarse, dt_coarse): two grids, both flows, uneven steps
INSTANCES = [
    (O.GALLOWAY_PROCTOR, 32, 0.57, 100.0, 0.02, 16, 0.05),
    (O.ROBERTS, 32, 1.0, 8.0, 0.025, 16, 0.05),
    (O.GALLOWAY_PROCTOR, 32, 1.3, 400.0, 0.0125, 16, 0.025),
    (O.ROBERTS, 16, 0.4, 60.0, 0.05, 16, 0.1),
    (O.GALLOWAY_PROCTOR, 16, 0.9, 20.0, 0.04, 16, 0.1),
]
T, N = 2.0, 4


def oracle_parareal(inst, b0, k_max, tol):
    flow, n, kz, Rm, dt, nc, dtc = inst
    prob = O.Problem(flow, n, kz, Rm)
    dT = T / N
    S, Sc = math.ceil(dT / dt - 1e-9), math.ceil(dT / dtc - 1e-9)
    fine = lambda u, i: O.propagate(u, prob, i * dT, dT / S, S)
    coarse = lambda u, i: O.coarse_propagate(u, prob, nc, i * dT, dT / Sc, Sc)
    return O.parareal(b0, fine, coarse, N, k_max, tol), O.serial_fine(b0, fine, N)


def run_sweep(kd, insts, seeds, k_max, tol, tune_cache=None):
    ins = [kd.make_instance(*x) for x in insts]
    b0 = [I.initial_field(x[1], x[2], s).astype(np.complex128) for x, s in zip(insts, seeds)]
    out = [np.zeros_like(b) for b in b0]
    status, res, st = kd.kd_sweep_run(ins, b0, T, N, k_max, tol, u_final=out, tune_cache=tune_cache)
    return status, res, st, b0, out


def test_sweep_matches_oracle_per_instance(kd):
    seeds = [101, 102, 103, 104, 105]
    status, res, st, b0, out = run_sweep(kd, INSTANCES, seeds, N, 1e-9)
    assert st.n_groups == 2
    for i, inst in enumerate(INSTANCES):
        par, ser = oracle_parareal(inst, b0[i], N, 1e-9)
        r = res[i]
        # defects of the first iterations are set by the method, not by rounding
        ks = min(r.k_con, par["k_con"], 3)
        for k in range(ks):
            if par["sigma"][k] > 1e-4:
                assert abs(r.sigma[k] - par["sigma"][k]) < 1e-3 * par["sigma"][k], (i, k, r.sigma[k], par["sigma"][k])
        # the final state is the serial fine solution at FP32 accuracy
        assert rel(out[i], ser[-1]) < 2e-5, (i, rel(out[i], ser[-1]))
        assert r.n_fine_steps == math.ceil((T / N) / inst[4] - 1e-9)


def test_sweep_iterates_match_oracle_iterates(kd):
    """k_max = 2 stops early: the state is the oracle's second Parareal iterate."""
    seeds = [201, 202, 203, 204, 205]
    status, res, st, b0, out = run_sweep(kd, INSTANCES, seeds, 2, 0.0)
    assert status == kd.KD_ENOTCONV
    for i, inst in enumerate(INSTANCES):
        par, _ = oracle_parareal(inst, b0[i], 2, 0.0)
        assert res[i].k_con == 2 and res[i].status == kd.KD_ENOTCONV
        assert rel(out[i], par["U"][-1]) < 2e-5, (i, rel(out[i], par["U"][-1]))


def test_sweep_single_instance_equals_parareal_run_order_of_magnitude(kd):
    """One GP instance alone: the sweep converges to the same tolerance as
    kd_parareal_run in the increment form, and both give the serial fine state."""
    inst = INSTANCES[0]
    status, res, st, b0, out = run_sweep(kd, [inst], [301], 16, 1e-6)
    assert status == kd.KD_OK and res[0].status == kd.KD_OK
    _, ser = oracle_parareal(inst, b0[0], 1, 0.0)
    assert rel(out[0], ser[-1]) < 2e-5
    assert res[0].sigma[res[0].k_con - 1] <= 1e-6


def test_sweep_with_autotuned_plan(kd, tmp_path):
    cache = str(tmp_path / "tune.json")
    seeds = [401, 402, 403, 404, 405]
    status, res, st, b0, out = run_sweep(kd, INSTANCES, seeds, N, 1e-9, tune_cache=cache)
    for i, inst in enumerate(INSTANCES):
        _, ser = oracle_parareal(inst, b0[i], 1, 0.0)
        assert rel(out[i], ser[-1]) < 2e-5
    import json
    assert len(json.load(open(cache))["entries"]) == 2    # one fine plan per group


def test_sweep_argument_errors(kd):
    ins = [kd.make_instance(*INSTANCES[0])]
    b0 = [I.initial_field(32, 0.57, 1).astype(np.complex128)]
    with pytest.raises(kd.KdError):
        kd.kd_sweep_run(ins, b0, T, 0, 4, 1e-6)
    bad = [kd.make_instance(O.ROBERTS, 48, 1.0, 8.0, 0.01, 16, 0.1)]
    with pytest.raises(kd.KdError):
        kd.kd_sweep_run(bad, b0, T, N, 4, 1e-6)


def test_sweep_object_repeats_and_graphs_change_no_value(kd):
    """A prepared sweep executed twice (the second exec replays the captured fine steps)
    and once without graphs gives kd_sweep_run's results bit for bit."""
    seeds = [501, 502, 503, 504, 505]
    ins = [kd.make_instance(*x) for x in INSTANCES]
    b0 = [I.initial_field(x[1], x[2], s).astype(np.complex128) for x, s in zip(INSTANCES, seeds)]
    ref = [np.zeros_like(b) for b in b0]
    s_ref, r_ref, _ = kd.kd_sweep_run(ins, b0, T, N, N, 1e-9, u_final=ref)
    sw = kd.Sweep(ins, T, N)
    try:
        runs = []
        for graphs in (True, True, False):
            sw.set_graphs(graphs)
            out = [np.zeros_like(b) for b in b0]
            s, res, st = sw.exec(b0, N, 1e-9, u_final=out)
            assert s == s_ref
            runs.append((out, res, st))
    finally:
        sw.close()
    for out, res, st in runs:
        for i in range(len(INSTANCES)):
            assert np.array_equal(out[i], ref[i]), i
            assert res[i].k_con == r_ref[i].k_con
            assert list(res[i].sigma[:res[i].k_con]) == list(r_ref[i].sigma[:r_ref[i].k_con])
    assert runs[0][2].n_launches == runs[1][2].n_launches == runs[2][2].n_launches


@pytest.mark.parametrize("n,flow", [(64, O.ROBERTS), (128, O.GALLOWAY_PROCTOR), (256, O.ROBERTS),
                                    (512, O.GALLOWAY_PROCTOR)])
def test_sweep_recipe_grid_sides_against_oracle(kd, n, flow):
    """One instance of each grid side of the Rm / kz sweep (Rm = 50 (n / 64)^2, the recipe's
    steps: GP dt = 0.128 / n, Roberts dt = 1.6 / n, coarse grid n / 2 with
    dt_c = min(20 dt (GP) or 10 dt (Roberts), 2 / n_c)), run to K = N on a short horizon:
    the final state is the oracle's serial fine solution at FP32 accuracy."""
    Rm, kz = 50.0 * (n / 64) ** 2, 0.8
    dt = 0.128 / n if flow == O.GALLOWAY_PROCTOR else 1.6 / n
    nc = n // 2
    dtc = min((20 if flow == O.GALLOWAY_PROCTOR else 10) * dt, 2.0 / nc)
    TT, NN = (0.02, 4) if flow == O.GALLOWAY_PROCTOR else (0.2, 4)
    ins = [kd.make_instance(flow, n, kz, Rm, dt, nc, dtc)]
    b0 = [I.initial_field(n, kz, 600 + n).astype(np.complex128)]
    out = [np.zeros_like(b0[0])]
    status, res, st = kd.kd_sweep_run(ins, b0, TT, NN, NN, 0.0, u_final=out)
    assert res[0].k_con == NN
    prob = O.Problem(flow, n, kz, Rm)
    dT = TT / NN
    S = res[0].n_fine_steps
    ser = O.serial_fine(b0[0], lambda u, i: O.propagate(u, prob, i * dT, dT / S, S), NN)
    assert rel(out[0], ser[-1]) < 2e-5, rel(out[0], ser[-1])
