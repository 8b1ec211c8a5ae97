"""Slice blocks of the multi-rank Parareal (kd_block_*) driven by the pipeline schedule:
ranks run as threads of one process on one GPU, each with its own context and stream,
exchanging boundary states through host queues (the kernels of different ranks never
wait on one another).  The result equals the single-GPU kd_parareal_run bit for bit and
the oracle's serial fine solution to FP32 accuracy."""
import queue
import threading

import numpy as np
import pytest

import kd_inputs as I
from oracle import kd_oracle as O

pytestmark = pytest.mark.gpu

N_GRID, KZ, RM, DT, DTC, NC = 32, 0.57, 100.0, 5e-3, 0.05, 16
T, N_SLICES = 2.0, 8


@pytest.fixture(scope="module")
def kd():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_00387_gb300 as kd
    kd.load()
    torch.cuda.init()
    return kd


class LoopComm:
    """Host-queue messages between the rank threads of one process."""

    def __init__(self, world):
        self.q = {(a, b): queue.Queue() for a in range(world) for b in range(world)}
        self.world = world
        self.rank = None

    def bind(self, rank):
        c = LoopComm.__new__(LoopComm)
        c.q, c.world, c.rank = self.q, self.world, rank
        return c

    def send(self, buf, dst):
        self.q[(self.rank, dst)].put(buf.detach().clone())

    def recv(self, buf, src):
        buf.copy_(self.q[(src, self.rank)].get(timeout=120))

    def bcast_scalar(self, value, root, like):
        if self.rank == root:
            for r in range(self.world):
                if r != root:
                    self.q[(root, r)].put(value)
            return value
        return self.q[(root, self.rank)].get(timeout=120)


def params(kd):
    return kd.make_params(O.GALLOWAY_PROCTOR, N_GRID, KZ, RM, DT, kd.KD_C64, n_coarse=NC, dt_coarse=DTC,
                          prec_coarse=kd.KD_C64, fine_form=kd.KD_FINE_INCREMENT)


def run_ranks(kd, world, b0, k_max, tol):
    import torch
    from paper_1902_00387_gb300 import pipeline
    comm = LoopComm(world)
    out, errs = [None] * world, []

    def body(rank):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                ctx = kd.kd_create(params(kd), st.cuda_stream)
                try:
                    blk = pipeline.LibBlock(kd, ctx)
                    res = pipeline.parareal_pipeline(blk, comm.bind(rank), rank, world, b0, T, N_SLICES, k_max, tol)
                    nl = res["hi"] - res["lo"]
                    U = torch.zeros((nl + 1, 3, N_GRID, N_GRID), dtype=torch.complex128, device="cuda")
                    for i in range(nl + 1):
                        kd.kd_block_get_state(ctx, i, U[i])
                    res["U"] = U.cpu().numpy()
                    out[rank] = res
                finally:
                    kd.kd_destroy(ctx)
        except Exception as e:   # reported by the main thread
            errs.append(e)

    th = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errs, errs
    return out


def single_gpu(kd, b0, k_max, tol):
    ctx = kd.kd_create(params(kd))
    try:
        U = np.zeros((N_SLICES + 1, 3, N_GRID, N_GRID), np.complex128)
        s, st = kd.kd_parareal_run(ctx, b0, T, N_SLICES, k_max, tol, U)
        return U, st
    finally:
        kd.kd_destroy(ctx)


@pytest.mark.parametrize("world", [1, 2, 3])
def test_blocks_reproduce_single_gpu_parareal(kd, world):
    b0 = I.initial_field(N_GRID, KZ, 77)
    ref, st = single_gpu(kd, b0, 3, 0.0)
    out = run_ranks(kd, world, b0, 3, 0.0)
    for o in out:
        assert o["k_con"] == 3 and len(o["sigma"]) == 3
        assert np.array_equal(o["U"], ref[o["lo"]:o["hi"] + 1])
        assert o["sigma"] == list(st.sigma[:3])


def test_blocks_reach_the_serial_fine_solution(kd):
    """After N iterations (finite termination) the last slice is the serial fine state."""
    b0 = I.initial_field(N_GRID, KZ, 78)
    out = run_ranks(kd, 2, b0, N_SLICES, 0.0)
    ref, st = single_gpu(kd, b0, N_SLICES, 0.0)
    assert out[-1]["sigma"] == list(st.sigma[:N_SLICES])
    prob = O.Problem(O.GALLOWAY_PROCTOR, N_GRID, KZ, RM)
    S = int(np.ceil((T / N_SLICES) / DT - 1e-9))
    ser = O.serial_fine(b0, lambda u, n: O.propagate(u, prob, n * T / N_SLICES, T / N_SLICES / S, S), N_SLICES)
    last = out[-1]["U"][-1]
    assert np.linalg.norm(last - ser[-1]) / np.linalg.norm(ser[-1]) < 2e-5


def test_block_argument_errors(kd):
    ctx = kd.kd_create(params(kd))
    try:
        with pytest.raises(kd.KdError):
            kd.kd_block_fine(ctx, 1)                 # before kd_block_init
        with pytest.raises(kd.KdError):
            kd.kd_block_init(ctx, 6, 4, T, N_SLICES)  # block beyond the last slice
        kd.kd_block_init(ctx, 0, 4, T, N_SLICES)
        with pytest.raises(kd.KdError):
            kd.kd_block_fine(ctx, 0)
    finally:
        kd.kd_destroy(ctx)
