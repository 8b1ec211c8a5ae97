"""Multi-rank Parareal schedule (paper_1902_00387_gb300.pipeline) on CPU ranks over gloo,
with oracle-backed slice blocks: every rank's slice states, the iteration count and the
defect history equal the single-process oracle Parareal bit for bit."""
import os
import socket

import numpy as np
import pytest

import kd_inputs as I
from oracle import kd_oracle as O

N_SLICES, T, N_GRID = 6, 1.2, 16


class OracleBlock:
    """A rank's slices with the oracle's propagators (Eq. 8 in the evaluation order
    F(U^k_n) + (G(U^{k+1}_n) - G(U^k_n)))."""

    def __init__(self, prob, dt, dtc, nc):
        self.prob, self.dt, self.dtc, self.nc = prob, dt, dtc, nc

    def init(self, lo, n_local, T, n_slices):
        import math
        self.lo, self.nl, self.N = lo, n_local, n_slices
        self.dT = T / n_slices
        self.S = math.ceil(self.dT / self.dt - 1e-9)
        self.Sc = math.ceil(self.dT / self.dtc - 1e-9)
        self.U = [None] * (n_local + 1)
        self.F = [None] * n_local
        self.G = [None] * n_local

    def fine_op(self, u, n):
        return O.propagate(u, self.prob, n * self.dT, self.dT / self.S, self.S)

    def coarse_op(self, u, n):
        return O.coarse_propagate(u, self.prob, self.nc, n * self.dT, self.dT / self.Sc, self.Sc)

    def make_buffer(self):
        import torch
        return torch.zeros(2 * 3 * N_GRID * N_GRID, dtype=torch.float64)

    def set_initial(self, b0):
        self.U[0] = np.array(b0, np.complex128)

    def set_boundary(self, buf):
        self.U[0] = buf.numpy().view(np.complex128).reshape(3, N_GRID, N_GRID).copy()

    def get_boundary(self, buf):
        import torch
        buf.copy_(torch.from_numpy(np.ascontiguousarray(self.U[self.nl]).view(np.float64).ravel()))

    def fine(self, k):
        for i in range(self.nl):
            self.F[i] = self.fine_op(self.U[i], self.lo + i)

    def sweep(self, k):
        prev = None if self.U[self.nl] is None else self.U[self.nl].copy()
        for i in range(self.nl):
            g = self.coarse_op(self.U[i], self.lo + i)
            self.U[i + 1] = g.copy() if k == 0 else self.F[i] + (g - self.G[i])
            self.G[i] = g
        if k >= 1 and self.lo + self.nl == self.N:
            return O.l2(self.U[self.nl] - prev) / O.l2(self.U[self.nl])
        return 0.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, k_max, tol, outdir):
    import torch.distributed as dist
    from paper_1902_00387_gb300 import pipeline
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = O.Problem(O.ROBERTS, N_GRID, 1.0, 8.0)
        blk = OracleBlock(prob, 0.02, 0.1, 16)
        b0 = I.initial_field(N_GRID, 1.0, 5)
        res = pipeline.parareal_pipeline(blk, pipeline.TorchDistComm(), rank, world, b0, T, N_SLICES, k_max, tol)
        np.savez(os.path.join(outdir, "rank%d.npz" % rank), U=np.stack(blk.U), lo=res["lo"], hi=res["hi"],
                 k_con=res["k_con"], sigma=np.array(res["sigma"]))
    finally:
        dist.destroy_process_group()


def _run(world, k_max, tol, tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, k_max, tol, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    return [dict(np.load(os.path.join(str(tmp_path), "rank%d.npz" % r))) for r in range(world)]


def _reference(k_max, tol):
    prob = O.Problem(O.ROBERTS, N_GRID, 1.0, 8.0)
    blk = OracleBlock(prob, 0.02, 0.1, 16)
    blk.init(0, N_SLICES, T, N_SLICES)
    b0 = I.initial_field(N_GRID, 1.0, 5)
    return O.parareal(b0, blk.fine_op, blk.coarse_op, N_SLICES, k_max, tol)


@pytest.mark.parametrize("world", [2, 3])
def test_pipeline_equals_single_process_parareal(world, tmp_path):
    out = _run(world, 3, 0.0, tmp_path)
    ref = _reference(3, 0.0)
    for r, o in enumerate(out):
        lo, hi = int(o["lo"]), int(o["hi"])
        assert (lo, hi) == (r * N_SLICES // world, (r + 1) * N_SLICES // world)
        assert np.array_equal(o["U"], np.stack(ref["U"][lo:hi + 1]))   # bit for bit
        assert np.array_equal(o["sigma"], np.array(ref["sigma"]))
        assert int(o["k_con"]) == 3


def test_pipeline_stops_at_tolerance_on_every_rank(tmp_path):
    tol = 1e-6
    ref = _reference(N_SLICES, tol)
    out = _run(2, N_SLICES, tol, tmp_path)
    assert ref["k_con"] < N_SLICES
    for o in out:
        assert int(o["k_con"]) == ref["k_con"]
        assert np.array_equal(o["sigma"], np.array(ref["sigma"]))


def test_block_bounds_cover_the_slices():
    from paper_1902_00387_gb300.pipeline import block_of
    for N in (1, 5, 64, 257):
        for world in range(1, min(N, 9) + 1):
            blocks = [block_of(r, world, N) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == N
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1


# ---- failure detection on the host: lost and late messages, a failing rank

class FaultyComm:
    """Wraps a communicator and injects faults on the host: `drop` = (rank, n) loses the
    n-th boundary state that rank sends; `delay` = (rank, seconds) holds every send of
    that rank back; `fail` = (rank, k) makes that rank's block raise in its fine step of
    iteration k (a rank that fails between steps)."""

    def __init__(self, inner, rank, drop=None, delay=None):
        self.inner, self.rank, self.drop, self.delay = inner, rank, drop, delay
        self.sent = 0

    def send(self, buf, dst):
        import time
        self.sent += 1
        if self.drop and self.drop == (self.rank, self.sent):
            return
        if self.delay and self.delay[0] == self.rank:
            time.sleep(self.delay[1])
        self.inner.send(buf, dst)

    def recv(self, buf, src):
        self.inner.recv(buf, src)

    def bcast_scalar(self, value, root, like):
        return self.inner.bcast_scalar(value, root, like)


class FailingBlock(OracleBlock):
    def __init__(self, *a, fail_at=None):
        super().__init__(*a)
        self.fail_at = fail_at

    def fine(self, k):
        if self.fail_at == k:
            raise MemoryError("injected host failure in the fine step of iteration %d" % k)
        super().fine(k)


def _faulty_rank_main(rank, world, port, fault, outdir):
    import datetime
    import json
    import torch.distributed as dist
    from paper_1902_00387_gb300 import pipeline
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=6))
    rec = {}
    try:
        prob = O.Problem(O.ROBERTS, N_GRID, 1.0, 8.0)
        blk = FailingBlock(prob, 0.02, 0.1, 16, fail_at=fault.get("fail", {}).get(str(rank)))
        comm = FaultyComm(pipeline.TorchDistComm(timeout=3.0), rank, drop=tuple(fault["drop"]) if "drop" in fault
                          else None, delay=tuple(fault["delay"]) if "delay" in fault else None)
        b0 = I.initial_field(N_GRID, 1.0, 5)
        res = pipeline.parareal_pipeline(blk, comm, rank, world, b0, T, N_SLICES, 3, 0.0)
        np.save(os.path.join(outdir, "U%d.npy" % rank), np.stack(blk.U))
        rec = {"ok": True, "sigma": res["sigma"]}
    except Exception as e:   # recorded for the test; the process then leaves cleanly
        rec = {"ok": False, "type": type(e).__name__, "msg": str(e)[:300]}
    finally:
        with open(os.path.join(outdir, "rank%d.json" % rank), "w") as f:
            json.dump(rec, f)
        dist.destroy_process_group()


def _run_faulty(fault, tmp_path, world=2, limit=60.0):
    import json
    import time
    import torch.multiprocessing as mp
    port = _free_port()
    t = time.time()
    ctx = mp.start_processes(_faulty_rank_main, args=(world, port, fault, str(tmp_path)), nprocs=world, join=False,
                             start_method="spawn")
    while not ctx.join(timeout=1.0):
        if time.time() - t > limit:
            for p in ctx.processes:     # the processes this test started, by handle
                if p.is_alive():
                    p.kill()
            raise AssertionError("a rank did not finish within %.0f s" % limit)
    out = [json.load(open(os.path.join(str(tmp_path), "rank%d.json" % r))) for r in range(world)]
    return out, time.time() - t


def test_late_boundary_state_changes_nothing(tmp_path):
    out, _ = _run_faulty({"delay": [0, 0.4]}, tmp_path)
    ref = _reference(3, 0.0)
    assert all(o["ok"] for o in out)
    for r in range(2):
        lo, hi = r * N_SLICES // 2, (r + 1) * N_SLICES // 2
        assert np.array_equal(np.load(os.path.join(str(tmp_path), "U%d.npy" % r)), np.stack(ref["U"][lo:hi + 1]))
        assert out[r]["sigma"] == list(ref["sigma"])


def test_lost_boundary_state_fails_every_rank_in_bounded_time(tmp_path):
    # rank 0's second send is the boundary state of iteration 1's serial sweep
    out, wall = _run_faulty({"drop": [0, 2]}, tmp_path)
    assert not out[0]["ok"] and not out[1]["ok"]
    assert out[1]["type"] == "PipelineError" and "iteration 1" in out[1]["msg"] and "rank 0" in out[1]["msg"]
    assert out[0]["type"] == "PipelineError" and "iteration 1" in out[0]["msg"]
    assert wall < 45


def test_failed_rank_is_detected_by_its_peer(tmp_path):
    out, wall = _run_faulty({"fail": {"1": 2}}, tmp_path)
    assert out[1] == {"ok": False, "type": "MemoryError",
                      "msg": "injected host failure in the fine step of iteration 2"}
    assert not out[0]["ok"] and out[0]["type"] == "PipelineError" and "iteration 2" in out[0]["msg"]
    assert wall < 45


def test_receive_timeout_refused_on_nccl_groups(monkeypatch):
    # a receive the host stops waiting for would stay queued on the GPU with NCCL, so the
    # communicator refuses the timeout there (the process group's own timeout bounds NCCL)
    import torch.distributed as dist
    from paper_1902_00387_gb300 import pipeline
    monkeypatch.setattr(dist, "get_backend", lambda group=None: "nccl")
    with pytest.raises(ValueError):
        pipeline.TorchDistComm(timeout=2.0)
    pipeline.TorchDistComm()                # no timeout: accepted
    monkeypatch.setattr(dist, "get_backend", lambda group=None: "gloo")
    assert pipeline.TorchDistComm(timeout=2.0).timeout == 2.0
