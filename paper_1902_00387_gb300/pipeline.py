"""Parareal over several ranks: the paper's time communicator (Sec. 4.1, Algorithms 1-3).

Rank r owns the contiguous slices [lo_r, hi_r) of N.  Iteration 0 is the serial coarse
sweep passed from rank to rank; in iteration k >= 1 every rank takes its parallel step
(fine propagation of its slices, no communication), then the serial sweep runs through
the ranks: rank r receives U_{lo_r} from rank r - 1, sweeps its block and sends U_{hi_r}
to rank r + 1.  The rank holding the last slice measures the defect of Eq. 9 and
broadcasts it (8 bytes); every rank stops at the same iteration.

The per-rank work is done by a block object (the library's kd_block_* calls in
`LibBlock`); messages go through a communicator object (`TorchDistComm` for
torch.distributed, one GPU per rank over NCCL or host tensors over gloo).  This module
holds only the schedule: no arithmetic of the method.

Failure detection (the paper assumes reliable MPI): with a `timeout`, a rank that waits
longer than that for a boundary state, or whose send or defect broadcast fails (a peer
that failed or left; the process group's own timeout bounds the broadcast), raises
PipelineError naming the iteration and the peer instead of waiting forever.  A rank
leaves only between its steps, so no device work of its own is in flight then.

The receive timeout applies to host-side groups (gloo).  On an NCCL group a receive that
the host stops waiting for stays queued on the GPU, waiting for a peer that never sends,
so `TorchDistComm` refuses a receive timeout there: the bound on NCCL is the process
group's own timeout (init_process_group(timeout=...)), whose watchdog aborts the
communicator and fails the pending operation on the device as well; a failed send
surfaces through that watchdog too, not as an exception of the send call.
"""
import datetime
import math


class PipelineError(RuntimeError):
    """A rank gave up on a peer: a boundary state that never arrived or could not be sent,
    or a failed defect broadcast."""


def block_of(rank, world, n_slices):
    """Contiguous block [lo, hi) of slices owned by `rank` (sizes differ by at most one)."""
    lo = rank * n_slices // world
    hi = (rank + 1) * n_slices // world
    return lo, hi


class TorchDistComm:
    """Point-to-point boundary messages and the defect broadcast over torch.distributed.
    timeout (seconds, optional): how long a receive waits for its boundary state; not on
    an NCCL group, whose process-group timeout bounds every operation instead."""

    def __init__(self, group=None, timeout=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.timeout = timeout
        if timeout is not None and str(dist.get_backend(group)).lower() == "nccl":
            raise ValueError("a receive timeout would leave the NCCL receive queued on the GPU; bound NCCL "
                             "operations with the process group's timeout (init_process_group(timeout=...))")

    def send(self, buf, dst):
        try:
            self.dist.send(buf, dst, group=self.group)
        except RuntimeError as e:
            raise PipelineError("boundary state to rank %d failed: %s" % (dst, e)) from e

    def recv(self, buf, src):
        if self.timeout is None:
            self.dist.recv(buf, src, group=self.group)
            return
        req = self.dist.irecv(buf, src, group=self.group)
        try:
            done = req.wait(timeout=datetime.timedelta(seconds=self.timeout))
        except RuntimeError as e:
            raise PipelineError("no boundary state from rank %d within %.1f s" % (src, self.timeout)) from e
        if done is False:
            raise PipelineError("no boundary state from rank %d within %.1f s" % (src, self.timeout))

    def bcast_scalar(self, value, root, like):
        import torch
        t = torch.tensor([float(value)], dtype=torch.float64, device=like.device)
        try:
            self.dist.broadcast(t, root, group=self.group)
        except RuntimeError as e:
            raise PipelineError("defect broadcast from rank %d failed: %s" % (root, e)) from e
        return float(t.item())


class LibBlock:
    """A rank's slice block on its GPU through the library (kd_block_*)."""

    def __init__(self, kd, ctx, device="cuda"):
        self.kd, self.ctx, self.device = kd, ctx, device

    def init(self, lo, n_local, T, n_slices):
        self.kd.kd_block_init(self.ctx, lo, n_local, T, n_slices)

    def make_buffer(self):
        import torch
        return torch.empty(self.kd.kd_block_boundary_bytes(self.ctx) // 8, dtype=torch.float64, device=self.device)

    def set_initial(self, b0):
        self.kd.kd_block_set_initial(self.ctx, b0)

    def set_boundary(self, buf):
        self.kd.kd_block_set_boundary(self.ctx, buf)

    def get_boundary(self, buf):
        self.kd.kd_block_get_boundary(self.ctx, buf)

    def fine(self, k):
        self.kd.kd_block_fine(self.ctx, k)

    def sweep(self, k):
        return self.kd.kd_block_sweep(self.ctx, k)


def parareal_pipeline(block, comm, rank, world, b0, T, n_slices, k_max, tol):
    """Run Parareal for `rank` of `world`.  `b0` is used on rank 0 only.  Returns the
    rank's block bounds, the iteration count and the defect history (the same on every
    rank).  Raises FloatingPointError on a non-finite defect."""
    if world < 1 or not 0 <= rank < world or n_slices < world:
        raise ValueError("need 0 <= rank < world <= n_slices")
    lo, hi = block_of(rank, world, n_slices)
    block.init(lo, hi - lo, T, n_slices)
    if rank == 0:
        block.set_initial(b0)
    buf = block.make_buffer()
    last = world - 1

    def sweep(k):
        if rank > 0:
            comm.recv(buf, rank - 1)
            block.set_boundary(buf)
        s = block.sweep(k)
        if rank < last:
            block.get_boundary(buf)
            comm.send(buf, rank + 1)
        return s

    def step(k, fn):
        try:
            return fn()
        except PipelineError as e:
            raise PipelineError("rank %d, iteration %d: %s" % (rank, k, e)) from e

    step(0, lambda: sweep(0))
    sigmas = []
    k_con = k_max
    converged = False
    for k in range(1, k_max + 1):
        block.fine(k)
        s = step(k, lambda: comm.bcast_scalar(sweep(k), last, buf))
        sigmas.append(s)
        if not math.isfinite(s):
            raise FloatingPointError("non-finite Parareal defect at iteration %d" % k)
        if s <= tol:
            k_con, converged = k, True
            break
    return {"lo": lo, "hi": hi, "k_con": k_con if converged else min(k_max, len(sigmas)), "converged": converged,
            "sigma": sigmas}
