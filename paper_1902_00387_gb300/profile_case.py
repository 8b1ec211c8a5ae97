"""Small, repeatable launches for profiling with ncu.

    python -m paper_1902_00387_gb300.profile_case --n 128 --batch 64 --steps 2 [--plan 0,3]

builds the library if needed, propagates `batch` seeded Galloway-Proctor fields by
`steps` fine steps once to warm up and once more (the launches to capture), and
prints the device time of the second call.

    python -m paper_1902_00387_gb300.profile_case --parareal

runs one Parareal solve of the GP 128^2, 64-slice workload of bench.py (plan
autotuned first), for a launch list of a whole solve.

    python -m paper_1902_00387_gb300.profile_case --coarse --n 128 --n-coarse 128 --steps 51 [--cluster 16] [--sync 0|1]

runs the classical coarse propagator (one thread-block cluster, kd_coarse) on one field
twice and prints the device time per RK443 stage of the second call.

    python -m paper_1902_00387_gb300.profile_case --gemm 4096,4096,4096 [--engine 0|1]

runs the BF16 training GEMM (kd_gemm_bf16_tn; engine 0 tcgen05, 1 mma.sync) on seeded
operands twice and prints the TFLOP/s of the second call.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--kz", type=float, default=0.57)
    ap.add_argument("--Rm", type=float, default=100.0)
    ap.add_argument("--dt", type=float, default=5e-3)
    ap.add_argument("--plan", default=None, help="column,row variant of the fine kernels")
    ap.add_argument("--parareal", action="store_true")
    ap.add_argument("--coarse", action="store_true")
    ap.add_argument("--n-coarse", type=int, default=128)
    ap.add_argument("--cluster", type=int, default=0, help="blocks per cluster of the coarse solver (0: default)")
    ap.add_argument("--sync", type=int, default=0, help="coarse halo exchange: 0 cluster barrier, 1 point-to-point")
    ap.add_argument("--gemm", default=None, help="M,N,K of a BF16 GEMM to run")
    ap.add_argument("--engine", type=int, default=0, help="GEMM engine: 0 tcgen05, 1 mma.sync")
    args = ap.parse_args()
    import torch

    import kd_inputs
    from paper_1902_00387_gb300 import build as b
    b.build()
    import paper_1902_00387_gb300 as kd
    kd.load()
    torch.cuda.init()
    if args.parareal:
        import math
        n, N, T = 128, 64, 2 * math.pi * 8
        p = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, n, 0.57, 100.0, 5e-3, kd.KD_C64, n_coarse=128,
                           dt_coarse=2.0 / 128, prec_coarse=kd.KD_C64, fine_form=kd.KD_FINE_INCREMENT)
        ctx = kd.kd_create(p)
        if args.plan:
            kd.kd_set_plan(ctx, kd.KD_GRID_FINE, *(int(v) for v in args.plan.split(",")))
        else:
            kd.kd_autotune(ctx, kd.KD_GRID_FINE, N, 2)
        b0 = torch.tensor(kd_inputs.initial_field(n, 0.57, 1000), device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s, st = kd.kd_parareal_run(ctx, b0, T, N, 64, 1e-6)
        e1.record()
        torch.cuda.synchronize()
        print("parareal GP 128^2 x 64 slices: %.1f ms, k_con %d, plan %s" % (e0.elapsed_time(e1), st.k_con,
                                                                            kd.kd_get_plan(ctx)))
        kd.kd_destroy(ctx)
        return
    if args.gemm:
        M, N, K = (int(v) for v in args.gemm.split(","))
        g = torch.Generator(device="cuda").manual_seed(1)
        A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
        Bt = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
        C = torch.empty(M, N, device="cuda")
        kd.kd_gemm_bf16_tn(A, Bt, C, args.engine)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        kd.kd_gemm_bf16_tn(A, Bt, C, args.engine)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print("gemm %dx%dx%d engine %d: %.3f ms, %.1f TFLOP/s" % (M, N, K, args.engine, ms, 2.0 * M * N * K / ms / 1e9))
        return
    if args.coarse:
        p = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, args.n, args.kz, args.Rm, args.dt, kd.KD_C64,
                           n_coarse=args.n_coarse, dt_coarse=2.0 / args.n_coarse, prec_coarse=kd.KD_C64)
        ctx = kd.kd_create(p)
        if args.cluster:
            kd.kd_set_coarse_cluster(ctx, args.cluster)
        kd.kd_set_coarse_sync(ctx, args.sync)
        x = torch.tensor(kd_inputs.initial_batch(args.n, args.kz, [7]), dtype=torch.complex128, device="cuda")
        y = torch.empty_like(x)
        t0 = torch.zeros(1, dtype=torch.float64, device="cuda")
        kd.kd_coarse(ctx, x, y, t0, args.steps, 1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        kd.kd_coarse(ctx, x, y, t0, args.steps, 1)
        e1.record()
        torch.cuda.synchronize()
        print("coarse N_C=%d steps=%d cluster=%d sync=%d: %.3f ms, %.3f us per stage" % (
            args.n_coarse, args.steps, args.cluster, args.sync, e0.elapsed_time(e1),
            e0.elapsed_time(e1) * 1000 / (4 * args.steps)))
        kd.kd_destroy(ctx)
        return
    p = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, args.n, args.kz, args.Rm, args.dt, kd.KD_C64)
    ctx = kd.kd_create(p)
    if args.plan:
        c, r = (int(v) for v in args.plan.split(","))
        kd.kd_set_plan(ctx, kd.KD_GRID_FINE, c, r)
    x = torch.tensor(kd_inputs.initial_batch(args.n, args.kz, range(args.batch)), dtype=torch.complex64,
                     device="cuda")
    t0 = torch.arange(args.batch, dtype=torch.float64, device="cuda") * 0.785
    kd.kd_fine_batched(ctx, x, x, t0, args.steps, args.batch)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    kd.kd_fine_batched(ctx, x, x, t0, args.steps, args.batch)
    e1.record()
    torch.cuda.synchronize()
    print("n=%d batch=%d steps=%d: %.3f ms" % (args.n, args.batch, args.steps, e0.elapsed_time(e1)))
    kd.kd_destroy(ctx)


if __name__ == "__main__":
    main()
