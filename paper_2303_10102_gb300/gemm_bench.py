"""Shape study of the FP64-class digit-slice product (hodlr_dgemm_slices) on one GPU.

    python -m paper_2303_10102_gb300.gemm_bench --shape M,N,K,batch,tA,tB [--shape ...] [--iters I] [--plan P,T,C]

For each shape the product C = A B (+ C when --beta 1) of random FP64 operands runs `iters` times
after one warm-up call, timed with CUDA events on the library's stream around the whole call
(slicing passes, tensor-core products, split-K reduction).  Printed per shape: milliseconds per
call, the FP64-equivalent rate 2 M N K batch / t, and the FP64 operand bytes (A, B, and C read
and written) over t; both against the measured peaks the library's own microbenchmark gives
(hodlr_peak: BF16 tensor pipe / 28 digit products, and the copy bandwidth passed in --hbm-gbs).
The shapes of the HODLR construction are the defaults: short-K peeling updates (A B, K = rank),
long-K Gram and projection products (A^T B, K = block size) and the DST of the 2-D physics.
"""
from __future__ import annotations

import argparse
import ctypes
import json

DEFAULT_SHAPES = ["524288,136,64,1,0,0", "131072,136,45,4,0,0", "64,136,524288,1,1,0", "45,136,131072,4,1,0",
                  "1024,16416,1024,1,0,0"]


def main(argv=None):
    import torch

    from . import lib as plib

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--shape", action="append", default=None, help="M,N,K,batch,tA,tB")
    ap.add_argument("--iters", type=int, default=5)
    ap.add_argument("--beta", type=float, default=1.0)
    ap.add_argument("--work-mb", type=int, default=2048)
    ap.add_argument("--hbm-gbs", type=float, default=None, help="copy bandwidth for the HBM fraction")
    ap.add_argument("--plan", default=None, help="path,tile,cprx (hodlr_dgemm_slices_plan); default automatic")
    args = ap.parse_args(argv)
    lib = plib.load()
    if args.plan:
        if lib.hodlr_dgemm_slices_plan(*(int(x) for x in args.plan.split(","))) != 0:
            raise ValueError(f"bad plan {args.plan}")
    dev = "cuda:0"
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    pk = ctypes.c_double(0.0)
    if lib.hodlr_peak(3, ctypes.byref(pk)) != 0:
        raise RuntimeError("hodlr_peak failed")
    bf16 = pk.value
    work = torch.empty(args.work_mb << 20, dtype=torch.uint8, device=dev)
    gen = torch.Generator(device=dev).manual_seed(0)
    for s in args.shape or DEFAULT_SHAPES:
        M, N, K, nb, tA, tB = (int(x) for x in s.split(","))
        A = torch.randn(nb * M * K, dtype=torch.float64, device=dev, generator=gen)
        B = torch.randn(nb * K * N, dtype=torch.float64, device=dev, generator=gen)
        C = torch.randn(nb * M * N, dtype=torch.float64, device=dev, generator=gen)
        lda, ldb = (K if tA else M), (N if tB else K)
        st = ctypes.c_void_p(stream.cuda_stream)

        def call():
            rc = lib.hodlr_dgemm_slices(M, N, K, nb, ctypes.c_void_p(A.data_ptr()), lda, M * K, tA,
                                        ctypes.c_void_p(B.data_ptr()), ldb, K * N, tB, 0, 1.0, args.beta,
                                        ctypes.c_void_p(C.data_ptr()), M, M * N, ctypes.c_void_p(work.data_ptr()),
                                        work.numel(), st)
            if rc != 0:
                raise RuntimeError(f"hodlr_dgemm_slices returned {rc} for {s}")

        torch.cuda.synchronize()
        call()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for _ in range(args.iters):
            ev0.record(stream)
            call()
            ev1.record(stream)
            ev1.synchronize()
            ms += ev0.elapsed_time(ev1)
        ms /= args.iters
        flops = 2.0 * M * N * K * nb
        byts = 8.0 * nb * (M * K + K * N + M * N * (2 if args.beta != 0.0 else 1))
        row = {"shape": s, "ms": round(ms, 4), "fp64_tflops": round(flops / ms / 1e9, 2),
               "frac_bf16_pipe": round(flops * 28 / ms / 1e9 / bf16, 3), "operand_gbs": round(byts / ms / 1e6, 1)}
        if args.hbm_gbs:
            row["frac_hbm"] = round(byts / ms / 1e6 / args.hbm_gbs, 3)
        print(json.dumps(row), flush=True)
        del A, B, C


if __name__ == "__main__":
    main()
