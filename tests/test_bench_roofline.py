"""The roofline object of bench.py (host arithmetic, no GPU): the slice-product families are judged
against the larger of their tensor-pipe and HBM bounds, with the sustained BF16 peak for kernels
timed inside a step, and carry the ncu traffic only when a capture of the current kernel exists."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PK = {"hbm_gbs": 6700.0, "bf16_tflops": 1943.0, "bf16_tflops_sustained": 1720.0}


def prof(fam, ms, flops, nbytes, launches=10):
    fams = {k: {"ms": 0.0, "flops": 0.0, "launches": 0, "bytes": 0.0}
            for k in ("gemm_kernel", "oz_mma_kernel", "oz_atb_kernel", "oz_ab_kernel")}
    fams[fam] = {"ms": ms, "flops": flops, "launches": launches, "bytes": nbytes}
    return {"families": fams}


def test_tensor_bound_family_uses_the_sustained_peak_over_28_products():
    # 1 s of 30 TFLOP useful FP64-class work, few bytes: tensor bound at 30 / (1720 / 28)
    r = bench.roofline_entry(prof("oz_mma_kernel", 1000.0, 30e12, 1e9), 1000.0, 1, PK, "bf16")
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(1720.0 / 28) and r["frac"] == pytest.approx(30.0 / (1720.0 / 28))
    assert r["traffic"] is None                       # no capture of the current plane kernel


def test_hbm_bound_family_reports_bytes_over_copy_bandwidth():
    # 1 s moving 3.35 TB with little arithmetic: HBM bound at 0.5 of 6700 GB/s
    r = bench.roofline_entry(prof("oz_ab_kernel", 1000.0, 1e12, 3.35e12), 2000.0, 1, PK, "bf16")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(3350.0) and r["frac"] == pytest.approx(0.5)
    assert r["kernel_share_of_step"] == pytest.approx(0.5)
    assert r["traffic"] == bench.NCU_TRAFFIC["oz_ab_kernel"]["bytes"]
    assert r["tensor_frac"] == pytest.approx(28 * 1e12 / 1720e12)
