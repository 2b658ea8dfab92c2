"""bench.py's roofline object from given launch timings, on the CPU.

The roofline of each stencil form is arithmetic on the profiled launches: the
algorithmic bytes (or FP64 flops) of one launch over its mean CUDA-event time,
and the ncu DRAM bytes of that kernel as `traffic`.  These checks feed
roofline() a workload object and launch timings and recompute each figure by
hand:
- native FP64 (the headline): bound "alu", FP64 flops a point weighted 21 for
  the exact-norm launches and 17 for the bracketed ones, against the derived
  FP64 peak; the HBM figures at 72 B a point-iteration beside it;
- the float-float form: bound "hbm" at 72 B a point-iteration, two iterations
  a launch, the pair kernel's DRAM bytes as traffic;
- a constant operator (the combustion step): 32 B a point-iteration; when the
  launches read the coefficient table the stored count is 32 B and the
  traffic the table kernel's, else 88 B and the array kernel's.
No GPU, no library calls.
"""
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

NPTS = 256 ** 3
ARGS = SimpleNamespace(steps=20)


def _wl(cls, **attrs):
    wl = object.__new__(cls)
    for k, v in attrs.items():
        setattr(wl, k, v)
    return wl


def _run(prof_ms, prof_n, fused, st, prof_bounded=0):
    return {"prof_ms": prof_ms, "prof_n": prof_n, "fused": fused, "prof_bytes": 0,
            "last": st, "prof_bounded": prof_bounded}


def test_native_headline_roofline():
    wl = _wl(bench.Adr3d, arith=1, dtype="f64", bytes_per_point=bench.BYTES_PER_POINT)
    avg_us, n, nb = 325.0, 46, 45
    out = bench.roofline(wl, _run(avg_us * n / 1e3, n, 1, SimpleNamespace(), nb), ARGS, NPTS)
    fpp = (21.0 * (n - nb) + 17.0 * nb) / n
    peak = bench.SMS * bench.FP64_FLOPS_PER_SM_CLK * bench.peaks_sm_mhz() * 1e6 / 1e12
    tf = fpp * NPTS / (avg_us * 1e-6) / 1e12
    assert out["bound"] == "alu" and out["unit"] == "TFLOP/s"
    assert out["flops_per_point"] == pytest.approx(fpp)
    assert out["achieved"] == pytest.approx(tf)
    assert out["peak"] == pytest.approx(peak)
    assert out["frac"] == pytest.approx(tf / peak)
    assert out["traffic"] == pytest.approx(bench.NATIVE_DRAM_BYTES_PER_POINT * NPTS)
    hbm, _ = bench.peaks()
    hb = out["hbm"]
    assert hb["bytes_per_point"] == 72
    assert hb["achieved"] == pytest.approx(72.0 * NPTS / (avg_us * 1e-6) / 1e9)
    assert hb["frac"] == pytest.approx(hb["achieved"] / hbm)


def test_float_float_form_roofline():
    wl = _wl(bench.Adr3dFF, arith=0, dtype=bench.DTYPE_FF, bytes_per_point=bench.BYTES_PER_POINT)
    avg_us, n = 413.0, 46
    out = bench.roofline(wl, _run(avg_us * n / 1e3, n, 2, SimpleNamespace()), ARGS, NPTS)
    hbm, _ = bench.peaks()
    alg = 72.0 * NPTS * 2 / (avg_us * 1e-6) / 1e9
    assert out["bound"] == "hbm" and out["unit"] == "GB/s"
    assert out["achieved"] == pytest.approx(alg)
    assert out["frac"] == pytest.approx(alg / hbm)
    assert out["iterations_per_launch"] == 2
    assert out["us_per_iteration"] == pytest.approx(avg_us / 2)
    assert out["traffic"] == pytest.approx(bench.PAIR_DRAM_BYTES_PER_POINT * NPTS)


@pytest.mark.parametrize("table", [True, False])
def test_constant_operator_roofline(table):
    wl = _wl(bench.Combustion3d, arith=0, dtype=bench.DTYPE_FF,
             bytes_per_point=bench.CONST_BYTES_PER_POINT,
             bytes_per_point_stored=bench.BYTES_PER_POINT)
    avg_us, n = 327.0, 21
    st = SimpleNamespace(coef_table=n if table else 0)
    out = bench.roofline(wl, _run(avg_us * n / 1e3, n, 2, st), ARGS, NPTS)
    hbm, _ = bench.peaks()
    alg = 32.0 * NPTS * 2 / (avg_us * 1e-6) / 1e9
    assert out["achieved"] == pytest.approx(alg)
    assert out["frac"] == pytest.approx(alg / hbm)
    stored = 32 if table else 88
    assert out["bytes_per_point_stored"] == stored
    assert out["frac_stored"] == pytest.approx(stored * NPTS / (avg_us * 1e-6) / 1e9 / hbm)
    per_pt = (bench.TABLE_PAIR_DRAM_BYTES_PER_POINT if table
              else bench.PAIR_DRAM_BYTES_PER_POINT)
    assert out["traffic"] == pytest.approx(per_pt * NPTS)
    assert ("coefficient table" in out["kernel"]) == table
