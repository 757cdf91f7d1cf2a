"""The arithmetic peak probes that the bench divides by (schur_peak_probe): each runs, reports a
positive rate, and the rates are ordered as the hardware's units are (FP32 FMA far above FP64 FMA,
the TF32 tensor pipe above FP32 FMA).  The bounds are loose physical limits of one GB300 (152 SMs
at up to 2.07 GHz), not tuning targets."""
import pytest

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1312_5653_gb300 import schur as S


def test_peak_probes_run_and_are_ordered():
    r = {name: S.schur_peak_probe(kind, {0: 20, 1: 200, 2: 20, 3: 5000}[kind]) for kind, name in S.PEAK_KINDS.items()}
    for name, v in r.items():
        assert v > 0, (name, v)
    # FP32: 152 SMs x 128 lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s is the ceiling
    assert 10.0 < r["fp32_fma"] <= 81.0, r
    assert r["fp64_fma"] < r["fp32_fma"], r
    assert r["tf32_tcgen05"] > r["fp32_fma"], r


def test_peak_probe_rejects_bad_arguments():
    with pytest.raises(S.SchurError):
        S.schur_peak_probe(7, 10)
    with pytest.raises(S.SchurError):
        S.schur_peak_probe(0, 0)
