"""Host-side work models of bench.py (no GPU): the tensor-core formation counts agree with the
library's partition (interface slots per subdomain) and with a chunk-by-chunk enumeration of the
kernel's layer products (8 complex K values per operand chunk, two 8-wide K steps per full chunk)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_1312_5653_gb300 import schur as S  # noqa: E402


@pytest.mark.parametrize("N,P", [(128, 16), (64, 8), (32, 8), (24, 4)])
def test_tc_form_columns_match_partition(N, P):
    cnt = bench.tc_form_counts(N, P)
    info = S.schur_partition(3, N, P)
    assert cnt["ncol"] == info["n_delta"] + 8
    assert info["n_local"] == (N // P + 1) ** 3


@pytest.mark.parametrize("N,P", [(128, 16), (64, 8), (32, 8)])
def test_tc_form_executed_flops_by_enumeration(N, P):
    cnt = bench.tc_form_counts(N, P)
    s = N // P
    b, L = (s + 1) ** 2, s + 1
    steps = 0
    for c in range((b + 7) // 8):  # operand chunks of one layer product
        left = 2 * (b - 8 * c)
        steps += 2 if left >= 16 else (left + 7) // 8
    assert steps == cnt["ksteps"]
    per_mma = 2 * 128 * cnt["nb"] * 8
    assert cnt["executed"] == P ** 3 * cnt["ntile"] * (2 * L - 2) * steps * 3 * per_mma
    # 128^3 workload: 386 columns = 3 tensor-core tiles + 2 columns on the CUDA cores
    if (N, P) == (128, 16):
        assert (cnt["ncol"], cnt["ncol_tc"], cnt["ntile"], cnt["nb"]) == (386, 384, 3, 176)


def test_apply_models_count_packed_storage():
    """The HBM models of the local and coarse applies count the stored (packed) operators: the upper
    triangle of each symmetric nD x nD block, and for the coarse solve the level-0 blocks of the
    reduction and the upper 32 x 32 tiles of the reduced inverse."""
    info = S.schur_partition(2, 1024, 64)
    nsd, nD, nlam, nco = info["n_sub"], info["n_delta"], info["n_lambda"], info["n_coarse"]
    assert (nsd, nD, nco) == (4096, 60, 63 * 63)
    cb = 8
    _, f = bench.algorithmic("apply_F", info, 4)
    assert f == nsd * (1830 + 60 * 4) * cb + nlam * cb + nsd * 64 * cb
    _, sb = bench.algorithmic("apply_S", info, 4)
    assert sb == nsd * 1830 * cb + nlam * cb + nsd * 60 * cb
    # coarse solve: 63 layers, level 0 eliminates the 32 even layers (two without an outer
    # neighbour): 156 blocks of 63 x 63; the reduced matrix on 31 layers (1953 unknowns) as
    # 62 * 63 / 2 tiles; corner couplings read twice, two reduced vectors and the output
    _, c = bench.algorithmic("coarse_apply", info, 4)
    assert c == (156 * 63 * 63 + 62 * 63 // 2 * 1024 + 2 * nsd * 4 + 2 * 1953 + nco) * cb


def test_recorded_traffic_follows_the_kernel_sources(tmp_path):
    """A recorded ncu DRAM figure is used only while the kernel's sources hash to the recorded value."""
    k = "k_form_rr_cols<float, 17>"
    h = bench.kernel_source_hash(k)
    good = tmp_path / "t.md"
    good.write_text("| kernel | launches | dram bytes per launch | source hash |\n|---|---|---|---|\n"
                    "| `%s` | 3 | 1,234,567 | `%s` |\n" % (k, h))
    assert bench.recorded_traffic(k, str(good)) == 1234567.0
    stale = tmp_path / "s.md"
    stale.write_text("| `%s` | 3 | 1234567 | `0000000000000000` |\n" % k)
    assert bench.recorded_traffic(k, str(stale)) is None
    assert bench.recorded_traffic("k_other", str(good)) is None
    assert bench.recorded_traffic(k, str(tmp_path / "missing.md")) is None


def test_category_roofline_units():
    """HBM categories: bytes per launch / average launch time vs GB/s; ALU: flops per launch vs TFLOP/s."""
    info = S.schur_partition(2, 1024, 64)
    peaks = {"hbm_gbs": 6000.0, "fp32_fma": 60.0, "fp64_fma": 1.0}
    r = bench.category_roofline("apply_F", info, 100, 2.0, 1, peaks)  # 100 launches, 20 us each
    _, byts = bench.algorithmic("apply_F", info, 4)
    assert r["bound"] == "hbm" and abs(r["achieved"] - byts / 20e-6 / 1e9) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 6000.0) < 1e-12
    f = bench.category_roofline("form", info, 2, 2.0, 2, peaks)  # one launch per step, 1 ms each
    _, flops = bench.algorithmic("form", info, 4)
    assert f["bound"] == "alu" and abs(f["achieved"] - flops / 1e-3 / 1e12) < 1e-9 * f["achieved"]
    assert f["peak"] == 60.0 and f["algorithmic_bytes_per_launch"] > 0
