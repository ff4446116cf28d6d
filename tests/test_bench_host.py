"""Host-side arithmetic of the benchmark (no GPU): the algorithmic byte counts behind the roofline
fractions, checked against brute-force counts of the coefficient sets; and the oracle arm's JSON
line (`bench.py --impl reference`), which runs the FP64 oracle on the host cores."""
import itertools
import json
import os
import subprocess
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def count_multi(dim, bound):
    """Multi-indices of `dim` non-negative entries with total at most `bound`, by enumeration."""
    return sum(1 for e in itertools.product(range(bound + 1), repeat=dim) if sum(e) <= bound)


@pytest.mark.parametrize("order,levels,grid", [(6, 5, 64), (4, 3, 16), (8, 5, 64), (1, 2, 8)])
def test_separable_bytes_match_enumeration(order, levels, grid):
    """Per transform: pass X reads the P-row and writes the 4-indexed rows, pass Y reads and writes
    4-indexed rows, pass Z reads 4-indexed rows and writes the P-row; one chain of intermediates
    at the finest level, two above it.  P and the 4-indexed size from enumeration."""
    P = count_multi(3, order)
    Q4 = count_multi(4, order)
    want = 0
    for l in range(levels):
        cells = (grid >> l) ** 3
        ch = 1 if l == 0 else 2
        floats = (P + ch * Q4) + (2 * ch * Q4) + (ch * Q4 + P)
        want += 4 * cells * floats
    assert bench.separable_bytes(P, levels, grid) == want


def test_m2l_algorithmic_bytes_at_the_bench_size():
    """Moments read once and locals written once over the five levels of 64^3 at order 6:
    299,584 cells x 84 values x 4 bytes x 2."""
    import bench
    cells = sum((64 >> l) ** 3 for l in range(5))
    assert cells == 299_584
    assert bench.m2l_algorithmic_bytes(84, 5, 64) == cells * 84 * 4 * 2 == 201_320_448


def test_separable_bytes_at_the_bench_size():
    # 64^3, order 6, five levels: 1.334 GB per transform (2.667 GB per step of two transforms)
    assert bench.separable_bytes(84, 5, 64) == 1_333_721_088


def _measured(order, levels, stage_ms):
    m = types.SimpleNamespace()
    m.info = {"coefficients": count_multi(3, order), "levels": levels}
    m.stage_ms = stage_ms
    return m


def test_stage_bytes_two_level_l2p():
    """Few targets per finest cell: L2L stops at level 1 and L2P also reads the level-1 rows."""
    wl = types.SimpleNamespace(grid=8, order=2, N=100, M=200)
    m = _measured(2, 2, {"sort": 1.0, "p2m": 1.0, "m2m": 1.0, "l2l": 1.0, "l2p": 1.0})
    out = bench.stage_roofline(m, wl, {"hbm_gbs": 1000.0})
    row = 4 * 12                                      # P = 10 at order 2, padded to 12
    G0, G1 = 8 ** 3, 4 ** 3
    assert out["m2m"]["bytes_per_step"] == 2 * row * (G0 + G1)
    assert "l2l" not in out or out["l2l"]["bytes_per_step"] == 0
    assert out["l2p"]["bytes_per_step"] == (16 * 200 + row * (G0 + G1) + 4 * 200) + \
        (16 * 100 + row * (G0 + G1) + 16 * 100)
    assert out["p2m"]["bytes_per_step"] == (16 * 100 + row * G0) + (16 * 200 + row * G0)
    # frac = bytes / time / peak
    assert out["p2m"]["frac_of_hbm"] == pytest.approx(out["p2m"]["bytes_per_step"] / 1e-3 / 1e9 / 1000.0)


def test_stage_bytes_full_l2l():
    """Many targets per finest cell (more than 8 at order 2): L2L runs down to the finest level."""
    G = [8 ** 3, 4 ** 3]
    wl = types.SimpleNamespace(grid=8, order=2, N=9 * G[0] + 1, M=9 * G[0] + 1)
    m = _measured(2, 2, {"l2l": 1.0, "l2p": 1.0})
    out = bench.stage_roofline(m, wl, {"hbm_gbs": 1000.0})
    row = 4 * 12
    assert out["l2l"]["bytes_per_step"] == 2 * row * (G[1] + 2 * G[0])
    assert out["l2p"]["bytes_per_step"] == (16 * wl.M + row * G[0] + 4 * wl.M) + \
        (16 * wl.N + row * G[0] + 16 * wl.N)


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference`: the oracle timed on the host cores on a bounded sample of the
    benchmark workload, one JSON line with the contract's keys."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, res.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0
    assert d["config"]["workload"] == "uniform3d"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_roofline_forms_and_traffic_keys():
    """The bench's roofline per M2L form: the CUDA-core forms (plain and occupied-cell) against the
    FP32 ALU peak derived from the SM clock, the separable form against HBM with the DRAM-traffic
    figure only where a capture of that form, grid and order exists, the tensor-core forms against
    the measured BF16 peak (TF32 scaled)."""
    import bench
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops_sustained": 1800.0, "sm_max_mhz": 2000.0}

    def meas(mode, grid=64, P=84, levels=5):
        m = bench.Measured()
        m.mode, m.grid = mode, grid
        m.stage_ms = {"m2l": 2.0}
        m.info = {"m2l_useful_flops": 1e11, "m2l_issued_flops": 3e11, "coefficients": P, "levels": levels}
        return m

    for mode in ("fp32", "occupied"):
        r = bench.roofline_for(meas(mode), peaks)
        assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
        assert abs(r["achieved"] - 2 * 1e11 / 2e-3 / 1e12) < 1e-9       # two transforms per step
        assert abs(r["peak"] - 152 * 128 * 2 * 2000e6 / 1e12) < 1e-6
    assert "k_m2l_occ" in bench.roofline_for(meas("occupied"), peaks)["kernel"]
    sep = bench.roofline_for(meas("separable"), peaks)
    assert sep["bound"] == "hbm" and sep["traffic"] == bench.M2L_TRAFFIC_BYTES[("separable", 64, 84)]
    assert bench.roofline_for(meas("separable", P=165, levels=5), peaks)["traffic"] is None   # order 8: no capture
    tf = bench.roofline_for(meas("tf32"), peaks)
    assert tf["bound"] == "tensor" and abs(tf["peak"] - 1800.0 * 1.1 / 2.25) < 1e-9 and tf["traffic"] is None
