"""The benchmark's roofline bookkeeping on the CPU: the dense per-term counts
add up to the per-kernel and per-step figures the design tabulates at N = 4, the
algorithmic bytes are the state read and written plus the static record, and the
composite roofline divides the three parts by their own peaks."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_dense_counts_at_degree_4():
    terms = bench.hot_path_terms(4)
    # (contraction, pointwise) per element update of each term at N = 4 (L = 35, 125 volume
    # nodes, 25 face nodes, 5 time nodes)
    expect = {
        "ck_predictor": (294000, 84000),
        "damage_source_i1": (70000, 5000),
        "volume_evaluation": (306250, 71000),
        "volume_projection": (87500, 6750),
        "face_traces": (350000, 0),
        "rusanov_flux": (0, 72500),
        "face_projection": (70000, 0),
        "strain_rows": (22050, 0),
        "time_integration": (0, 3500),
    }
    assert {k: (c, p) for k, (_, c, p) in terms.items()} == expect
    kf = bench.kernel_flops(4)
    assert sum(c for c, _ in kf.values()) == 1199800
    assert sum(p for _, p in kf.values()) == 242750
    assert kf["corrector"] == (485800, 81250)
    assert bench.algorithmic_bytes(4) == 2976


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_kernels_cover_every_term(N):
    terms = bench.hot_path_terms(N)
    kf = bench.kernel_flops(N)
    assert set(kf) == {"predictor", "faces", "corrector"}
    assert sum(c for c, _ in kf.values()) == sum(c for _, c, _ in terms.values())
    assert sum(p for _, p in kf.values()) == sum(p for _, _, p in terms.values())


def test_composite_roofline():
    pk = {"tensor_3xtf32_tflops": 100.0, "alu_fp32_tflops": 50.0, "hbm_gbs": 1000.0}
    r = bench.composite(2e6, 1e6, 1000, 0.1, pk, bytes_=4000.0)
    # 2e9 / 100e12 + 1e9 / 50e12 + 4e6 / 1e12 seconds = 0.02 + 0.02 + 0.004 ms
    assert r["t_tensor_ms"] == pytest.approx(0.02)
    assert r["t_alu_ms"] == pytest.approx(0.02)
    assert r["t_hbm_ms"] == pytest.approx(0.004)
    assert r["t_min_ms"] == pytest.approx(0.044)
    assert r["frac"] == pytest.approx(0.44)
    assert bench.composite(1.0, 1.0, 1, 0.0, pk)["frac"] is None
