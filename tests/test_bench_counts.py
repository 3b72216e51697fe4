"""Host-side byte and flop counts of bench.py's roofline lines, checked
against hand arithmetic for the 1024x16x8 wire (L = 2048, Py = 32, Pz = 16)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from paper_1903_07884_gb300 import inputs  # noqa: E402

N = 1024 * 16 * 8            # voxels
N3 = 3 * N
T = 3 * 1024 * 32 * 16       # yz-transformed intermediate [3][Pz][Py][nx]
OCT = 6 * 1025 * 17 * 9      # stored spectrum octants (L/2+1)(Py/2+1)(Pz/2+1) per generator


def test_matvec_pass_bytes():
    p = inputs.workload_long_straight()
    assert bench.algorithmic("mv_yz_fwd_c64", p, {}) == ("hbm", 8 * (N3 + T))
    assert bench.algorithmic("mv_x_c64", p, {}) == ("hbm", 8 * (2 * T + OCT))
    assert bench.algorithmic("mv_yz_inv_c64", p, {}) == ("hbm", 8 * (T + N3 + N + N3))


def test_matvec_summary_floor_and_three_pass():
    p = inputs.workload_long_straight()
    table = {"mv_yz_fwd_c64": (10, 0.1), "mv_x_c64": (10, 0.3), "mv_yz_inv_c64": (10, 0.2)}
    s = bench.matvec_summary(table, p, 6701.5)
    assert abs(s["ms_per_matvec"] - 0.06) < 1e-12
    assert s["floor_bytes"] == 8 * (7 * N + OCT) == 14_867_632
    assert s["three_pass_bytes"] == 68_345_008
    assert abs(s["three_pass_gbs"] - 68_345_008 / 0.06e-3 / 1e9) < 1e-6
    # a missing pass (another matvec path ran) gives no summary rather than a wrong one
    assert bench.matvec_summary({"mv_x_c64": (1, 1.0)}, p, 6701.5) is None


def test_arnoldi_bytes_grow_with_the_basis():
    p = inputs.workload_long_straight()
    meta = {"mean_j": 20.0}
    assert bench.algorithmic("arnoldi_dot_c64", p, meta) == ("hbm", 8 * 22.0 * N3)
    assert bench.algorithmic("arnoldi_update_c64", p, meta) == ("hbm", 8 * 24.0 * N3)
