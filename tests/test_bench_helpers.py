"""Host-side pieces of bench.py: the algorithmic byte counts the roofline
divides by, and the ncu traffic table's link to the kernel sources."""
import hashlib
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_per_pixel():
    # binary: u read and written (8), four flows read and written (8 s), two
    # cost planes read (8), the alpha field read (4)
    assert bench.algorithmic_bytes_per_px("binary", 2, 0, True) == 52
    assert bench.algorithmic_bytes_per_px("binary", 2, 0, False) == 48
    assert bench.algorithmic_bytes_per_px("binary", 2, 1, True) == 36
    # Potts: per label u (8) and q_x, q_y, p_i (6 s) read and written and one
    # cost plane read; p_s read and written (8, float32 for every storage)
    assert bench.algorithmic_bytes_per_px("potts", 4, 0, False) == 152
    assert bench.algorithmic_bytes_per_px("potts", 16, 0, True) == 588
    assert bench.algorithmic_bytes_per_px("potts", 16, 1, True) == 396
    assert bench.algorithmic_bytes_per_px("potts", 16, 1, True, "f16") == 364
    assert bench.algorithmic_bytes_per_px("potts", 16, 0, True, "levels") == 16 * 32 + 4 + 8 + 4


def test_sixteen_bit_count_of_the_headline_workload():
    # every stored field in 16 bits: L (8 s + s_c) + 2 s + 4 with s = s_c = 2
    L, s, sc = bench.L, 2, 2
    assert bench.BYTES_PER_PX_16BIT == L * (8 * s + sc) + 2 * s + 4 == 296


def test_traffic_table_matches_the_sources():
    """Every entry of the committed ncu traffic table was taken on the
    kernel source as committed (the bench reads none that is stale)."""
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        table = json.load(f)
    assert table
    for name, e in table.items():
        with open(os.path.join(ROOT, e["source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        assert sha == e["src_sha256"], name
        assert bench._traffic(e["source"], name) == float(e["dram_bytes_per_launch_full_size"])
    assert bench._traffic("paper_2004_11227_gb300/csrc/cmf_potts_strip.cu", "no-such") is None


def test_phase_one_end_follows_the_switch_rule():
    """The bench recovers where a two-phase solve switched storage from its
    history: the first gap <= the switch gap, or a stall (tested every
    ceil(200 / check_every) checks, below 10x the switch gap, above 0.7x the
    previous tested gap)."""
    import numpy as np

    def hist(gaps):
        h = np.zeros((len(gaps), 5))
        h[:, 0] = 50 * (np.arange(len(gaps)) + 1)
        h[:, 3] = gaps
        return h

    # reaches the switch gap at row 3
    assert bench.phase_one_end(hist([1e-1, 1e-2, 5e-3, 1e-3, 5e-4]), 2e-3, 50) == 3
    # window of 4 checks at check_every 50: rows 0, 4, 8 tested; row 4 (6e-4 <
    # 1.5e-3, 6e-4 > 0.7 x 8e-4) stalls
    g = [8e-4, 7.5e-4, 7e-4, 6.5e-4, 6e-4, 5e-4]
    assert bench.phase_one_end(hist(g), 1.5e-4, 50) == 4
    # falling fast enough: no stall; the last row is returned
    g = [1e-2, 5e-3, 3e-3, 2e-3, 1e-3, 8e-4, 6e-4, 5e-4, 3e-4]
    assert bench.phase_one_end(hist(g), 1.5e-4, 50) == len(g) - 1
    # a stall far above 10x the switch gap does not count
    g = [1e-1] * 9 + [1e-3]
    assert bench.phase_one_end(hist(g), 1.5e-4, 50) == len(g) - 1
