"""Host-side consistency of bench.py's measured tables with the library's autotuner.

The bench reports the push's DRAM traffic for the layout the autotuner returns. It looks the figure up in
a table of ncu measurements, so that table must cover every layout the autotuner can choose. The figures
must also sit where the push's stored state puts them: the mixed path reads 32 B and writes 24 B per
particle, and the last writes of a launch may still be in L2 when it ends.
"""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _tuner_candidates():
    src = open(os.path.join(ROOT, "paper_1009_2727_gb300", "csrc", "pic_tune.cu")).read()
    tiles = [int(v) for v in re.search(r"kTiles\[\d+\]\s*=\s*\{([^}]*)\}", src).group(1).split(",")]
    cads = [int(v) for v in re.search(r"kCadences\[\d+\]\s*=\s*\{([^}]*)\}", src).group(1).split(",")]
    return tiles, cads


def test_traffic_table_covers_every_autotuner_layout():
    tiles, cads = _tuner_candidates()
    want = {(tx, tz, se) for tx in tiles for tz in tiles for se in cads}
    have = set(bench.TRAFFIC_BYTES_PER_PARTICLE)
    assert want <= have, sorted(want - have)
    assert have <= want, sorted(have - want)


def test_traffic_figures_are_the_stored_state():
    # 56 B of stored state at most; reads (32 B) and most of the writes always reach DRAM
    for lay, b in bench.TRAFFIC_BYTES_PER_PARTICLE.items():
        assert 40.0 < b <= 56.0, (lay, b)
    for key, b in bench.TRAFFIC_BYTES_PER_PARTICLE_3D.items():
        assert b <= bench.BYTES_PER_PARTICLE_3D[key[0]] + 8.0, (key, b)


def test_algorithmic_bytes_cover_the_stored_state():
    # the algorithmic figure counts positions at FP64-equivalent width, so it bounds the stored state
    assert bench.BYTES_PER_PARTICLE["mixed"] >= 56
    assert bench.BYTES_PER_PARTICLE["fp64"] > bench.BYTES_PER_PARTICLE["mixed"]
    assert bench.BYTES_PER_CELL["fp64"] == 2 * bench.BYTES_PER_CELL["mixed"]
