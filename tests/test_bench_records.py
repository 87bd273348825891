"""The stored ncu traffic record that bench.py's roofline `traffic` reads
(profiles/hop_lb_f32_traffic.json) is consistent with its own definitions.

* Algorithmic bytes: each captured launch's figure is recomputed from the stated
  workload. The workload is 24^4 with 7^4 cores and frame 1, so 81 framed 9^4
  blocks, with per-parity site counts from the oracle's geometry, and 12 rhs.
  A launch moves, per output (site, rhs), the input spinor and the output once,
  each self term once, and the 8 links of the site shared by the 12 systems.
* Ratio: DRAM bytes are read + write, and the stored ratio is the mean DRAM
  bytes over the mean algorithmic bytes.
* Variant: the record names the launch form the library calls variant 13.

CPU only.
"""

import json
import os

import numpy as np
import pytest

from oracle.geometry import Decomposition, uniform_cores
from paper_2211_06902_gb300 import dd4d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _parity_counts(L, mask):
    x = np.indices(L).sum(axis=0) % 2
    return int(np.sum(mask & (x == 0))), int(np.sum(mask & (x == 1)))


def test_traffic_record_matches_its_workload():
    rec = json.load(open(os.path.join(ROOT, "profiles", "hop_lb_f32_traffic.json")))
    L = (24, 24, 24, 24)
    geo = Decomposition(L, uniform_cores(L, 7, 1))
    assert len(geo.omega_mask) == 81
    counts = {_parity_counts(L, m) for m in geo.omega_mask}
    assert len(counts) == 1                      # every block has the same parity split
    split = counts.pop()
    n_even, n_odd = max(split), min(split)       # the block-local parity of the corner site has more
    assert (n_even, n_odd) == (3281, 3280)
    nrhs, c = 12, 8                              # FP32 complex: 8 bytes
    per_unit = {1: 12 * c * 3 + 8 * 9 * c / nrhs, 0: 12 * c * 2 + 8 * 9 * c / nrhs}
    assert per_unit == {1: 336.0, 0: 240.0}
    for k, ln in enumerate(rec["launches"]):
        self_term = 1 if "self term" in ln["role"] else 0
        n = n_even if ln["role"].startswith("even") else n_odd
        assert ln["algorithmic_bytes"] == pytest.approx(81 * nrhs * n * per_unit[self_term], rel=1e-12), k
        assert ln["bytes"] == pytest.approx(ln["read"] + ln["write"], rel=1e-12), k
        assert 1.0 <= ln["bytes"] / ln["algorithmic_bytes"] < 1.2, k
    mb = np.mean([ln["bytes"] for ln in rec["launches"]])
    ma = np.mean([ln["algorithmic_bytes"] for ln in rec["launches"]])
    assert rec["dram_over_algorithmic"] == pytest.approx(mb / ma, rel=1e-12)
    assert rec["bytes_per_full_launch"] == pytest.approx(mb, rel=1e-12)


def test_traffic_record_names_the_captured_variant():
    if not os.path.exists(dd4d.LIB_PATH):
        from paper_2211_06902_gb300 import build
        build.build()
    rec = json.load(open(os.path.join(ROOT, "profiles", "hop_lb_f32_traffic.json")))
    assert rec["variant_name"] == dd4d.hop_variant_name("f32", 13)
    assert "--variant 13" in rec["command"] and "--clock-control none" in rec["command"]
