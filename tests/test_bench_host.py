"""Host logic of bench.py that needs no GPU: the key of the captured ncu traffic figures."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1004_2503_b300", "csrc")


def _read(f):
    with open(os.path.join(CSRC, f), encoding="utf-8") as fh:
        return fh.read()


def test_kernel_hash_ignores_comments_but_not_code():
    base = bench.kernel_hash(_read)
    assert base == bench.kernel_hash()
    commented = bench.kernel_hash(lambda f: "// a note\n/* a block\n note */\n" + _read(f) + "\n\n")
    assert commented == base
    edited = bench.kernel_hash(lambda f: _read(f).replace("kNTiny = 1e-30f", "kNTiny = 2e-30f"))
    assert edited != base


def test_traffic_figures_are_bytes_per_cell_near_the_algorithmic_52():
    for key, b in bench.NCU_TRAFFIC.items():
        assert len(key) == 12
        assert 40.0 < b < 60.0
