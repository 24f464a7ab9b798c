"""Host logic of bench.py on CPU: the code digest that ties a recorded DRAM
traffic figure to the kernel sources it was measured on, and the rule that
reports the figure only for the measured configuration and code.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_digest_ignores_comments_and_white_space():
    a = "int f(int x)\n{\n    return x + 1;   // one more\n}\n"
    b = "/* header */ int   f(int x) {\n\treturn x + 1; }"
    assert bench.code_digest(a) == bench.code_digest(b)


def test_digest_sees_code_changes():
    assert bench.code_digest("int a = 1;") != bench.code_digest("int a = 2;")
    assert bench.code_digest("x = y + z;") != bench.code_digest("x = y - z;")


def test_traffic_only_for_the_measured_configuration():
    rec = bench.MEASURED_TRAFFIC
    n, k = bench.N_KEYS, bench.K
    bu = rec["bottom_up"]
    # any other workload, node size, block count or insert variant: no figure
    assert bench.measured_traffic("delete", n // 2, k, 0, bu) is None
    assert bench.measured_traffic("delete", n, k // 2, 0, bu) is None
    assert bench.measured_traffic("delete", n, k, 64, bu) is None
    assert bench.measured_traffic("delete", n, k, 0, not bu) is None


def test_traffic_null_once_the_code_differs(monkeypatch):
    rec = dict(bench.MEASURED_TRAFFIC)
    rec["sources"] = {name: "0" * 64 for name in rec["sources"]}
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", rec)
    assert bench.measured_traffic("delete", bench.N_KEYS, bench.K, 0, rec["bottom_up"]) is None


def test_traffic_reported_when_sources_match(monkeypatch):
    # a recorded figure is returned as is when every named source hashes to
    # its recorded digest (sources read from the package's csrc directory)
    csrc = os.path.join(ROOT, "paper_1906_06504_gb300", "csrc")
    rec = dict(bench.MEASURED_TRAFFIC)
    rec["sources"] = {}
    for name in bench.MEASURED_TRAFFIC["sources"]:
        with open(os.path.join(csrc, name)) as f:
            rec["sources"][name] = bench.code_digest(f.read())
    rec["delete"] = 123456789
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", rec)
    assert bench.measured_traffic("delete", bench.N_KEYS, bench.K, 0, rec["bottom_up"]) == 123456789


@pytest.mark.parametrize("kind", ["insert", "delete"])
def test_recorded_figures_are_byte_counts(kind):
    v = bench.MEASURED_TRAFFIC[kind]
    assert isinstance(v, int) and 1e8 < v < 1e11
