"""The roofline arithmetic of bench.py, on the host: the algorithmic work it
divides by the measured durations matches the counts the scale supports of
Sec. 2.2 give (7.17e8 (l, m', m) triples and 1.58e10 flop per contraction at
L = 1024, N = 5, lambda = 2; 1.80e8 Delta entries of the eighth domain), and
a DRAM-traffic record is only used while the kernel sources are unchanged."""
import importlib.util
import json
import os
import sys

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


class _Supports:
    """Stands in for a plan: the wavelet scales' supports of Sec. 2.2, cut at L - 1."""

    def __init__(self, L, N, lam):
        self.L, self.N = L, N
        self.nscale = O.n_scales(L, lam, 0) + 1
        self._s = [O.support(j, L, lam) for j in range(self.nscale)]

    def support(self, j):
        lo, hi = self._s[j]
        return lo, min(hi, self.L - 1)


def test_contraction_work_at_the_headline_size(bench):
    p = _Supports(1024, 5, 2.0)
    flops = bench.contraction_flops(p)
    triples = flops / (2 + 4 * 5)
    assert triples == pytest.approx(7.17e8, rel=2e-3)
    assert flops == pytest.approx(1.58e10, rel=2e-3)
    # brute force over the (l, m', m >= 0) triples of every scale at a small size
    q = _Supports(24, 3, 2.0)
    brute = sum(1 for j in range(q.nscale) for l in range(q.support(j)[0], q.support(j)[1] + 1)
                for mp in range(l + 1) for m in range(l + 1))
    assert bench.contraction_flops(q) == brute * (2 + 4 * 3)


def test_delta_eighth_domain_bytes(bench):
    b = bench.delta_eighth_bytes(1024)
    assert b / 4 == pytest.approx(1.80e8, rel=3e-3)
    L = 17
    assert bench.delta_eighth_bytes(L) == 4 * sum(1 for l in range(L) for mp in range(l + 1) for m in range(mp, l + 1))


def test_traffic_record_needs_unchanged_sources(bench, tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    rel = os.path.relpath(str(src), ROOT)
    rec = {"kernel": "k", "bytes_per_launch": 123, "files": [rel], "date": "d",
           "fingerprint": bench.source_fingerprint([rel])}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps({"stage": rec}))
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(path))
    assert bench.recorded_traffic("stage")[0] == 123
    assert bench.recorded_traffic("other") == (None, None)
    src.write_text("__global__ void k() { }\n")
    b, why = bench.recorded_traffic("stage")
    assert b is None and "changed" in why
