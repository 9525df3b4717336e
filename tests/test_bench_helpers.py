"""Host logic the bench's reported numbers rest on: the DRAM-traffic record is reported only
for the kernel sources and launch shape it was captured on, and the parsers of the e2e
host-buffer diagnostics read this process's own mappings."""
import hashlib
import mmap
import os

import numpy as np

import bench


def _current_sha():
    h = hashlib.sha256()
    for f in bench.FUSED_TRAFFIC["sources"]:
        with open(os.path.join(bench.ROOT, "paper_1210_7683_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def test_traffic_record_tied_to_sources_workload_and_shape(monkeypatch):
    rec = dict(bench.FUSED_TRAFFIC, sha256=_current_sha())
    monkeypatch.setattr(bench, "FUSED_TRAFFIC", rec)
    w = rec["workload"]
    for cap in rec["captures"]:
        assert bench.fused_traffic(w, dict(cap["shape"])) == cap["read"] + cap["write"]
    first = rec["captures"][0]
    shape = dict(first["shape"])
    assert bench.fused_traffic(w) == first["read"] + first["write"]       # shape unknown: the default
    assert bench.fused_traffic((w[0], w[1], w[2] // 2, w[3]), shape) is None
    assert bench.fused_traffic(w, dict(shape, group=32)) is None           # no capture of this shape
    assert bench.fused_traffic(w, dict(shape, cs=2, pair=1)) is None
    monkeypatch.setattr(bench, "FUSED_TRAFFIC", dict(rec, sha256="0" * 64))  # sources changed since
    assert bench.fused_traffic(w, shape) is None


def test_host_buffer_parsers_read_own_mapping():
    nbytes = 32 << 20
    mm = mmap.mmap(-1, nbytes, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
    try:
        a = np.frombuffer(mm, dtype=np.uint8)
        a[::4096] = 1                                   # fault every page in
        frac = bench.hugepage_fraction(a.ctypes.data, nbytes)
        assert frac is None or 0.0 <= frac <= 1.0
        pages = bench.numa_pages(a.ctypes.data, nbytes)
        if pages is not None:
            page = mmap.PAGESIZE
            assert all(k.startswith("N") for k in pages)
            assert sum(pages.values()) * page >= nbytes // 2   # resident pages are counted
        # a range no mapping of this process covers
        assert bench.hugepage_fraction(8, 4096) in (None, 0.0)
        assert bench.numa_pages(8, 4096) in (None, {})
        del a
    finally:
        mm.close()


def test_serving_loads_default_headline_first():
    import sys
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        args = bench.parse()
    finally:
        sys.argv = argv
    loads = [float(x) for x in args.serving_load.split(",")]
    assert loads[0] == 0.8 and sorted(loads) == [0.5, 0.8, 0.95]
