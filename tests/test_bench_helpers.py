"""Host logic the bench's reported numbers rest on: the DRAM-traffic model and the rule that it
is reported only for the kernel sources its ncu check was taken on, and the parsers of the e2e
host-buffer diagnostics read this process's own mappings."""
import hashlib
import mmap
import os

import numpy as np

import bench


def _current_sha():
    return bench.sources_sha(bench.FUSED_TRAFFIC_CHECK["sources"])


def test_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1210_7683_gb300" / "csrc"
    csrc.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (csrc / "k.cu").write_text("int a = 1;  // one\n/* block\n comment */\nint b = a;\n")
    h0 = bench.sources_sha(["k.cu"])
    (csrc / "k.cu").write_text("int a = 1;  // another comment\n\nint b = a;   \n")
    assert bench.sources_sha(["k.cu"]) == h0
    (csrc / "k.cu").write_text("int a = 2;\nint b = a;\n")
    assert bench.sources_sha(["k.cu"]) != h0


def test_traffic_model_terms():
    # one traversal group: every operand read once, every result written once (64 traits: three
    # tiles of 24 in the interpolated kernel)
    mod = bench.fused_traffic_model(1000, 128 * 16, 64, group=16)
    kpad = 1024
    assert mod["write"] == 8.0 * 128 * 16 * 64
    assert mod["read"] == 2048 * kpad * 2 + 25 * 4 * 2048 + 3 * 240 * kpad * 2
    # the trait operands are read once per group of 16 SNP tiles (32 for the CTA pair's 2 x 16)
    one = bench.fused_traffic_model(1000, 128 * 64, 10_000, group=16)
    pair = bench.fused_traffic_model(1000, 128 * 64, 10_000, group=16, cs=2)
    trait = 417 * 240 * kpad * 2
    assert one["read"] - pair["read"] == 2 * trait
    # contracting S_BR adds the three x'^2 planes and the C2 trait rows
    ex = bench.fused_traffic_model(1000, 128 * 16, 64, group=16, interp=False)
    assert ex["read"] == 2048 * kpad * 2 * 4 + 2 * 448 * kpad * 2


def test_traffic_reported_only_for_the_checked_sources(monkeypatch):
    w = (1000, 3, 1_000_000, 10_000)
    monkeypatch.setattr(bench, "FUSED_TRAFFIC_CHECK", dict(bench.FUSED_TRAFFIC_CHECK, sha256=_current_sha()))
    mod = bench.fused_traffic_model(1000, 1_000_000, 10_000)
    assert bench.fused_traffic(w) == mod["read"] + mod["write"]
    monkeypatch.setattr(bench, "FUSED_TRAFFIC_CHECK", dict(bench.FUSED_TRAFFIC_CHECK, sha256="0" * 64))
    assert bench.fused_traffic(w) is None


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


def test_traffic_model_fp4_terms():
    # e2m1 operands: half a byte per genotype and per digit, K padded to 256, three digit rows per
    # C1 row; the coefficients and the results as on bf16 operands
    mod = bench.fused_traffic_model(1000, 128 * 16, 64, group=16, cs=2, fp4=True)
    assert mod["write"] == 8.0 * 128 * 16 * 64
    assert mod["read"] == 2048 * 1024 // 2 + 25 * 4 * 2048 + 3 * 3 * 240 * 1024 // 2
    bf = bench.fused_traffic_model(1000, 128 * 16, 64, group=16, cs=2)
    assert mod["read"] < bf["read"]
    # n = 1100: Kpad = 1152, Kp4 = 1280
    m4 = bench.fused_traffic_model(1100, 128, 24, group=1, fp4=True)
    assert m4["read"] == 128 * 640 + 25 * 4 * 128 + 3 * 240 * 640


def test_hugepage_share_of_a_range_inside_a_mapping():
    # two mappings of 4 MiB: the first on huge pages, the second on base pages
    smaps = ["10000000-10400000 rw-p 00000000 00:00 0", "Size:               4096 kB", "AnonHugePages:      4096 kB",
             "10400000-10800000 rw-p 00000000 00:00 0", "Size:               4096 kB", "AnonHugePages:         0 kB"]
    mib = 1 << 20
    assert bench.hugepage_share(smaps, 0x10000000, 4 * mib) == 1.0
    assert bench.hugepage_share(smaps, 0x10000000, 2 * mib) == 1.0          # half of the first mapping
    assert bench.hugepage_share(smaps, 0x10200000, 4 * mib) == 0.5          # its second half and half the next
    assert bench.hugepage_share(smaps, 0x10400000, 4 * mib) == 0.0
