"""bench.py's host-side pieces, on CPU: the DRAM-traffic table lookup (a row counts only
for its kernel, its ion count and the current hash of the pair kernels' sources; a changed
source makes every row read as null), and the ALU roofline constants of the pair kernels."""
import os
import shutil

import pytest

import bench


def _fake_root(tmp_path, rows, sources_extra=b""):
    root = tmp_path / "root"
    csrc = root / "paper_2205_06557_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        src = os.path.join(bench.ROOT, "paper_2205_06557_gb300", "csrc", f)
        shutil.copy(src, csrc / f)
    if sources_extra:
        with open(csrc / bench.KERNEL_SOURCES[0], "ab") as fh:
            fh.write(sources_extra)
    (root / "profiles").mkdir()
    table = ["| kernel | n_ions | dram bytes per launch | sources sha256 | read / write |", "|---|---|---|---|---|"]
    table += ["| %s | %s | %s | %s | x |" % r for r in rows]
    (root / "profiles" / "dram_traffic.md").write_text("\n".join(table) + "\n")
    return str(root)


def test_traffic_rows_need_the_kernel_the_size_and_the_sources_hash(tmp_path, monkeypatch):
    h = bench.kernel_sources_hash()
    assert len(h) == 16 and all(c in "0123456789abcdef" for c in h)
    root = _fake_root(tmp_path, [("k_forces_sym2<64,8>", "1,005,310", "40,802,560", h),
                                 ("k_forces_sym2<64,8>", "199,969", "8,527,872", "0000000000000000")])
    monkeypatch.setattr(bench, "ROOT", root)
    assert bench.kernel_sources_hash() == h
    assert bench.ncu_traffic("k_forces_sym2<64,8>", 1005310) == 40802560
    assert bench.ncu_traffic("k_forces_sym2<64,8>", 199969) is None  # another hash
    assert bench.ncu_traffic("k_forces_sym2<64,8>", 1005311) is None  # another size
    assert bench.ncu_traffic("k_forces_sym2<128,8>", 1005310) is None  # another kernel


def test_a_changed_source_voids_the_table(tmp_path, monkeypatch):
    h = bench.kernel_sources_hash()
    root = _fake_root(tmp_path, [("k_forces_sym2<64,8>", "1,005,310", "40,802,560", h)], sources_extra=b"\n// x\n")
    monkeypatch.setattr(bench, "ROOT", root)
    assert bench.kernel_sources_hash() != h
    assert bench.ncu_traffic("k_forces_sym2<64,8>", 1005310) is None


def test_missing_table_reads_as_null(tmp_path, monkeypatch):
    root = _fake_root(tmp_path, [])
    os.remove(os.path.join(root, "profiles", "dram_traffic.md"))
    monkeypatch.setattr(bench, "ROOT", root)
    assert bench.ncu_traffic("k_forces_sym2<64,8>", 1005310) is None


def test_pair_kernel_roofline_constants():
    # ordered kernel: 14 FP32 ops per pair against 128 lanes; symmetric: 8.5 per ordered pair;
    # the SFU (rsqrt at 16, ex2 at 32 per clock per SM) is not the limit of either
    assert bench.PAIRS_PER_CLK_SM[0] == pytest.approx(128 / 14)
    assert bench.PAIRS_PER_CLK_SM[1] == pytest.approx(128 / 8.5)
    assert 1 / bench.SFU_CLK_PER_PAIR > 128 / 14
    # 152 SMs at 2070 MHz: the symmetric kernels' peak of 4.738e12 ordered pairs/s
    assert 152 * 2.07e9 * bench.PAIRS_PER_CLK_SM[1] == pytest.approx(4.738e12, rel=1e-3)
