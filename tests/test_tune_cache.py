"""Persistent autotune cache: the text format, its checks and the file
round trip (host only: no call here touches the GPU)."""
import pytest


@pytest.fixture(scope="module")
def tsg():
    from paper_2603_21444_gb300 import build
    build.build()
    import paper_2603_21444_gb300 as m
    return m


@pytest.fixture(autouse=True)
def clean(tsg):
    tsg.tune_cache_clear()
    yield
    tsg.tune_cache_clear()


def fields(t):
    nb = t.num_bins
    return nb, list(t.bin_upper)[:nb], list(t.bin_kernel)[:nb], t.warps_per_block, t.sym_warps_per_block


def coarse(tsg):
    t = tsg.default_tune()
    t.num_bins = 4
    for b, (u, k) in enumerate([(128, 2), (512, 4), (2048, 6), (8192, 8)]):
        t.bin_upper[b], t.bin_kernel[b] = u, k
    t.warps_per_block = 32
    return t


def test_store_then_reload(tsg, tmp_path):
    f = tmp_path / "tune.txt"
    assert tsg.tune_cache_open(str(f)) == 0  # a missing file counts as empty
    a = tsg.default_tune()
    a.warps_per_block = 8
    b = coarse(tsg)
    tsg.tune_cache_store(0x1234, a)
    tsg.tune_cache_store(0xFEDCBA9876543210, b)
    lines = f.read_text().splitlines()
    assert len(lines) == 2
    assert lines[0].startswith("tsg-tune-1 0000000000001234 12 8 8 16 10 32 0 64 1")
    assert lines[1] == "tsg-tune-1 fedcba9876543210 4 32 8 128 2 512 4 2048 6 8192 8"
    tsg.tune_cache_clear()
    assert tsg.tune_cache_entries() == []
    assert f.exists()  # clearing leaves the file alone
    assert tsg.tune_cache_open(str(f)) == 2
    got = dict(tsg.tune_cache_entries())
    assert fields(got[0x1234]) == fields(a)
    assert fields(got[0xFEDCBA9876543210]) == fields(b)


def test_bad_lines_skipped_and_last_line_wins(tsg, tmp_path):
    f = tmp_path / "tune.txt"
    f.write_text("tsg-tune-1 00000000000000aa 1 16 0 128 2\n"
                 "garbage\n"
                 "tsg-tune-2 00000000000000bb 1 16 0 128 2\n"   # another format version
                 "tsg-tune-1 00000000000000cc 1 16 0 128 99\n"  # no such variant
                 "tsg-tune-1 00000000000000dd 2 16 0 128 2\n"   # fewer bins than announced
                 "tsg-tune-1 00000000000000ee 1 16 0 1024 2\n"  # bound above the variant's capacity
                 "tsg-tune-1 00000000000000ef 2 16 0 256 3 128 4\n"  # bounds not increasing
                 "tsg-tune-1 00000000000000ff 1 16 0 128 2 7\n"  # trailing token
                 "tsg-tune-1 0000000000000100 1 0 0 128 2\n"    # warps per block out of range
                 + "x" * 2000 + "\n"                             # longer than any entry
                 "tsg-tune-1 00000000000000aa 1 4 0 64 1\n")
    assert tsg.tune_cache_open(str(f)) == 2
    ent = tsg.tune_cache_entries()
    assert len(ent) == 1 and ent[0][0] == 0xAA
    assert fields(ent[0][1]) == (1, [64], [1], 4, 0)


def test_environment_variable_names_the_file(tsg, tmp_path, monkeypatch):
    f = tmp_path / "env.txt"
    f.write_text("tsg-tune-1 0000000000000001 1 16 0 128 2\n")
    monkeypatch.setenv("TRIDENT_SPGEMM_TUNE_CACHE", str(f))
    assert tsg.tune_cache_open(None) == 1
    tsg.tune_cache_store(2, tsg.default_tune())
    assert len(f.read_text().splitlines()) == 2
    monkeypatch.delenv("TRIDENT_SPGEMM_TUNE_CACHE")
    assert tsg.tune_cache_open(None) == 0  # no variable: no file
    tsg.tune_cache_store(3, tsg.default_tune())
    assert len(f.read_text().splitlines()) == 2
    assert sorted(k for k, _ in tsg.tune_cache_entries()) == [1, 2, 3]


def test_refusals(tsg, tmp_path):
    from paper_2603_21444_gb300._abi import SpgemmError
    t = tsg.default_tune()
    t.warps_per_block = 0
    with pytest.raises(SpgemmError) as e:
        tsg.tune_cache_store(1, t)
    assert e.value.code == 1
    with pytest.raises(SpgemmError) as e:
        tsg.tune_cache_open(str(tmp_path))  # a directory is not a readable file
    assert e.value.code == 1
    # an append that cannot be written is reported; the entry stays cached
    tsg.tune_cache_open(str(tmp_path / "missing_dir" / "tune.txt"))
    with pytest.raises(SpgemmError):
        tsg.tune_cache_store(5, tsg.default_tune())
    assert [k for k, _ in tsg.tune_cache_entries()] == [5]
