"""The autotuner's record table survives a save and a load (host only: no
GPU is needed to read or write the table), and malformed files load
nothing."""
import os

import pytest

import paper_1601_00221_gb300 as gp


def test_records_round_trip_through_a_file(tmp_path):
    gp.autotune_clear()
    p = tmp_path / "tuned.txt"
    p.write_text("# family several log2_cases log2_progs variant k block chunk stack_registers\n"
                 "1 0 16 12 1 8 256 0 4\n"
                 "6 1 18 13 6 4 128 32768 0\n"
                 "100 1 20 10 1 4 64 8192 0\n")
    gp.autotune_load(str(p))
    q = tmp_path / "again.txt"
    gp.autotune_save(str(q))
    lines = [ln.split() for ln in q.read_text().splitlines() if not ln.startswith("#")]
    assert sorted(lines) == sorted(ln.split() for ln in p.read_text().splitlines()[1:])
    gp.autotune_clear()
    gp.autotune_save(str(q))
    assert [ln for ln in q.read_text().splitlines() if not ln.startswith("#")] == []


@pytest.mark.parametrize("bad", ["1 0 16 12 1 8 256\n", "1 0 16 12 1 3 256 0 0\n", "1 0 16 12 99 8 256 0 0\n"])
def test_malformed_record_files_load_nothing(tmp_path, bad):
    gp.autotune_clear()
    p = tmp_path / "bad.txt"
    p.write_text("1 0 16 12 1 8 256 0 0\n" + bad)
    with pytest.raises(gp.GPError):
        gp.autotune_load(str(p))
    q = tmp_path / "out.txt"
    gp.autotune_save(str(q))
    assert [ln for ln in q.read_text().splitlines() if not ln.startswith("#")] == []
    with pytest.raises(gp.GPError):
        gp.autotune_load(str(tmp_path / "missing.txt"))


def test_split_records_round_trip_and_query(tmp_path):
    """A width-split record (the float tuner's, for many-input populations)
    survives a save and a load beside the single-launch records, and
    gp_autotune_split_record reports it for its shape and nothing for
    another."""
    gp.autotune_clear()
    p = tmp_path / "tuned.txt"
    p.write_text("4 1 18 10 4 2 256 65536 0\n"
                 "split 4 1 18 10 6 4 8 256 0 4 2 256 65536\n")
    gp.autotune_load(str(p))
    q = tmp_path / "again.txt"
    gp.autotune_save(str(q))
    lines = sorted(ln.split() for ln in q.read_text().splitlines() if not ln.startswith("#"))
    assert lines == sorted(ln.split() for ln in p.read_text().splitlines())
    th, narrow, wide = gp.autotune_split_record(gp.VARIANT_EXTENDED, 41, 494021, 1024)
    assert th == 6 and (narrow.variant, narrow.k, narrow.block) == (gp.VARIANT_EXTENDED, 8, 256)
    assert (wide.k, wide.block, wide.chunk_cases) == (2, 256, 65536)
    assert gp.autotune_split_record(gp.VARIANT_EXTENDED, 41, 494021, 70000)[0] == 0  # another shape
    assert gp.autotune_split_record(gp.VARIANT_REGISTER, 41, 494021, 1024)[0] == 0   # another family
    gp.autotune_clear()
    assert gp.autotune_split_record(gp.VARIANT_EXTENDED, 41, 494021, 1024)[0] == 0


@pytest.mark.parametrize("bad", ["split 4 1 18 10 6 4 8 256 0 4 2 256\n",      # a number short
                                 "split 4 1 18 10 0 4 8 256 0 4 2 256 65536\n",  # no threshold
                                 "split 4 1 18 10 6 4 3 256 0 4 2 256 65536\n"])  # k = 3
def test_malformed_split_records_load_nothing(tmp_path, bad):
    gp.autotune_clear()
    p = tmp_path / "bad.txt"
    p.write_text("1 0 16 12 1 8 256 0 0\n" + bad)
    with pytest.raises(gp.GPError):
        gp.autotune_load(str(p))
    q = tmp_path / "out.txt"
    gp.autotune_save(str(q))
    assert [ln for ln in q.read_text().splitlines() if not ln.startswith("#")] == []
