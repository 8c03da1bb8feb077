"""Host logic of the bench's DRAM-traffic bookkeeping: an ncu launch list (csv) is grouped into the
rendering stages of the first plain frame (each stage's first launches, up to the first SH backward),
units are scaled to bytes and microseconds, every kernel is summed over the whole pass, and each stage
carries the hash of the sources that decide its traffic.  Also the stage models' algorithmic counts on
a small hand-checked case."""
import csv
import io
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _csv(rows):
    buf = io.StringIO()
    w = csv.writer(buf, quoting=csv.QUOTE_ALL)
    w.writerow(["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"])
    for i, (name, rd, wr, us) in enumerate(rows):
        w.writerow([i, name, "dram__bytes_read.sum", "Mbyte", rd])
        w.writerow([i, name, "dram__bytes_write.sum", "Kbyte", wr])
        w.writerow([i, name, "gpu__time_duration.sum", "usecond", us])
    return "==PROF== preamble\n" + buf.getvalue()


def test_traffic_grouping_and_units(tmp_path):
    launches = [
        ("k_project(BatchParams)", "2.0", "500", "10"),
        ("void k_os_pass<unsigned long, 4>(x)", "1.0", "0", "5"),
        ("void k_os_pass<unsigned long, 4>(x)", "1.5", "0", "6"),
        ("k_records_emit(x)", "3.0", "1000", "20"),
        ("void k_os_pass<unsigned int, 8>(x)", "0.5", "0", "7"),
        ("k_pair_mask(x)", "0.25", "0", "2"),
        ("k_tile_count(x)", "0.25", "0", "1"),
        ("void k_composite<0, 1, 0, 0, 0>(x)", "4.0", "0", "100"),
        ("void k_composite<1, 1, 0, 0, 0>(x)", "8.0", "0", "200"),
        ("void k_sh_bwd<0>(x)", "2.0", "2000", "15"),
        # a second frame (with normals): counted per kernel, not per stage
        ("k_project(BatchParams)", "9.0", "0", "99"),
    ]
    src = tmp_path / "launches.csv"
    src.write_text(_csv(launches))
    out = tmp_path / "traffic.json"
    assert bench.build_traffic(str(src), str(out)) == 0
    t = json.loads(out.read_text())
    st = t["stages"]
    assert st["project"]["bytes_per_launch"] == 2_500_000 and st["project"]["us_ncu"] == 10.0
    assert st["sort_vox"]["bytes_per_launch"] == 2_500_000 and st["sort_vox"]["us_ncu"] == 11.0
    assert st["records"]["bytes_per_launch"] == 4_000_000
    assert st["ranges"]["bytes_per_launch"] == 500_000 and st["ranges"]["us_ncu"] == 3.0
    assert st["composite_bwd"]["bytes_per_launch"] == 8_000_000
    assert st["sh_bwd"]["bytes_per_launch"] == 4_000_000
    for name, rec in st.items():
        assert rec["source_hash"] == bench.sources_hash(bench.STAGE_KERNELS[name][1])
    k = t["kernels"]["k_project"]
    assert k["launches"] == 2 and k["bytes"] == 11_500_000.0 and k["us"] == 109.0


def test_stage_models_hand_checked():
    stats = {"n_visible": 10, "n_pairs": 40, "n_tiles": 300}
    work = {"tests": 1000, "box_tests": 50, "segments": 400}
    m = bench.stage_models(stats, work, n_vox_total=100, n_pix=64, K=1, sh_bytes_per_vox=192, key_bits=20)
    assert m["project"] == ("hbm", 100 * 8 + 10 * 24)
    assert m["sort_vox"] == ("hbm", 3 * 10 * 24)                 # 20-bit keys: three 8-bit passes
    assert m["sort_pairs"] == ("hbm", 2 * 40 * 16)               # 300 tiles: 9 bits, two passes
    assert m["composite_fwd"] == ("alu", 1000 * 20 + 50 * 20 + 400 * (31 + 16))
    assert m["composite_bwd"] == ("alu", 1000 * 20 + 50 * 20 + 400 * (31 + 35 + 16 + 43))
