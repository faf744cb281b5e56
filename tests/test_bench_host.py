"""Host logic of bench.py that needs no GPU: the counts file's parser and the code-only hash that ties the
counts to the transport kernels' sources."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_only_drops_comments_and_layout_but_keeps_literals():
    src = 'int a; // line comment\n/* block\n comment */ float  b =\t1.f;\nconst char* s = "x // y /* z */";\nchar c = \'/\';'
    assert bench.code_only(src) == 'int a; float b = 1.f; const char* s = "x // y /* z */"; char c = \'/\';'
    # an escaped quote inside a literal does not end it
    assert bench.code_only('f("a\\"//b") // c') == 'f("a\\"//b")'


def test_hash_ignores_comments_but_not_code(tmp_path):
    csrc = os.path.join(ROOT, "paper_0902_3092_gb300", "csrc")
    base = tmp_path / "a"
    (base / "paper_0902_3092_gb300" / "csrc").mkdir(parents=True)
    for f in ("common.cuh", "transport.cuh", "transport_f32.cu"):
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            (base / "paper_0902_3092_gb300" / "csrc" / f).write_text(fh.read(), encoding="utf-8")
    h0 = bench.transport_source_hash(str(base))
    assert h0 == bench.transport_source_hash()
    p = base / "paper_0902_3092_gb300" / "csrc" / "transport_f32.cu"
    p.write_text(p.read_text(encoding="utf-8") + "\n// a comment\n/* another */\n", encoding="utf-8")
    assert bench.transport_source_hash(str(base)) == h0
    p.write_text(p.read_text(encoding="utf-8") + "static int x_added = 1;\n", encoding="utf-8")
    assert bench.transport_source_hash(str(base)) != h0


def test_counts_file_parses():
    """(Whether its hash matches the current sources decides, in the bench, whether the roofline is given.)"""
    c = bench.transport_counts()
    for k in ("source_sha16", "steps_per_launch", "warp_inst_per_step", "thread_inst_per_step", "dram_bytes_per_launch"):
        assert k in c
    assert len(c["source_sha16"]) == 16
    assert 10 < c["warp_inst_per_step"] < 100 and c["steps_per_launch"] > 1e10
