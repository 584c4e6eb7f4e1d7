"""The render-source digest that guards the recorded ncu counters: it
follows the code and ignores comments and blank lines."""
import os
import shutil

import bench


def _copy(tmp_path):
    src = os.path.join(bench.ROOT, "paper_2606_21381_gb300", "csrc")
    dst = tmp_path / "csrc"
    shutil.copytree(src, dst)
    return dst


def test_comments_and_blank_lines_do_not_change_the_digest(tmp_path):
    d = _copy(tmp_path)
    base = bench.source_digest(str(d))
    assert base == bench.source_digest()
    p = d / "osog_strip.cuh"
    text = p.read_text()
    p.write_text("// a new comment line\n\n/* and a block\n   comment */\n" + text + "\n// trailing\n")
    assert bench.source_digest(str(d)) == base


def test_a_code_change_changes_the_digest(tmp_path):
    d = _copy(tmp_path)
    base = bench.source_digest(str(d))
    p = d / "osog_render.cu"
    p.write_text(p.read_text().replace("pdl_enter();", "pdl_enter(); __syncthreads();", 1))
    assert bench.source_digest(str(d)) != base
