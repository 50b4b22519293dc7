"""The in-tree build on CPU: every CUDA translation unit is compiled, for
sm_103a only, with line info, and a stale object is rebuilt."""
import os

from paper_2511_09413_gb300 import build as B


def test_every_translation_unit_is_built():
    cu = sorted(f for f in os.listdir(B.CSRC) if f.endswith(".cu"))
    assert sorted(B.SOURCES) == cu


def test_flags_target_sm_103a_only():
    f = B._flags()
    assert f[:2] == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert f.count("-gencode") == 1
    assert "-lineinfo" in f and "-O3" in f
    assert not any("march" in x or "arch=sm_" in x for x in f)


def test_stale_detection(tmp_path):
    src, obj = tmp_path / "a.cu", tmp_path / "a.o"
    src.write_text("x")
    assert B._stale(str(obj), [str(src)])            # missing object
    obj.write_text("o")
    os.utime(src, (1000, 1000))
    os.utime(obj, (2000, 2000))
    assert not B._stale(str(obj), [str(src)])
    os.utime(src, (3000, 3000))
    assert B._stale(str(obj), [str(src)])            # source newer than object
