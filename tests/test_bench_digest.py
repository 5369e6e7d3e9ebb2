"""The round kernel's traffic digest in bench.py: comments and blank lines do
not change it, code does (the captured traffic ratio is dropped only when the
kernel itself changed)."""
import os
import shutil


def _copy_sources(bench, root):
    for f in bench.ROUNDS_SOURCES:
        dst = os.path.join(root, f)
        os.makedirs(os.path.dirname(dst), exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, f), dst)


def test_digest_ignores_comments_and_tracks_code(tmp_path, monkeypatch):
    import bench
    base = bench.rounds_sources_digest()
    _copy_sources(bench, str(tmp_path))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.rounds_sources_digest() == base
    f = os.path.join(str(tmp_path), bench.ROUNDS_SOURCES[0])
    with open(f, "a") as fh:
        fh.write("\n// a remark\n\n/* another\n   remark */\n")
    assert bench.rounds_sources_digest() == base
    with open(f, "a") as fh:
        fh.write("static int unused_marker_for_the_test = 1;\n")
    assert bench.rounds_sources_digest() != base
