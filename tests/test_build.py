"""The in-tree build's staleness check (CPU only, no compilation): touching any source or header
the library is built from must make build.up_to_date() false."""
import os

from paper_2010_00626_b300 import build


def test_deps_cover_every_source_and_header():
    csrc = os.path.join(build.HERE, "csrc")
    want = {os.path.join(csrc, f) for f in os.listdir(csrc) if f.endswith((".cu", ".cuh", ".h"))}
    want.add(os.path.join(build.ROOT, "include", "kcycle.h"))
    assert want <= set(build.deps())
    for name in ("lines.cuh", "stream_f32.cuh", "kernels.cuh", "kcycle.cu"):
        assert os.path.join(csrc, name) in build.deps()


def test_touching_any_dependency_makes_the_library_stale(tmp_path, monkeypatch):
    lib = tmp_path / "libkcycle.so"
    lib.write_bytes(b"")
    monkeypatch.setattr(build, "LIB", str(lib))
    newest = max(os.path.getmtime(p) for p in build.deps())
    os.utime(lib, (newest + 10, newest + 10))
    assert build.up_to_date()
    for name in ("lines.cuh", "stream_f32.cuh"):
        dep = os.path.join(build.HERE, "csrc", name)
        st = os.stat(dep)
        try:
            os.utime(dep, (st.st_atime, newest + 20))
            assert not build.up_to_date(), name
        finally:
            os.utime(dep, (st.st_atime, st.st_mtime))
        assert build.up_to_date()
