"""Guards on the repository's structure: the library never reaches the
oracle (so no result of the CUDA path can come from it), the oracle never
reaches the library, no committed file uses the scratch folder, and no
source uses the batched-copy runtime calls.  CPU only."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2608_14911_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("_build", "__pycache__")]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def _text(path):
    with open(path, encoding="utf-8", errors="replace") as fh:
        return fh.read()


def test_library_does_not_reach_the_oracle():
    imp = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|from\s+\.\.\s*import\s+oracle)", re.M)
    for p in _files(PKG, (".py",)):
        assert not imp.search(_text(p)), p
    inc = re.compile(r'#\s*include\s*[<"][^>"]*(oracle|orc\.h)')
    for p in _files(PKG, (".cu", ".cuh", ".cpp", ".h")):
        assert not inc.search(_text(p)), p
    for p in _files(os.path.join(ROOT, "include"), (".h",)):
        assert not inc.search(_text(p)), p


def test_oracle_does_not_reach_the_library():
    for p in _files(ORACLE, (".py", ".c", ".h")):
        t = _text(p)
        assert "paper_2608_14911_gb300" not in t and "espp.h" not in t and "libespp" not in t, p


def test_no_committed_file_uses_the_scratch_folder():
    pat = re.compile(r"(^|[^A-Za-z0-9])_work/")
    tops = [PKG, ORACLE, os.path.join(ROOT, "tests"), os.path.join(ROOT, "include")]
    files = [os.path.join(ROOT, f) for f in ("bench.py", "__graft_entry__.py")]
    for top in tops:
        files += list(_files(top, (".py", ".c", ".h", ".cu", ".cuh", ".cpp", ".sh")))
    for p in files:
        if os.path.abspath(p) == os.path.abspath(__file__):
            continue
        assert not pat.search(_text(p)), p


def test_sources_avoid_batched_copies():
    pat = re.compile(r"[Mm]emcpy(3D)?Batch")
    for top in (PKG, ORACLE, os.path.join(ROOT, "include"), os.path.join(ROOT, "tests")):
        for p in _files(top, (".py", ".c", ".h", ".cu", ".cuh", ".cpp")):
            assert not pat.search(_text(p)), p
    assert not pat.search(_text(os.path.join(ROOT, "bench.py")))
