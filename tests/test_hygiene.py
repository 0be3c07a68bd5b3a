"""Structural checks on the sources (CPU): the CUDA path and the oracle stay independent, the
product path has no CPU fallback into the oracle, and every ncu command kept with a profile
leaves the GPU clocks alone."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2606_14173_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for dirpath, dirnames, filenames in os.walk(top):
        dirnames[:] = [d for d in dirnames if not d.startswith((".", "_", "__"))]
        for f in filenames:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def _read(path):
    with open(path, encoding="utf-8") as fh:
        return fh.read()


def test_package_never_reaches_the_oracle():
    """No source of the CUDA path imports, includes or loads anything under oracle/."""
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|#\s*include\s*[<\"][^>\"]*oracle)|[\"']oracle[\"'/]|liboracle",
                     re.M)
    for path in _files(PKG, (".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
        m = pat.search(_read(path))
        assert m is None, f"{os.path.relpath(path, ROOT)}: {m.group(0)!r}"


def test_oracle_never_reaches_the_package():
    """The oracle is written from the paper alone: it shares no header, kernel or helper with the
    CUDA path (the seeded scene generators are the one shared input module)."""
    pat = re.compile(r"hpt_internal|hpt_device|hpt_wave|hpt_real|csrc/|libhpt|from\s+paper_2606_14173_gb300\s+import\s+"
                     r"(?!scenes\b)\w+|import\s+paper_2606_14173_gb300\.(?!scenes\b)")
    for path in _files(ORACLE, (".py", ".c", ".h")):
        m = pat.search(_read(path))
        assert m is None, f"{os.path.relpath(path, ROOT)}: {m.group(0)!r}"


def test_profile_commands_leave_the_clocks_alone():
    """Every ncu command line kept in profiles/ (and in bench.py) passes --clock-control none."""
    paths = [os.path.join(ROOT, "profiles", f) for f in sorted(os.listdir(os.path.join(ROOT, "profiles")))]
    paths.append(os.path.join(ROOT, "bench.py"))
    seen = 0
    for path in paths:
        text = _read(path).replace("\\\n", " ")
        for line in text.splitlines():
            command = re.search(r"(^|[\s=\"'`])ncu\s+-(-set|-metrics|-section|k\b|s\b|c\b)", line) and \
                re.search(r"\$\w|python|--log-file|\s-o\s", line)
            if command and " -i " not in line:
                seen += 1
                assert "--clock-control none" in line, f"{os.path.relpath(path, ROOT)}: {line.strip()}"
    assert seen >= 5


def test_profiles_are_text_summaries():
    """profiles/ holds short text summaries, nothing that runs and no raw reports."""
    for f in os.listdir(os.path.join(ROOT, "profiles")):
        assert f.endswith((".md", ".txt")), f
        assert os.path.getsize(os.path.join(ROOT, "profiles", f)) < 16 * 1024, f
