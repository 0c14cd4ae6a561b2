"""The CUDA path and the oracle are independent: the product package never
imports, loads or names the oracle; the oracle's C source includes nothing of
the library's; the library's sources include nothing outside their own
folder, CUDA and the C/C++ runtime; and the loaded library does not link the
oracle."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2301_03636_gb300")
CSRC = os.path.join(PKG, "csrc")
ORACLE = os.path.join(ROOT, "oracle")


def _sources(folder, exts):
    for dirpath, dirnames, files in os.walk(folder):
        dirnames[:] = [d for d in dirnames if not d.startswith(("_", "."))]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def test_package_never_reaches_the_oracle():
    # imports, loads and the oracle's C symbols (a docstring may still name it)
    pat = re.compile(r"import\s+oracle|from\s+oracle|oracle\.|liboracle|advisor_oracle|\borc_")
    hits = []
    for path in _sources(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")):
        for i, line in enumerate(open(path), 1):
            if pat.search(line):
                hits.append(f"{os.path.relpath(path, ROOT)}:{i}: {line.strip()}")
    assert not hits, hits


def test_includes_stay_on_their_own_side():
    inc = re.compile(r'#include\s+[<"]([^>"]+)[>"]')
    oracle_incs = set(inc.findall(open(os.path.join(ORACLE, "advisor_oracle.c")).read()))
    assert oracle_incs <= {"math.h", "stdint.h", "stdlib.h", "string.h", "stddef.h", "omp.h"}, oracle_incs
    local = set(os.listdir(CSRC)) | {"advisor.h"}
    for path in _sources(CSRC, (".cu", ".cuh")):
        for name in inc.findall(open(path).read()):
            if "/" in name or name.endswith((".cuh", ".h")) and not name.startswith(("cuda", "cublas")):
                assert name in local or name in {"stdint.h", "stddef.h"}, (path, name)


def test_library_does_not_link_the_oracle():
    from paper_2301_03636_gb300 import build
    lib = build.build()
    r = subprocess.run(["readelf", "-d", lib], capture_output=True, text=True)
    if r.returncode != 0:   # no binutils: nothing more to check here
        return
    needed = re.findall(r"\(NEEDED\).*\[(.+)\]", r.stdout)
    assert needed and not any("oracle" in n for n in needed), needed


def test_product_path_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """With no built library there is no fallback: loading it, and any call
    that reaches it, raises."""
    import pytest
    from paper_2301_03636_gb300 import advisor
    monkeypatch.setattr(advisor, "_lib", None)
    monkeypatch.setattr(advisor, "library_path", lambda: str(tmp_path / "libadvisor.so"))
    with pytest.raises(RuntimeError, match="not built"):
        advisor.lib()
    with pytest.raises(RuntimeError, match="not built"):
        advisor.launch_count()
