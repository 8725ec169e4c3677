"""Separation rules of the repository, checked on the sources: the product
package never reaches the oracle (so no result can come from a CPU path), the
oracle never reaches the product, nothing committed refers to the scratch
folder, and profiles/ holds text summaries whose commands run committed files."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tracked():
    try:
        out = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True, check=True).stdout
        return [f for f in out.splitlines() if f]
    except (OSError, subprocess.CalledProcessError):  # not a git checkout: walk the tree
        files = []
        for d, dirs, fs in os.walk(ROOT):
            dirs[:] = [x for x in dirs if not x.startswith((".", "_work", "gpurun_out", "__pycache__", "_build"))]
            files += [os.path.relpath(os.path.join(d, f), ROOT) for f in fs]
        return files


def _read(rel):
    with open(os.path.join(ROOT, rel), encoding="utf-8", errors="replace") as f:
        return f.read()


def test_product_package_never_reaches_the_oracle():
    for rel in _tracked():
        if rel.startswith("paper_1905_03525_gb300/") and rel.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
            src = _read(rel)
            assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), rel
            assert "rmat_oracle" not in src, rel


def test_oracle_never_reaches_the_product():
    for rel in _tracked():
        if rel.startswith("oracle/"):
            src = _read(rel)
            assert "paper_1905_03525_gb300" not in src and not re.search(r"librmat(?!_oracle)", src), rel
            assert "rmat_device" not in src and "rmat_kernels" not in src, rel


# Reviews written into the repository from outside (not product files).
REVIEWS = ("VERDICT.md", "ADVICE.md")


def test_nothing_committed_uses_the_scratch_folder():
    scratch = "_" + "work/"  # spelled in two parts so that this file does not match itself
    for rel in _tracked():
        if rel in REVIEWS:
            continue
        if rel.endswith((".py", ".cu", ".cpp", ".h", ".cuh", ".c", ".md", ".txt", ".sh")):
            assert scratch not in _read(rel), rel


def test_profiles_are_text_summaries_with_commands():
    profs = [f for f in _tracked() if f.startswith("profiles/")]
    assert profs
    for rel in profs:
        assert rel.endswith((".md", ".txt")), rel
        if os.path.basename(rel) == "README.md":
            continue
        src = _read(rel)
        assert "ncu " in src and "--clock-control none" in src, rel
        assert os.path.getsize(os.path.join(ROOT, rel)) < 16 * 1024, rel
