"""Repository rules that later changes must keep: every C-ABI entry point documents the passage
it follows (or that it has none), code and comments stand on their own without naming planning
documents or the machines they were built on, and no built artefact is committed."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CITE = re.compile(r"Alg\.|Sec\.|Fig\.|Table|counterpart")


def test_every_entry_point_cites_its_passage():
    txt = open(os.path.join(ROOT, "include", "tocab.h")).read()
    decl = re.compile(r"^(?:int|void|int32_t|int64_t|const char \*)\s*\*?\s*(tc_[a-z0-9_]+)\s*\(", re.M)
    missing = []
    for m in decl.finditer(txt):
        before = txt[:m.start()]
        end = before.rfind("*/")
        comment = before[before.rfind("/*", 0, end):end]
        between = before[end + 2:]
        # the comment may serve a run of declarations that directly follow it
        only_decls = all(ln.strip() == "" or decl.match(ln) or ln.startswith(" ")
                         for ln in between.splitlines())
        if not CITE.search(comment) or (between.count("\n") > 2 and not only_decls):
            missing.append(m.group(1))
    assert not missing, missing


def _ignored_dirs():
    """Top-level folders that .gitignore lists (scratch and run output, never committed)."""
    names = {".git", "__pycache__", "_build", "baseline"}
    try:
        for ln in open(os.path.join(ROOT, ".gitignore")):
            ln = ln.strip()
            if ln and not ln.startswith("#") and ln.endswith("/") and "*" not in ln:
                names.add(ln.strip("/").split("/")[0])
    except OSError:
        pass
    return names


def _code_files():
    out = []
    skip = _ignored_dirs()
    for base, dirs, files in os.walk(ROOT):
        dirs[:] = [d for d in dirs if d not in skip]
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp", ".sh")) and f != "test_repo_rules.py":
                out.append(os.path.join(base, f))
    return out


def test_code_names_no_planning_documents_or_machines():
    banned = ["SUR" + "VEY", "VER" + "DICT", "AD" + "VICE.md", "north" + "_star", "gpu" + "run",
              "/ro" + "ot/", "BASELINE" + ".json", "configs" + "["]
    hits = []
    for path in _code_files():
        text = open(path, errors="replace").read()
        for b in banned:
            if b in text:
                hits.append((os.path.relpath(path, ROOT), b))
    assert not hits, hits


def test_no_built_artefacts_are_tracked():
    if not os.path.isdir(os.path.join(ROOT, ".git")):
        pytest.skip("not a git checkout")
    r = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("git unavailable")
    bad = [f for f in r.stdout.splitlines()
           if f.endswith((".so", ".o", ".ncu-rep", ".nsys-rep")) or "/_build/" in f or f.startswith("_work/")]
    assert not bad, bad
