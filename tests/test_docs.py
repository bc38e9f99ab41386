"""Repository layout rules (CPU): the design notes' file map names only files that exist and
covers every source; the product package never uses the oracle."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1901_09593_gb300")


def _file_map_paths():
    txt = open(os.path.join(ROOT, "DESIGN.md"), encoding="utf-8").read()
    sec = txt[txt.index("## 14."):]
    return sorted(set(re.findall(r"`([A-Za-z0-9_./*-]+\.(?:py|cu|cuh|h|c|md|txt))`", sec)))


def _exists(p):
    for base in (ROOT, PKG, os.path.join(PKG, "csrc")):
        full = os.path.join(base, p)
        if "*" in p:
            import glob
            if glob.glob(full):
                return True
        elif os.path.exists(full):
            return True
    return False


def test_file_map_names_existing_files():
    paths = _file_map_paths()
    assert len(paths) > 20
    missing = [p for p in paths if not _exists(p)]
    assert not missing, missing


def test_every_source_file_is_in_the_file_map():
    named = " ".join(_file_map_paths())
    srcs = [f for f in os.listdir(os.path.join(PKG, "csrc")) if f.endswith((".cu", ".cuh", ".h"))]
    srcs += [f for f in os.listdir(PKG) if f.endswith(".py") and f != "__init__.py"]
    unnamed = [f for f in srcs if f not in named]
    assert not unnamed, unnamed


def test_product_package_never_uses_the_oracle():
    # the oracle is test infrastructure: nothing under the package imports, loads or builds it
    hits = []
    for dirpath, _, files in os.walk(PKG):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn), encoding="utf-8").read()
                if re.search(r"^\s*(import oracle|from oracle\b)|liboracle|msbm_oracle", txt, re.M):
                    hits.append(fn)
    assert not hits, hits


def test_profile_summaries_give_their_command():
    # each ncu summary states the command that made it: clocks left alone, committed files only
    pdir = os.path.join(ROOT, "profiles")
    names = [f for f in os.listdir(pdir) if f.endswith(".md") and f != "README.md"]
    assert names
    index = open(os.path.join(pdir, "README.md"), encoding="utf-8").read()
    for fn in names:
        txt = open(os.path.join(pdir, fn), encoding="utf-8").read()
        assert "ncu " in txt and "--clock-control none" in txt, fn
        assert "_work" not in txt, fn
        assert f"`{fn}`" in index, fn
