"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/pimc.h declares (no compute calls: runs without a GPU)."""
import os
import re
import subprocess

import pytest

from paper_1103_4887_gb300 import build as pbuild
from paper_1103_4887_gb300 import pimc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(pimc_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    return pbuild.build()


def test_header_lists_the_boundary():
    names = declared_functions()
    for must in ("pimc_create", "pimc_set_data", "pimc_sweep", "pimc_action", "pimc_grad",
                 "pimc_moments", "pimc_histograms"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(pimc_[a-z0-9_]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert set(pimc.EXPORTS) <= exported


def test_library_loads_and_binds(libpath):
    L = pimc.load(libpath)
    for name in declared_functions():
        assert hasattr(L, name)
