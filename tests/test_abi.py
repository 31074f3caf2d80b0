"""The C-ABI library builds, loads without a GPU and exports every symbol the header
declares; its host-side constants (computed independently of the oracle) agree with the
oracle's exact ones.  No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dartminhash.h")


@pytest.fixture(scope="module")
def lib():
    import paper_2005_11547_gb300 as pkg
    pkg.build()
    return pkg.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["dm_create", "dm_destroy", "dm_sketch", "dm_sketch_bbit", "dm_lsh",
                     "dm_sync_status", "dm_strerror", "dm_sketch_host"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    import paper_2005_11547_gb300 as pkg
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dm_[a-z_0-9]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_checked_build_exports_the_same_symbols(lib):
    """The checked build (index checks compiled in) is built beside the product library, loads
    without a GPU, exports every declared symbol and says that it is the checked build."""
    import paper_2005_11547_gb300 as pkg
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_CHECKED], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dm_[a-z_0-9]+)", out))
    assert not [n for n in declared_functions() if n not in exported]
    checked = ctypes.CDLL(pkg.LIB_CHECKED)
    checked.dm_build_flags.restype = ctypes.c_int32
    assert checked.dm_build_flags() & 1 == 1
    assert pkg.dm_build_flags() & 1 == 0


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "h.c"
    src.write_text('#include "dartminhash.h"\nint main(void){return DM_OK;}\n')
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", f"-I{os.path.dirname(HEADER)}",
                           "-c", str(src), "-o", str(tmp_path / "h.o")])


def test_t_of_k_matches_oracle(lib, oracle_mod):
    import paper_2005_11547_gb300 as pkg
    for k in list(range(1, 2049)) + [4095, 4096, 8191, 8192]:
        assert pkg.dm_t_of_k(k) == oracle_mod.t_of_k(k), k
    assert pkg.dm_t_of_k(0) == 0


def test_poisson_table_matches_oracle(lib, oracle_mod):
    import paper_2005_11547_gb300 as pkg
    assert pkg.dm_poisson_thresholds() == [int(v) for v in oracle_mod.poisson_thresholds()]


def test_strerror(lib):
    import paper_2005_11547_gb300 as pkg
    assert pkg.dm_strerror(0) == "ok"
    assert "range" in pkg.dm_strerror(5)


def test_product_path_does_not_touch_oracle():
    """The library and its binding never import, load or run anything under oracle/."""
    pkg_dir = os.path.join(ROOT, "paper_2005_11547_gb300")
    for dirpath, _, files in os.walk(pkg_dir):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "dm_oracle" not in text and "dmo_" not in text, f
