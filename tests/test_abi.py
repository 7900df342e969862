"""The C-ABI library loads on a CPU-only host and exports every declared symbol.

No compute calls are made here (there may be no GPU): the library is loaded
with ctypes and each function named in include/difvm.h is looked up.
"""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "difvm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(difvm_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    names = declared()
    for n in ["difvm_mesh_create", "difvm_grad_gauss", "difvm_div_flux", "difvm_laplacian_apply",
              "difvm_krylov_solve", "difvm_piso_step", "difvm_windkessel_update",
              "difvm_grad_gauss_bwd", "difvm_div_flux_bwd", "difvm_laplacian_apply_bwd",
              "difvm_krylov_solve_bwd", "difvm_windkessel_update_bwd", "difvm_piso_step_record",
              "difvm_piso_step_bwd", "difvm_piso_tape_bytes"]:
        assert n in names, n


def test_library_exports_every_declared_symbol():
    from paper_2603_15920_b300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_oracle_library_builds_and_loads():
    import oracle
    assert hasattr(oracle.lib(), "om_piso_step")
    assert hasattr(oracle.lib(), "om_piso_step_bwd")
