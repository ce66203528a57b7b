"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/pbbem.h declares; the Python binding declares the same
set. No compute call is made here."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pbbem.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(pb_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pb_mesh_load", "pb_near_build", "pb_op_apply", "pb_rhs_charges", "pb_solve", "pb_energy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2108_10481_gb300 import build, native
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(native.SIGNATURES) == set(declared_functions())
    L = native.load()
    assert L.pb_version().decode().startswith("pbbem")


def test_init_without_gpu_fails_loudly():
    """On a machine without a CUDA device the context cannot be created and
    the binding raises instead of falling back to anything."""
    import torch
    if torch.cuda.is_available():
        return
    import paper_2108_10481_gb300 as pb
    try:
        pb.pb_init(0)
    except pb.PBError as e:
        assert e.code in (-1, -6)
    else:
        raise AssertionError("pb_init succeeded without a GPU")
