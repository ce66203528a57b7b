"""Builds (with gcc) and loads the oracle's C core. Test infrastructure only."""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bem_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_OUT = os.path.join(_OUT_DIR, "libbem_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile bem_oracle.c into a shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        # no contraction into fused multiply-adds: the distance band's decision
        # is then the same on every machine and in the CUDA library's host code
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", "-std=c11", _SRC, "-o", tmp,
               "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I = ctypes.c_int
            D = ctypes.c_double
            # singular rules: sizes int[3] (coincident, edge, vertex), nodes and weights concatenated
            L.oracle_pair_blocks.argtypes = [P, P, I64, I64, I, P, P, P, P, P, D, D, I, P, P, P]
            L.oracle_assemble_dense.argtypes = [P, I64, P, I64, I, P, P, P, P, P, D, D, I, P, P, I] + [P] * 7
            L.oracle_assemble_rows.argtypes = [P, I64, P, I64, P, I64, I, P, P, P, P, P, D, D, I, P, P, I] + [P] * 7
            L.oracle_rhs.argtypes = [P, I64, P, I64, I, P, P, P, P, I64, D, P, P]
            L.oracle_reaction_potential.argtypes = [P, I64, P, I64, I, P, P, P, P, P, I64, P]
            L.oracle_band_pair_count.argtypes = [P, P, I64, D, I]
            L.oracle_band_pair_count.restype = I64
            for f in (L.oracle_pair_blocks, L.oracle_assemble_dense, L.oracle_assemble_rows,
                      L.oracle_rhs, L.oracle_reaction_potential):
                f.restype = ctypes.c_int
            _lib = L
    return _lib
