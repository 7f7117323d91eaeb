"""Build and load the host build of the CUDA path's device arithmetic
(gpss_host_harness.cu compiled by nvcc as host code into a shared library),
for CPU tests of the device functions."""
import ctypes
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
SRC = os.path.join(HERE, "gpss_host_harness.cu")
OUT = os.path.join(HERE, "_build", "libgpss_hostmath.so")
CSRC = os.path.join(ROOT, "paper_2601_02527_gb300", "csrc")


def load():
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    deps = [SRC] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < max(map(os.path.getmtime, deps)):
        nvcc = "/usr/local/cuda/bin/nvcc"
        tmp = OUT + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                               "-I", os.path.join(ROOT, "include"), "-I", CSRC, SRC, "-o", tmp])
        os.replace(tmp, OUT)
    lib = ctypes.CDLL(OUT)
    P = ctypes.POINTER
    d, f, i32, i64 = ctypes.c_double, ctypes.c_float, ctypes.c_int, ctypes.c_int64
    vp = ctypes.c_void_p
    lib.hh_discretize.argtypes = [i32, d, d, d, P(d)]
    lib.hh_discretize_dual.argtypes = [d, d, d, P(d)]
    lib.hh_discretize_tangents.argtypes = [d, d, d, P(d)]
    lib.hh_solve.argtypes = [i32, P(f), P(f), P(f), i32]
    lib.hh_solve.restype = f
    lib.hh_dim.argtypes = [i32]
    lib.hh_table_check.argtypes = [d, d, i32]
    lib.hh_table_check.restype = d
    lib.hh_taylor_k_check.argtypes = [d, d]
    lib.hh_taylor_k_check.restype = d
    lib.hh_combine.argtypes = [i32, P(f), P(f), P(f)]
    lib.hh_chunk_loglik.argtypes = [i32, P(f), P(f), P(f), P(f), d, d, d]
    lib.hh_chunk_loglik.restype = d
    lib.hh_boundary_adjoint.argtypes = [i32, P(f), P(f), P(f), P(f), P(f), P(f)]
    lib.hh_obs_dim.argtypes = [i32]
    lib.hh_prod_disc.argtypes = [i32, d, P(d), P(d), P(d)]
    lib.hh_observe.argtypes = [i32, i32, f, P(f), P(f), P(f), P(f), P(f), P(f)]
    lib.hh_table_df_check.argtypes = [d, d]
    lib.hh_table_df_check.restype = d
    lib.hh_span_nc.argtypes = [i32]
    lib.hh_span_element.argtypes = [i32, vp, vp, vp, vp, vp, i64, i64, i32, vp]
    lib.hh_span_fold.argtypes = [i32, vp, i32]
    lib.hh_span_fold.restype = d
    lib.hh_predict_cov.argtypes = [i32, vp, vp]
    return lib
