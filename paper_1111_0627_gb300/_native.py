"""Build and load the solver's shared library (``libocm.so``, C ABI of
``include/ocm.h``).

The library is compiled in-tree with nvcc for sm_103a only.  There is no
fallback: if the library cannot be built or loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
CSRC = os.path.join(_PKG, "csrc")
BUILD = os.path.join(_PKG, "_build")
LIB_PATH = os.path.join(BUILD, "libocm.so")
INCLUDE = os.path.join(_ROOT, "include")
SOURCES = ["sweep.cu", "sweep_tiles.cu", "sweep_window.cu", "evaluate.cu", "batch.cu", "batch_small.cu", "api.cu",
           "static_ws.cu", "scc.cu", "single.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]

_lock = threading.Lock()
_lib = None


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA solver cannot be built")


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "ocm.h"))
    return files


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu into _build/libocm.so (sm_103a), unless up to date."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(f) <= t for f in _deps()):
            return LIB_PATH
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + f".{os.getpid()}.o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"],
                       capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class OcmOptions(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("eta_num", ctypes.c_void_p), ("eta_den", ctypes.c_void_p),
                ("potential", ctypes.c_void_p), ("policy", ctypes.c_void_p),
                ("edges_per_lane", ctypes.c_int32), ("sweep_threads", ctypes.c_int32),
                ("sweep_kind", ctypes.c_int32), ("wait_limit_ms", ctypes.c_int32),
                ("init_policy", ctypes.c_void_p), ("transit", ctypes.c_void_p),
                ("batch_small_vertices", ctypes.c_int32), ("reserved1", ctypes.c_int32)]


class OcmStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("cycles", ctypes.c_int32),
                ("detect_rounds", ctypes.c_int32), ("value_rounds", ctypes.c_int32),
                ("switched", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("detect_items", ctypes.c_int64), ("value_items", ctypes.c_int64),
                ("graph_loop", ctypes.c_int32), ("rebuild_levels", ctypes.c_int32),
                ("batch_small_graphs", ctypes.c_int32), ("sweep_kind", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


# exported symbols and their signatures (kept in step with include/ocm.h)
SIGNATURES = {
    "ocm_workspace_size": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32]),
    "ocm_workspace_size_single": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32]),
    "ocm_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                 ctypes.c_int32, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_size_t,
                                 ctypes.c_void_p, ctypes.POINTER(OcmOptions),
                                 ctypes.POINTER(OcmStats)]),
    "ocm_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "ocm_backward_ratio": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "ocm_workspace_size_batch": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "ocm_backward_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "ocm_solve_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                       ctypes.POINTER(OcmOptions), ctypes.POINTER(OcmStats)]),
    "ocm_solve_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p,
                                        ctypes.POINTER(OcmOptions), ctypes.POINTER(OcmStats)]),
    "ocm_workspace_size_scc": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32]),
    "ocm_scc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                               ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p,
                               ctypes.c_size_t, ctypes.c_void_p]),
    "ocm_workspace_size_solve_scc": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32]),
    "ocm_solve_scc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                     ctypes.POINTER(OcmOptions), ctypes.POINTER(OcmStats)]),
    "ocm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ocm_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "ocm_profile_collect": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int64)]),
    "ocm_version": (ctypes.c_int, []),
}


def load(path: str | None = None):
    """Build if needed and load the library; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(path or build())
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib
