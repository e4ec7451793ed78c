"""Build the sm_103a shared library libgb300dft.so in-tree (paper_0910_1531_gb300/_build/).

The translation units are compiled in parallel with nvcc and linked with the static
CUDA runtime.  Usage:  python -m paper_0910_1531_gb300.build  [--force]
"""

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB_NAME = "libgb300dft.so"
# (source, object name, extra defines); kinst.cu is compiled once per (precision, axis length)
CT_SIZES = (0, 32, 48, 64, 96, 128, 256)
SOURCES = ([("api.cu", "api", []), ("bulk.cpp", "bulk", []), ("noalloc.cu", "noalloc", []),
            ("dispatch.cu", "dispatch", []), ("newton.cu", "newton", [])]
           + [("kinst.cu", f"kinst_{r}_{n}", [f"-DDFT_INST_REAL={r}", f"-DDFT_INST_N={n}"])
              for r in ("float", "double") for n in CT_SIZES])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgb300dft.so")
    return cand


def lib_path():
    return os.path.join(BUILD, LIB_NAME)


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "gb300dft.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date():
    lib = lib_path()
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _compile(entry, extra):
    src, name, defines = entry
    obj = os.path.join(BUILD, name + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17", "-lineinfo",
           "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + ARCH + defines + extra
    if src.endswith(".cpp"):
        cmd += ["-x", "c++"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
    return obj, res.stderr


def build(force=False, verbose=False, extra=()):
    """Compile and link; returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and up_to_date():
        return lib_path()
    workers = max(2, min(len(SOURCES), os.cpu_count() or 4))
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra)), SOURCES))
    objs = [r[0] for r in results]
    if verbose:
        for _, log in results:
            if log:
                print(log, file=sys.stderr)
    tmp = lib_path() + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-cudart=static"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib_path())
    return lib_path()


if __name__ == "__main__":
    args = sys.argv[1:]
    extra = ["-Xptxas", "-v"] if "--ptxas-v" in args else []
    print(build(force="--force" in args or bool(extra), verbose=bool(extra), extra=extra))
