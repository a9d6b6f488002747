"""Build libhyrf.so (sm_103a) in-tree from csrc/*.cu with nvcc.

Each translation unit is compiled in parallel; geom.cu (pre-cull and
projection) is compiled with -fmad=false so its integer decisions follow the
documented FP32 operation order. Output: paper_2509_17083_gb300/libhyrf.so.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
OUT = os.path.join(HERE, "libhyrf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# object name -> (source, extra nvcc flags)
UNITS = {
    "api": ("api.cu", []),
    "geom": ("geom.cu", ["-fmad=false"]),
    "fields0": ("fields.cu", ["-DHYRF_FIELDS_PART=0"]),
    "fields1": ("fields.cu", ["-DHYRF_FIELDS_PART=1"]),
    "fields2": ("fields.cu", ["-DHYRF_FIELDS_PART=2"]),
    "fields3": ("fields.cu", ["-DHYRF_FIELDS_PART=3"]),
    "fields_tc": ("fields_tc.cu", []),
    "fields_tc_bwd": ("fields_tc_bwd.cu", []),
    "gather": ("gather.cu", []),
    "optim": ("optim.cu", []),
    "densify": ("densify.cu", []),
    "explicit": ("explicit.cu", []),
    "codec": ("codec.cu", []),
    "proj_bwd": ("proj_bwd.cu", []),
    "sort": ("sort.cu", []),
    "noalloc": ("noalloc.cu", []),
    "raster": ("raster.cu", []),
    "loss": ("loss.cu", []),
}


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "hyrf.h"))
    return files


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(f) > t for f in _deps() + [__file__])


def _compile(name, spec, verbose):
    unit, extra = spec
    src = os.path.join(CSRC, unit)
    obj = os.path.join(BUILD, name + ".o")
    if not _stale(obj, src):
        return obj
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj + ".tmp"] + extra
    if verbose:
        cmd.append("-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {name} ({unit}):\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force=False, verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
    with cf.ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda kv: _compile(kv[0], kv[1], verbose), UNITS.items()))
    if os.path.exists(OUT) and all(os.path.getmtime(o) <= os.path.getmtime(OUT) for o in objs):
        return OUT
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
