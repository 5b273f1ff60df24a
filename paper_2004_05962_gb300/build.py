"""Builds the sm_103a shared library of the package in-tree with nvcc.

Three translation units (C ABI, forward kernels, adjoint kernels) compile in
parallel, then link into ``_build/libbsi_gb300.so`` with the CUDA runtime
linked statically.  ``checked=True`` builds ``libbsi_gb300_checked.so`` with
BSI_CHECKED defined: every global and shared-memory range a kernel touches is
tested first, and a violation sets a bit of the kernel error word (read with
``bsi_check_device_status``) and skips the access instead of faulting.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import pathlib
import subprocess

PKG = pathlib.Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
BUILD = PKG / "_build"
SOURCES = ["bsi_abi.cu", "bsi_forward.cu", "bsi_adjoint.cu", "bsi_probe.cu", "bsi_resample.cu", "bsi_variants.cu", "bsi_rational.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def lib_name(checked: bool = False) -> str:
    return "libbsi_gb300_checked.so" if checked else "libbsi_gb300.so"


def lib_path(checked: bool = False) -> pathlib.Path:
    return BUILD / lib_name(checked)


def _inputs():
    return [CSRC / s for s in SOURCES] + list(CSRC.glob("*.h")) + list(CSRC.glob("*.cuh")) + \
        [INCLUDE / "bsi.h"]


def up_to_date(checked: bool = False) -> bool:
    out = lib_path(checked)
    if not out.exists():
        return False
    t = out.stat().st_mtime
    return all(p.stat().st_mtime <= t for p in _inputs())


def nvcc() -> str:
    cand = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
    return cand if os.path.exists(cand) else "nvcc"


def build(checked: bool = False, force: bool = False, verbose: bool = False,
          ptxas_info: bool = False) -> pathlib.Path:
    """Compiles (if stale) and returns the path of the shared library."""
    if not force and up_to_date(checked):
        return lib_path(checked)
    BUILD.mkdir(parents=True, exist_ok=True)
    tag = "chk" if checked else "rel"
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                    "-I", str(INCLUDE), "-I", str(CSRC)]
    if checked:
        flags += ["-DBSI_CHECKED"]
    if ptxas_info:
        flags += ["-Xptxas", "-v"]

    def compile_one(src: str):
        obj = BUILD / f"{pathlib.Path(src).stem}.{tag}.o"
        cmd = [nvcc(), "-c", str(CSRC / src), "-o", str(obj)] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for _, log in results:
            if log.strip():
                print(log)
    out = lib_path(checked)
    tmp = out.with_name(out.name + f".tmp{os.getpid()}")
    cmd = [nvcc(), "-shared", "-o", str(tmp)] + [str(o) for o, _ in results] + ARCH + \
        ["-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    import argparse

    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--checked", action="store_true")
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true")
    a = ap.parse_args()
    print(build(checked=a.checked, force=a.force, verbose=True, ptxas_info=a.ptxas_info))
