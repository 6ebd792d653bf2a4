"""Build step of the CUDA library: nvcc for sm_103a into the package directory."""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = [os.path.join(_HERE, "csrc", f) for f in ("ce_mppi_api.cu", "k_rollout.cu", "k_cluster.cu",
                                                              "ce_mppi_noalloc.cu",
                                                              "ce_mppi_server.cu")]
HEADERS = [os.path.join(_HERE, "csrc", "ce_mppi_internal.cuh"),
           os.path.join(_HERE, "csrc", "ce_mppi_host.h"),
           os.path.join(os.path.dirname(_HERE), "include", "ce_mppi.h")]
OUT = os.path.join(_HERE, "libcemppi.so")
NVCC_FLAGS = ["-std=c++17", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared"]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libcemppi.so unless it is newer than every source."""
    deps = SOURCES + HEADERS
    if not force and os.path.exists(OUT) and all(
            os.path.getmtime(OUT) >= os.path.getmtime(s) for s in deps):
        return OUT
    cmd = ["nvcc", *NVCC_FLAGS, "-o", OUT, *SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    return OUT


if __name__ == "__main__":
    print(build(force=True, verbose=True))
