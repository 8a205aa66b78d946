"""Build step of the CUDA library: nvcc -> libcrm.so next to this file (sm_103a)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["crm_bin.cu", "crm_step.cu", "crm_bce.cu", "crm_active.cu", "crm_adjoint.cu", "crm_api.cu"]
LIB = os.path.join(HERE, "libcrm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(HERE, "csrc", f) for f in os.listdir(os.path.join(HERE, "csrc"))]
    deps.append(os.path.join(HERE, "..", "include", "crm.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu of csrc/ into libcrm.so (in-tree, so it ships with the repo)."""
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, "-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-shared",
           "-Xptxas", "-v" if verbose else "-O3", "-o", tmp,
           *[os.path.join(HERE, "csrc", s) for s in SOURCES]]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
