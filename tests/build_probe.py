"""Builds tests/philox_probe.cu (test infrastructure) with nvcc for sm_103a
into tests/_build/libphilox_probe.so."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "philox_probe.cu")
OUT = os.path.join(HERE, "_build", "libphilox_probe.so")
CSRC = os.path.join(os.path.dirname(HERE), "paper_0801_1222_gb300", "csrc")


def build() -> str:
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    deps = [SRC, os.path.join(CSRC, "hfq_device.cuh")]
    if os.path.exists(OUT) and os.path.getmtime(OUT) >= max(os.path.getmtime(d) for d in deps):
        return OUT
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = [os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
           "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-I", CSRC, "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build())
