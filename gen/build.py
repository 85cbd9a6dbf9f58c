"""Build gen/libahsgen.so (device input generators) with nvcc for sm_103a."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "device.cu")
LIB = os.path.join(HERE, "libahsgen.so")


def build() -> str:
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([nvcc if os.path.exists(nvcc) else "nvcc", "-gencode",
                               "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                               "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
                               "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build())
