"""Build and run the FP64 pipe throughput program (sm_103a):

    python -m paper_2009_10863_gb300.probe

It prints GFLOP/s of FP64 DFMA on the CUDA cores, of the FP64 tensor-core
MMA shapes, and of both interleaved.
"""
import os
import subprocess
import sys

from ..build import ARCH, BUILD, nvcc

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "fp64_pipes")
    src = os.path.join(HERE, "fp64_pipes.cu")
    subprocess.run([nvcc()] + ARCH + ["-O3", "-lineinfo", src, "-o", exe], check=True)
    sys.exit(subprocess.run([exe]).returncode)


if __name__ == "__main__":
    main()
