import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "_build", "pipe_peaks")


def main():
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                           "-o", OUT, os.path.join(HERE, "pipe_peaks.cu")])
    sys.exit(subprocess.call([OUT]))


if __name__ == "__main__":
    main()
