"""FP64/FP32 FMA throughput of the current GPU (corroborates the roofline peak).

  python -m paper_1412_5070_gb300.fma_peak

Compiles csrc/fma_peak.cu for sm_103a into _build/ and runs it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    exe = os.path.join(out, "fma_peak")
    subprocess.run(["nvcc", "-O3", "-gencode", "arch=compute_103a,code=sm_103a",
                    os.path.join(HERE, "csrc", "fma_peak.cu"), "-o", exe], check=True)
    subprocess.run([exe], check=True)


if __name__ == "__main__":
    main()
