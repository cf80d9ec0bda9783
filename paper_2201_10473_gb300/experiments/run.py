"""Compile (nvcc, sm_103a) and run one of the measurement programs of this directory."""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
PROGRAMS = ("tc_toeplitz", "bitsliced_leaf")


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    if len(argv) != 1 or argv[0] not in PROGRAMS:
        sys.exit(f"usage: python -m paper_2201_10473_gb300.experiments.run {{{','.join(PROGRAMS)}}}")
    name = argv[0]
    exe = os.path.join(tempfile.mkdtemp(prefix="gf2x_exp_"), name)
    cmd = [os.environ.get("NVCC", "nvcc"), "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "include"), os.path.join(HERE, name + ".cu"), "-o", exe]
    subprocess.run(cmd, check=True)
    sys.exit(subprocess.run([exe]).returncode)


if __name__ == "__main__":
    main()
