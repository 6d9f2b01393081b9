"""Compile the FP64 CPU oracle (test infrastructure only) into a shared library.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg use
the result.  Plain gcc, no CUDA: the oracle shares nothing with the CUDA path.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")


def lib_path(plant: int = 0, out_dir: str | None = None) -> str:
    out_dir = out_dir or os.path.join(HERE, "_build")
    name = "liboracle.so" if plant == 0 else f"liboracle_plant{plant}.so"
    return os.path.join(out_dir, name)


def build(plant: int = 0, out_dir: str | None = None, force: bool = False) -> str:
    """Build liboracle.so (or a planted-mistake variant); return its path."""
    out = lib_path(plant, out_dir)
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           f"-DORACLE_PLANT={int(plant)}", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
