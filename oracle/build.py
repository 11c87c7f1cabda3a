"""Compiles the C oracle (test infrastructure only) into oracle/_build/.

    python oracle/build.py            # the oracle
    python oracle/build.py --plant K  # a deliberately wrong variant for pin-sensitivity tests
"""
from __future__ import annotations

import argparse
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cfpq_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")


def lib_path(plant: int = 0) -> str:
    name = "liboracle.so" if plant == 0 else f"liboracle_plant{plant}.so"
    return os.path.join(OUT_DIR, name)


def build(plant: int = 0, force: bool = False) -> str:
    out = lib_path(plant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", f"-DORACLE_PLANT={plant}", SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--plant", type=int, default=0)
    ap.add_argument("--force", action="store_true")
    a = ap.parse_args()
    print(build(a.plant, a.force))
    sys.exit(0)
