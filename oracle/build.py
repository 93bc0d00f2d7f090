"""Compile the plain-C MicSA oracle into a shared library (test infrastructure).

The oracle is checked by the tests and used by the benchmark's CPU baseline;
the product library never links it. ``build(mutant=k)`` compiles a copy with
one planted mistake (``-DORC_MUTANT=k``) for the pin-sensitivity tests.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "micsa_oracle.c")
HDR = os.path.join(HERE, "micsa_oracle.h")
OUT_DIR = os.path.join(HERE, "_build")


def lib_path(mutant=0):
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(OUT_DIR, name)


def build(mutant=0, force=False):
    out = lib_path(mutant)
    newest_src = max(os.path.getmtime(SRC), os.path.getmtime(HDR), os.path.getmtime(__file__))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest_src:
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = f"{out}.{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra", "-ffp-contract=off",
           f"-DORC_MUTANT={int(mutant)}", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)  # atomic, so concurrent builders never load a partial file
    return out


if __name__ == "__main__":
    print(build(force=True))
