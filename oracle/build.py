"""Builds the oracle's C library (``libppo.so``) in place with gcc.

Test infrastructure: building the checker is not using it.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(HERE, "libppo.so")


def build(force: bool = False) -> str:
    out = library_path()
    src = os.path.join(HERE, "ppo.c")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
                           "-o", tmp, src])
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
