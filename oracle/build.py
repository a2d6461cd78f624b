"""Compile the C oracle into ``oracle/_build/liboracle.so`` (gcc, no FMA contraction).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(HERE, "_build", "liboracle.so")


def build(force: bool = False) -> str:
    out = library_path()
    src = os.path.join(HERE, "nnm_oracle.c")
    hdr = os.path.join(HERE, "nnm_oracle.h")
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-Wall", "-Wextra", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
