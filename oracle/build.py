"""Compiles the FP64 oracle (``lbm_oracle.c``) into ``liblbm_oracle.so``.

Test infrastructure: only the tests, the smoke check and the benchmark's
CPU-baseline leg use the library this builds.  Plain ``gcc``, no
machine-specific flags, so the same source builds on x86_64 and aarch64.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "liblbm_oracle.so")


def build(force: bool = False, src: str = SRC, out: str = LIB) -> str:
    """Builds the oracle library if it is missing or older than its source."""
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
