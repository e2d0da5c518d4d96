"""Compile the FP64 CPU oracle into ``oracle/liboracle.so`` (test infrastructure).

Plain ``g++ -O2 -ffp-contract=off``: no FMA contraction, no vectorisation
flags, no architecture-specific options, so the same source gives the same
results on x86-64 and aarch64 hosts.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(HERE, "fdbb_oracle.cpp")
library_path = os.path.join(HERE, "liboracle.so")

FLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its source."""
    if (not force and os.path.exists(library_path)
            and os.path.getmtime(library_path) >= os.path.getmtime(SOURCE)):
        return library_path
    tmp = library_path + f".tmp{os.getpid()}"
    cmd = ["g++", *FLAGS, SOURCE, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, library_path)
    return library_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
