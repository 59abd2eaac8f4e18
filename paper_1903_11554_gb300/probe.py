"""Build and run the FP64 pipe probe (csrc/probe_fp64.cu) on the current GPU:
python -m paper_1903_11554_gb300.probe"""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile

from . import build


def main() -> int:
    src = os.path.join(build.CSRC, "probe_fp64.cu")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "probe_fp64")
        subprocess.check_call([build.nvcc(), "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe, src])
        return subprocess.call([exe])


if __name__ == "__main__":
    sys.exit(main())
