"""Regenerate the per-process CUDA headers under csrc/gen/."""
import os
import sys

from .procgen import PROCS, generate

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "csrc", "gen")


def main(check: bool = False) -> int:
    os.makedirs(OUT, exist_ok=True)
    stale = []
    for pid in sorted(PROCS):
        text = generate(pid)
        path = os.path.join(OUT, "proc%d.cuh" % pid)
        old = open(path).read() if os.path.exists(path) else None
        if old != text:
            stale.append(path)
            if not check:
                with open(path, "w") as f:
                    f.write(text)
    if check and stale:
        print("stale generated files:", stale)
        return 1
    return 0


if __name__ == "__main__":
    sys.exit(main(check="--check" in sys.argv))
