"""Writes the stored expected values under tests/golden/ from the oracle only.

schedules.txt: level sizes and iteration counts of Algorithm 1 (n_l, round(w^(l/n_l)),
10 iterations at or below 32 x 32 else 2, Section III-D) for the three single-image
workloads. test_oracle_pins.py checks every entry against exact integer rounding too.

Run from the repository root: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    lines = ["# Algorithm 1 level schedule: WxH: w_l,h_l,k_l for l = 1..n_l",
             "# written by tests/golden/make_golden.py (oracle only)"]
    for w, h in [(128, 128), (2048, 1536), (7680, 4320)]:
        lv = oracle.schedule(w, h)
        lines.append(f"{w}x{h}: " + " ".join(f"{a},{b},{k}" for a, b, k in lv))
    with open(os.path.join(HERE, "schedules.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
