"""Writes tests/golden/tiny_primal_oracle.json by calling only the FP64 oracle.

Workload: the tiny dense primal problem (X 64 x 1024 iid N(0,1) from
synth.tiny_primal(seed=1), lambda = 1e-3, b = 4, H = 200, sampler seed 42),
run as Algorithm 1 (s = 1) and Algorithm 2 (s = 4), and the dual Algorithm 4
on the same X (b' = 8, s = 4, H = 200).  The stored iterates let a test check
that the oracle computes the same numbers on every host (x86 and Arm).

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth   # noqa: E402


def main():
    p = synth.tiny_primal(d=64, n=1024, seed=1)
    w1, _ = oracle.bcd(p.X, p.y, 1e-3, b=4, H=200, seed=42)
    w4, _ = oracle.ca_bcd(p.X, p.y, 1e-3, b=4, s=4, H=200, seed=42)
    a4, wd = oracle.ca_bdcd(p.X, p.y, 1e-3, b=8, s=4, H=200, seed=42)
    out = {
        "workload": "tiny dense primal: X 64x1024 N(0,1) seed 1, lambda 1e-3, seed 42",
        "bcd_b4_H200_w": w1.tolist(),
        "cabcd_b4_s4_H200_w": w4.tolist(),
        "cabdcd_b8_s4_H200_alpha_first16": a4[:16].tolist(),
        "cabdcd_b8_s4_H200_w": wd.tolist(),
        "first_blocks_seed42_b4_N64": oracle.sample_blocks(42, 0, 8, 4, 64).tolist(),
    }
    with open(os.path.join(HERE, "tiny_primal_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
