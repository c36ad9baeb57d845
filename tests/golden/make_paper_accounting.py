"""Writes paper_accounting.json: the paper's accounting formulas (Sec. 7)
evaluated with exact integer arithmetic at the configurations of its
rank-96 / rank-128 tables and sweeps (batch 20,000):
  flops      = batch (4 r^3 + 2 r^2 b)            (GFLOPS equation)
  bytes_2r2  = batch (2 r^2 + 2 r b) 8             (bandwidth, A64FX / EPYC)
  bytes_3r2  = batch (3 r^2 + 2 r b) 8             (bandwidth, Xeon 6148: result write counted)
"""
import json
import os

CASES = [(20000, 96, 512), (20000, 96, 1024), (20000, 96, 2048), (20000, 128, 512), (20000, 128, 1024),
         (20000, 128, 2048), (20000, 8, 512), (20000, 16, 1024), (20000, 32, 2048)]


def main():
    out = {"source": "arXiv 2311.07602, Sec. 7: GFLOPS = batch (4 r^3 + 2 r^2 b) / t; "
                     "BW = batch (2 r^2 + 2 r b) 8 B / t (A64FX, EPYC) or batch (3 r^2 + 2 r b) 8 B / t (Xeon 6148)",
           "cases": [{"batch": B, "r": r, "b": b, "flops": B * (4 * r ** 3 + 2 * r * r * b),
                      "bytes_2r2": B * (2 * r * r + 2 * r * b) * 8, "bytes_3r2": B * (3 * r * r + 2 * r * b) * 8}
                     for B, r, b in CASES]}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_accounting.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
