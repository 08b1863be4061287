"""Writes tests/golden/chen_tiny.json: tiny seeded pairs with k(x,y) from the
oracle's Chen-identity brute force (truncated signature inner product), the
one oracle routine that shares no arithmetic with the tile-series code.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402

cases = []
for seed, (L1, L2, d, scale, M) in enumerate([(3, 4, 2, 0.6, 18), (2, 2, 3, 0.8, 12),
                                               (4, 1, 2, 0.5, 18), (1, 5, 3, 0.4, 12),
                                               (3, 3, 2, 1.1, 22)]):
    rng = np.random.default_rng(900 + seed)
    dx = np.round(rng.standard_normal((L1, d)) * scale, 6)
    dy = np.round(rng.standard_normal((L2, d)) * scale, 6)
    k, levels = oracle.chen_pair(dx, dy, M, levels=True)
    cases.append({"name": f"chen_{L1}x{L2}_d{d}", "dx": dx.tolist(), "dy": dy.tolist(),
                  "level": M, "tail": float(levels[-1]), "k": k})
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "chen_tiny.json"), "w") as f:
    json.dump(cases, f, indent=1)
print("wrote", len(cases), "cases")
