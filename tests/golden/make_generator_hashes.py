"""Writes generator_hashes.json: SHA-256 digests that freeze the seeded
synthetic exemplar generator (pts_inputs).  Run from the repository root:
    python tests/golden/make_generator_hashes.py
"""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import pts_inputs as P  # noqa: E402

CASES = [(0, 64, 3.0), (0, 256, 4.0), (3, 96, 4.0)]

if __name__ == "__main__":
    out = {f"{s}_{n}_{k}": P.array_digest(P.synthetic_exemplar(s, n, k)) for s, n, k in CASES}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "generator_hashes.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
