#!/usr/bin/env python3
"""Writes tests/golden/inputs_fingerprint.json: SHA-256 prefixes of a few
seeded inputs drawn by paper_2203_04774_gb300.synth (the input generators,
which hold none of the listing method's arithmetic).

Stored results (the oracle's listing of the largest graph) are computed on
one machine and compared on another, so the same seed must give the same
bits everywhere; tests/test_inputs_fingerprint.py checks these digests on
every machine the tests run on.
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from paper_2203_04774_gb300 import synth  # noqa: E402


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:16]


def fingerprints() -> dict:
    fam = synth.chung_lu_family(64, (1000, 5_000_000), (8, 64), (2.1, 3.0), 5)
    return {
        "chung_lu_weights(2e6, 40, 2.2)": digest(synth.chung_lu_weights(2_000_000, 40, 2.2)),
        "chung_lu(1e5, 20, 2.5, 1)": digest(synth.chung_lu(100_000, 20, 2.5, 1)),
        "chung_lu(1e6, 40, 2.2, 4)": digest(synth.chung_lu(1_000_000, 40, 2.2, 4)),
        "chung_lu_family(64, ..., 5)": digest(np.concatenate(
            [fam["n"].astype(np.float64), fam["deg"], fam["gamma"]])),
        "rmat(16, 16, 0.57, 0.19, 0.19, 2)": digest(synth.rmat(16, 16, 0.57, 0.19, 0.19, 2)),
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "inputs_fingerprint.json"), "w") as f:
        json.dump(fingerprints(), f, indent=1)
        f.write("\n")
