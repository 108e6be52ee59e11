"""The seeded input generators give the same bits on every machine.

Stored expected values (tests/golden/chunglu1e8.json) are computed by the
oracle on one host and compared with the CUDA path on the GPU host, so a
seed must name the same graph on both.  The digests in
tests/golden/inputs_fingerprint.json were written by
tests/golden/make_inputs_fingerprint.py; the CPU run checks them here, the
GPU run (marked gpu) checks them again on the GPU host.
"""
import json
import os

import pytest

from tests.golden.make_inputs_fingerprint import fingerprints

GOLD = os.path.join(os.path.dirname(__file__), "golden", "inputs_fingerprint.json")


def _check():
    with open(GOLD) as f:
        want = json.load(f)
    assert fingerprints() == want


def test_generator_digests_on_this_host():
    _check()


@pytest.mark.gpu
def test_generator_digests_on_the_gpu_host():
    _check()
