"""Loader for the stored oracle values in tests/golden/oracle_nll.json."""
import hashlib
import json
import os

import numpy as np

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_nll.json")


def cases():
    with open(PATH) as f:
        return json.load(f)["cases"]


def columns_sha256(cols):
    h = hashlib.sha256()
    for c in cols:
        h.update(np.ascontiguousarray(c, dtype="<f8").tobytes())
    return h.hexdigest()
