"""Loader for the stored oracle values in tests/golden/oracle_nll.json."""
import hashlib
import json
import os

import numpy as np

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_nll.json")
BINNED_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_binned.json")


def cases():
    with open(PATH) as f:
        return json.load(f)["cases"]


def columns_sha256(cols):
    h = hashlib.sha256()
    for c in cols:
        h.update(np.ascontiguousarray(c, dtype="<f8").tobytes())
    return h.hexdigest()


def binned():
    """(doc, [(counts, [(theta, evaluation)])]) of the stored binned values;
    theta rebuilt from the stored recipe (the seeded workload draw + shift)."""
    from paper_2003_12861_gb300 import workloads as W

    with open(BINNED_PATH) as f:
        doc = json.load(f)
    P = W.binned_model()["n_params"]
    th = W.binned_toy_thetas(len(doc["cases"]), doc["theta_seed"], P)
    out = []
    for t, case in enumerate(doc["cases"]):
        counts = np.array([float(c) for c in case["counts"].split()])
        out.append((counts, [(th[t] + ev["shift"], ev) for ev in case["evaluations"]]))
    return doc, out
