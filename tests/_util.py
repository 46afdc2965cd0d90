"""Shared helpers for the test modules (no smoothing arithmetic here)."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Parity bar for the FP32 CUDA path against the FP64 oracle on [0,1] images.
MAX_ABS_TOL = 2e-4
RMS_TOL = 1e-5


def declared_symbols():
    """Every function name declared in include/*.h."""
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(ils_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def err_stats(a, b):
    d = np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)
    return float(np.abs(d).max()), float(np.sqrt(np.mean(d * d)))
