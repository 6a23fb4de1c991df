"""Test helpers: build/load libnfe, and run the oracle and the library on one input."""
import numpy as np

import paper_2605_22214_gb300 as nfe
from paper_2605_22214_gb300 import build as nfe_build


def lib():
    nfe_build.build()
    return nfe.load()


def rel(a, b):
    """max |a - b| / max |b| (relative error of a field)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.abs(b).max()
    return float(np.abs(a - b).max() / scale) if scale > 0 else float(np.abs(a - b).max())
