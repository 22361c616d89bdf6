"""Reader for the small text fixtures under tests/golden/ (each cites its source)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_kv(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=", 1)
            out[k.strip()] = v.strip()
    return out


def read_rows(name: str) -> np.ndarray:
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(t) for t in line.split()])
    return np.array(rows, dtype=np.int64)


def parse_terms(s: str):
    """'e e e : c ; e e e : c' -> (uint8 rows, float64 coefs)."""
    rows, coefs = [], []
    for part in s.split(";"):
        e, c = part.split(":")
        rows.append([int(t) for t in e.split()])
        coefs.append(float(c))
    return np.array(rows, dtype=np.uint8), np.array(coefs, dtype=np.float64)


def floats(s: str) -> np.ndarray:
    return np.array([float(t) for t in s.split()])


def ints(s: str) -> list:
    return [int(t) for t in s.split()]
