"""Reader for the hand-derived fixtures under tests/golden/ (key value... lines)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict:
    rows: dict[str, list[list[str]]] = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows.setdefault(key, []).append(vals)
    out: dict = {}
    for key in ("n", "m", "d", "k", "N"):
        out[key] = int(rows[key][0][0])
    for key in ("U", "P", "Q"):
        out[key] = np.array([[float(v) for v in r] for r in rows[key]], dtype=np.float32)
    out["topk"] = np.array([[int(v) for v in r] for r in rows["topk"]], dtype=np.int64)
    out["tau"] = np.array([float(v) for v in rows["tau"][0]])
    for key in ("tid", "scores", "topn_ids", "topn_scores", "uscore", "counts"):
        out[key] = np.array([int(v) for v in rows[key][0]], dtype=np.int64)
    return out


def names() -> list[str]:
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))
