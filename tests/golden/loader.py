"""Readers for the hand-worked fixtures in this folder."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _vecs(text):
    return np.array([[int(x) for x in part.split()] for part in text.split("|")], np.int64)


def stamp_cases():
    """Cases of stamp_hand_worked.txt as dicts with N, F, A, S, L."""
    cases, cur = [], None
    with open(os.path.join(HERE, "stamp_hand_worked.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tag, _, rest = line.partition(" ")
            if tag == "case":
                cur = {"name": rest}
                cases.append(cur)
            elif tag == "N":
                cur["N"] = int(rest)
            elif tag in ("F", "A", "S"):
                cur[tag] = _vecs(rest)
            elif tag == "L":
                cur["L"] = np.array([int(x) for x in rest.split()], np.int8)
    return cases
