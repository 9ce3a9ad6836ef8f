"""Readers for the text fixtures under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
LETTER = {c: i for i, c in enumerate("ABCDEF")}


def worked_example():
    """Parsed records of worked_example_figs1_3.txt, ids as ints 0..5."""
    out = {"batch": [], "rankall": [], "rank": [], "name": [], "chiplus": []}
    with open(os.path.join(GOLDEN, "worked_example_figs1_3.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, *rest = line.split()
            vals = [LETTER[t] if t in LETTER else int(t) for t in rest]
            out[kind].append(tuple(vals))
    return out
