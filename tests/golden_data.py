"""Reader of the text fixtures under tests/golden/ ('# ' comment lines, 'key: values')."""
from __future__ import annotations

import os
from fractions import Fraction

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict[str, str]:
    out = {}
    with open(os.path.join(GOLDEN, name), encoding="utf-8") as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, val = line.partition(":")
            out[key.strip()] = val.strip()
    return out


def numbers(text: str) -> list[float]:
    """Whitespace-separated numbers; 'a/b' is an exact ratio evaluated once."""
    vals = []
    for tok in text.split():
        if "/" in tok:
            num, den = tok.split("/")
            vals.append(float(Fraction(num) / Fraction(den)))
        else:
            vals.append(float(tok))
    return vals


def entries(name: str, key: str) -> list[str]:
    """Every value of a key that appears on several lines, in file order."""
    out = []
    with open(os.path.join(GOLDEN, name), encoding="utf-8") as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, _, val = line.partition(":")
            if k.strip() == key:
                out.append(val.strip())
    return out
