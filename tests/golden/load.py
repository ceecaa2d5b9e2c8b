"""Readers of the small text fixtures in this folder (each file cites its passage)."""
import os

_HERE = os.path.dirname(os.path.abspath(__file__))


def rows(name: str):
    """Non-comment lines of a fixture, split on whitespace."""
    out = []
    with open(os.path.join(_HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                out.append(line.split())
    return out


def eq8_table():
    """[((T_m, L, cp_s, cp_l, cp_g, C, He), (T, Fl), note), ...]"""
    out = []
    for r in rows("eq8_inversion.txt"):
        vals = [float(v) for v in r[:9]]
        out.append((tuple(vals[:7]), tuple(vals[7:9]), " ".join(r[9:])))
    return out


def keyed(name: str) -> dict:
    """key -> float, or list of floats when a line holds several values."""
    out = {}
    for r in rows(name):
        vals = [float(v) for v in r[1:]]
        out[r[0]] = vals[0] if len(vals) == 1 else vals
    return out
