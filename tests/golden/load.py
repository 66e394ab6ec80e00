"""Readers for the paper's printed values stored as text fixtures in this folder."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def printed():
    out = {}
    with open(os.path.join(HERE, "printed_values.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                out[k] = float(v)
    return out


def table1():
    rows = []
    with open(os.path.join(HERE, "table1_cascade.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                kl, ki, p, s = line.split()
                rows.append((int(kl), int(ki), p, s))
    return rows
