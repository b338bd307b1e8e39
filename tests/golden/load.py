"""Readers for the golden fixtures (plain text, each file cites its source)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def philox_kat():
    rows = []
    with open(os.path.join(HERE, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows
