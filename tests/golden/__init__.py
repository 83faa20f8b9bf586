"""Loader for the small golden files: values printed in the paper, with citations."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def paper_tables(path: str = os.path.join(HERE, "paper_tables.txt")) -> dict:
    out = {}
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            out[parts[0]] = [float(v) for v in parts[1:]]
    return out
