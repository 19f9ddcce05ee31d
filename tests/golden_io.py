"""Readers for the text fixtures under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def records(name):
    """Yield (kind, {key: value-string}) for every non-comment line."""
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, *fields = line.split()
            yield kind, dict(f.split("=", 1) for f in fields)


def ints(s):
    return [int(v) for v in s.split(",")]
