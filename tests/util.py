"""Small helpers shared by the tests."""
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def read_golden(name):
    """Parse a tests/golden fixture: 'key v1 v2 ...' lines or bare rows."""
    path = os.path.join(ROOT, "tests", "golden", name)
    keyed, rows = {}, []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            try:
                rows.append([int(p) for p in parts])
            except ValueError:
                keyed[parts[0]] = [int(p) for p in parts[1:]]
    return keyed, rows
