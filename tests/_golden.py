"""Reader for the small text fixtures under tests/golden (paper values)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read(name):
    """Return (keys, rows): 'key value...' lines go to keys, numeric-only
    lines to rows.  Lines starting with '#' are citations/comments."""
    keys, rows = {}, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0].lstrip("-").isdigit():
                rows.append([int(v) for v in parts])
            else:
                vals = [int(v) for v in parts[1:]]
                keys[parts[0]] = vals[0] if len(vals) == 1 else vals
    return keys, np.asarray(rows, dtype=np.int32)
