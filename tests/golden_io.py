"""Reader for the hand-worked fixtures in tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    """Return (windows, expected) where windows is a list of (src, dst) arrays."""
    windows, cur, expected = [], None, {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(":")
            vals = [int(v) for v in rest.split()]
            if key == "window":
                cur = []
                windows.append(cur)
            elif key == "packets":
                if cur is None:
                    cur = []
                    windows.append(cur)
                cur.append(tuple(vals))
            else:
                expected[key] = vals
    out = []
    for w in windows:
        a = np.array(w, dtype=np.uint32).reshape(-1, 2)
        out.append((a[:, 0].copy(), a[:, 1].copy()))
    return out, expected


FIXTURES = ["hand_window.txt", "extreme_addresses.txt", "star.txt", "reverse_star.txt"]
