"""Readers for the hand-derived fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_raster_case(name="raster_closed_form.txt"):
    m, screen, pts, win = None, None, [], []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            t = line.split("#")[0].split()
            if not t:
                continue
            if t[0] == "matrix":
                m = np.array([float(v) for v in t[1:]], np.float32)
            elif t[0] == "screen":
                screen = (int(t[1]), int(t[2]), float(t[3]), float(t[4]))
            elif t[0] == "point":
                pts.append([float(v) for v in t[1:]])
            elif t[0] == "winner":
                win.append((int(t[1]), int(t[2]), int(t[3], 16), int(t[4])))
    return m, screen, np.array(pts, np.float32), win
