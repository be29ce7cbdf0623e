"""Reader for the hand-worked stream fixtures in tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}


def load(name):
    H = W = None
    attrs, frames = [], []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *rest = line.split()
            if key == "H":
                H = int(rest[0])
            elif key == "W":
                W = int(rest[0])
            elif key == "attr":
                attrs.append((int(rest[0]), int(rest[1])))
            elif key == "frame":
                frames.append({"in": [], "out": [], "mode": None, "bytes": b""})
            elif key == "in":
                a = len(frames[-1]["in"])
                frames[-1]["in"].append(np.array([int(x) for x in rest], dtype=_DT[attrs[a][0]]).reshape(H, W))
            elif key == "out":
                a = len(frames[-1]["out"])
                frames[-1]["out"].append(np.array([int(x) for x in rest], dtype=_DT[attrs[a][0]]).reshape(H, W))
            elif key == "mode":
                frames[-1]["mode"] = [int(x) for x in rest]
            elif key == "bytes":
                frames[-1]["bytes"] += bytes(int(x, 16) for x in rest)
    return H, W, attrs, frames


def options(name):
    """Stream options of a fixture: 'force <mode>' (default -1, trial) and
    'stages <bits>' (default 0; 1 = no zero mask, 2 = no delta, 4 = no
    ZigZag, the ablations of Sec. IV-H)."""
    opt = {"force_mode": -1, "stages": 0}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line.startswith("force "):
                opt["force_mode"] = int(line.split()[1])
            elif line.startswith("stages "):
                opt["stages"] = int(line.split()[1])
    return opt


def names():
    return sorted(n for n in os.listdir(GOLDEN) if n.startswith("stream_") and n.endswith(".txt"))
