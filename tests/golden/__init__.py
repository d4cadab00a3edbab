"""Small text fixtures with their derivations (see each file's header)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    """Parse a fixture: 'key v1 v2 ...' lines, '#' comments, 'point x y z' rows."""
    out, pts = {}, []
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "point":
                pts.append([float(v) for v in vals])
            else:
                nums = [float(v) for v in vals]
                out[key] = nums[0] if len(nums) == 1 else np.array(nums)
    out["points"] = np.array(pts, dtype=np.float64)
    return out
