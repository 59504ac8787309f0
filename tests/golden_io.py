"""Load the worked-example fixtures under tests/golden/ ("inf" -> +inf)."""
import json
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _conv(x):
    if isinstance(x, list):
        return [_conv(v) for v in x]
    if x == "inf":
        return math.inf
    return x


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        d = json.load(f)
    return {k: _conv(v) for k, v in d.items()}


def arr(x, dtype=np.float64):
    return np.asarray(x, dtype=dtype)
