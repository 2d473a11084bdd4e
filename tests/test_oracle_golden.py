"""Printed-value pin: the block-Hankel size quoted in Sec. I.

The paper quotes 2116 x 54756 for four-coil 256x256 data with pencil 23.
With the oracle's Hankel convention (N - p + 1 window positions, p taps per
channel, channels concatenated), the 2D block analogue has p^2 * J taps and
(N - p + 1)^2 positions, which reproduces both printed numbers; a "full"
convolution convention (N + p - 1 positions) or N - p positions would not.
"""
import json
import os

import numpy as np

from oracle.hankel import hankel

HERE = os.path.dirname(os.path.abspath(__file__))


def test_block_hankel_size_from_sec_1():
    g = json.load(open(os.path.join(HERE, "golden", "block_hankel_size.json")))
    N, p, J = g["size"], g["pencil"], g["coils"]
    positions, taps = hankel(np.zeros(N, complex), p).shape
    assert taps * taps * J == g["rows"]
    assert positions * positions == g["cols"]
