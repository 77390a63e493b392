import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def tiny_workload():
    """64^3 float32 blob volume, K=2 z-slabs, 128x128, step 0.5, N_S=8 (the tiny configuration)."""
    import numpy as np

    import oracle
    import synth

    dims = (64, 64, 64)
    vol = synth.volume(dims, 16, 3, synth.SEED_VOLUME + 0, np.float32)
    lut = synth.transfer_function(synth.SEED_TF)
    cams = synth.orbit(dims, 16, 128, 128, synth.SEED_ORBIT)
    boxes = oracle.split_boxes(dims, (1, 1, 2))
    return dict(dims=dims, vol=vol, lut=lut, cams=cams, boxes=boxes, step=0.5, ref_len=1.0, n_s=8, gamma=0.02)
