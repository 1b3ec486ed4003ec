import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def plate_small():
    from paper_1906_08125_gb300 import inputs
    return inputs.plate_mesh(nx=6, ny=6, nz=12, lx=30e-9, ly=30e-9, lz=60e-9, name="plate_small")


@pytest.fixture(scope="session")
def tip_small():
    from paper_1906_08125_gb300 import inputs
    return inputs.tip_mesh(radius=3e-9, height=12e-9, width=24e-9, box_height=40e-9,
                           h_fine=0.8e-9, lateral_growth=1.3, h_lat_max=3e-9, h_shank=2e-9,
                           h_top_max=4e-9, vertical_growth=1.3, name="tip_small")
