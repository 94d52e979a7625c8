import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libmt.so")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def scenes_mod():
    from paper_2510_25660_gb300 import scenes
    return scenes


def pytest_terminal_summary(terminalreporter):
    """Divergent-path fractions of the per-contribution parity tests (GPU against
    the oracle on the same random numbers), one line per comparison."""
    mod = sys.modules.get("gpu_util")
    rows = getattr(mod, "PARITY", None) if mod is not None else None
    if not rows:
        return
    tr = terminalreporter
    tr.write_line("per-contribution parity: test | matched | divergent (fraction) | off > 1e-4 | bin mismatches")
    for test, nm, div, bad, bin_bad, worst in rows:
        frac = div / max(nm, 1)
        tr.write_line(f"  {test.split('::', 1)[-1]} | {nm} | {div} ({frac:.1e}) | {bad} | {bin_bad}")
