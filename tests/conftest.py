import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libgsp")
    config.addinivalue_line("markers", "slow: full-size parity cases (minutes of oracle time)")


def build_gsp() -> str:
    """Build libgsp.so and the bounds-checked libgsp_debug.so (load the build
    script by path: the package needs the library); returns libgsp.so's path."""
    import importlib.util
    path = os.path.join(ROOT, "paper_2603_08661_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("_gsp_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build(debug=True)


# Gradient parity (CUDA adjoint against the oracle's analytic adjoint), per
# entry: |gpu - oracle| <= GRAD_TOL * max(|oracle|, GRAD_FLOOR * RMS) +
# GRAD_ROUND * u * A, with u = 2^-24 and A the oracle's magnitude adjoint of
# that entry (the sum of the absolute values of the terms the adjoint adds up).
# The first part is the stated 1e-4 relative tolerance with a floor of 1e-3 x
# the RMS of the parameter group.  The second is the rounding bound of an
# FP32 evaluation: where an entry is a sum whose terms cancel (A >> |entry|),
# terms computed in FP32 with relative errors of a few u, summed in FP32 over
# the n tiles and views a Gaussian covers (about sqrt(n) u A for that sum),
# move it by tens of u A whatever the implementation.  Measured beyond the
# relative part: at most 0.82 u A on 32x32-pixel regions of 1M and 3M-Gaussian
# scenes (8 views), 17 u A on whole-view L1 gradients summed over 8 views;
# GRAD_ROUND = 64 keeps a margin of almost 4 over the largest.
U32 = 2.0 ** -24
GRAD_TOL, GRAD_FLOOR, GRAD_ROUND = 1e-4, 1e-3, 64.0


def grad_bound(b, mag, rms):
    """Allowed |gpu - oracle| per entry (see above); b and mag shaped alike."""
    return GRAD_TOL * np.maximum(np.abs(b), GRAD_FLOOR * rms) + GRAD_ROUND * U32 * mag


def assert_grads_match(name, a, b, mag, rms=None):
    """Every entry of a (CUDA) within grad_bound of b (oracle), elementwise.
    mag: the oracle's magnitude adjoint; rms: the group RMS (default: of b).
    Returns the largest error / bound ratio."""
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    mag = np.asarray(mag, dtype=np.float64).reshape(-1)
    if b.size == 0:
        return 0.0
    if rms is None:
        rms = float(np.sqrt(np.mean(b ** 2)))
    err = np.abs(a - b)
    ratio = err / np.maximum(grad_bound(b, mag, rms), 1e-300)
    w = int(np.argmax(ratio))
    assert ratio[w] <= 1.0, (name, int((ratio > 1).sum()), b.size, float(ratio[w]), float(err[w]), float(b[w]),
                             float(mag[w]), rms)
    return float(ratio[w])


# Gate exemption (rendering): a pixel whose oracle evaluation meets a gate
# (alpha = 1/255, or T (1 - alpha) = 1e-4) within GATE_REL relative may take
# that decision differently in FP32: alpha carries about (4 |power| + 3) u of
# rounding from the FP32 conic, pixel offset and exponential (|power| <= ln 255
# at the 1/255 gate), 25 u = 1.5e-6.  Such pixels, and the Gaussians whose
# results a flip there would move, are exempt; their number must stay below
# EXEMPT_FRAC of the pixels compared.
GATE_REL = 2e-6
EXEMPT_FRAC = 1e-4


@pytest.fixture(scope="session")
def gsp_lib():
    """The CUDA library binding; GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_gsp()
    import paper_2603_08661_gb300 as gsp
    return gsp
