import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# measured errors of the parity tests against their bounds: name -> worst error
_PARITY = {}


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_collection_modifyitems(config, items):
    # tests marked gpu are skipped cleanly when no GPU is present
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def parity():
    """parity(name, err, tol) -> err <= tol, for the test to assert.

    Records the measured error beside its bound (the worst one per name); at
    the end of the session the records are written as JSON to the file that
    the environment variable SPH_PARITY_REPORT names, if it is set.  A
    bit-exact comparison records the number of mismatching elements with
    bound 0."""
    def record(name, err, tol):
        err, tol = float(err), float(tol)
        prev = _PARITY.get(name)
        if prev is None or not err <= prev["err"]:
            _PARITY[name] = {"err": err, "tol": tol}
        return err <= tol
    return record


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("SPH_PARITY_REPORT")
    if path and _PARITY:
        with open(path, "w") as f:
            json.dump(dict(sorted(_PARITY.items())), f, indent=1)
            f.write("\n")
