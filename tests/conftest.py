import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libtaser")


def pytest_sessionfinish(session, exitstatus):
    """Under TASER_LIBRARY=debug (the bounds-checked libtaser_debug.so): read its counters
    once the tests have run.  Any failed index check fails the session; TASER_DEBUG_REPORT,
    if set, names a JSON file that receives the counters."""
    if os.environ.get("TASER_LIBRARY") != "debug":
        return
    import json
    from paper_1609_01797_gb300 import _native
    if _native._lib is None:   # no test loaded the library
        return
    import torch
    if not torch.cuda.is_available():
        return
    from paper_1609_01797_gb300.api import debug_report
    rep = debug_report()
    path = os.environ.get("TASER_DEBUG_REPORT")
    if path:
        with open(path, "w") as f:
            json.dump(rep, f)
    if rep["fails"]:
        print("\nbounds-checked build: %d failed index checks, first %s" % (rep["fails"], rep["first"]))
        session.exitstatus = 1
