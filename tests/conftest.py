import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    # files named test_zz_* run after everything else
    items.sort(key=lambda it: 1 if os.path.basename(str(it.fspath)).startswith("test_zz_") else 0)


@pytest.fixture(autouse=True)
def _parity_test_id(request):
    from tests import _parity
    _parity.CURRENT["test"] = request.node.nodeid
    yield


def pytest_terminal_summary(terminalreporter):
    """Largest ratio of the GPU's deviation from the oracle to the oracle's
    own rounding spread, per test (what the parity margin must cover)."""
    try:
        from tests import _parity
    except ImportError:
        return
    if not _parity.RECORD:
        return
    per = {}
    for test, what, gov, allr in _parity.RECORD:
        g, a = per.get(test, (0.0, 0.0))
        per[test] = (max(g, gov), max(a, allr))
    tr = terminalreporter
    tr.write_sep("-", f"parity: deviation from the oracle / its own spread (margin {_parity.MARGIN:g}); "
                      f"deviation / 1e-10 where the plain bar holds")
    for test, (g, a) in sorted(per.items(), key=lambda kv: -kv[1][0]):
        tr.write_line(f"{g:10.3g} {a:10.3g}  {test}")
    gmax = max(g for g, _ in per.values())
    tr.write_line(f"largest ratio where the spread sets the bar: {gmax:.3g}")
    path = os.environ.get("PLSS_PARITY_LOG")
    if path:
        import json
        with open(path, "w") as f:
            json.dump({"margin": _parity.MARGIN, "max_ratio_spread_governed": gmax,
                       "per_test": {t: {"spread_governed": g, "floor": a} for t, (g, a) in per.items()}},
                      f, indent=1)
