import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: large-size case (minutes)")
    _plant_python_oracle_mistake()


def _plant_python_oracle_mistake():
    """For tests/test_oracle_mutants.py only: ORACLE_PY_MUTANT = "function|old|new"
    redefines that function of the oracle's Python part with one text
    replacement in its source, for this pytest process (the file is unchanged)."""
    spec = os.environ.get("ORACLE_PY_MUTANT")
    if not spec:
        return
    import inspect
    import textwrap

    import oracle
    fn, old, new = spec.split("|")
    src = textwrap.dedent(inspect.getsource(getattr(oracle, fn)))
    if old not in src:
        raise RuntimeError(f"planting site not found in oracle.{fn}")
    exec(compile(src.replace(old, new), f"<planted oracle.{fn}>", "exec"), oracle.__dict__)
