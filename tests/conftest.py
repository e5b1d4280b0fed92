import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running case (full-size workloads)")


def _gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _gpu_available():
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as o
    o.build()
    return o


def read_golden_cases(path):
    cases, tables = [], {}
    cur = None
    with open(path) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "case":
                cases.append((parts[1].encode(), parts[2].encode(), int(parts[3]), parts[4].encode()))
            elif parts[0] == "table":
                cur = (parts[1].encode(), parts[2].encode())
                tables[cur] = {"c": [], "b": []}
            elif parts[0] == "c":
                tables[cur]["c"].append([int(v) for v in parts[1:]])
            elif parts[0] == "b":
                tables[cur]["b"].append(parts[1:])
            elif parts[0] == "end":
                cur = None
    return cases, tables
