"""The Python usage example of README.md runs as printed."""
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def _example():
    text = open(os.path.join(ROOT, "README.md")).read()
    start = text.index("Use from Python")
    end = text.index("The C interface takes", start)
    lines = [ln[4:] for ln in text[start:end].splitlines() if ln.startswith("    ")]
    assert lines, "no indented example block"
    return "\n".join(lines)


def test_readme_python_example():
    ns = {}
    exec(compile(_example(), "README.md example", "exec"), ns)
    out, summary = ns["out"], ns["summary"]
    assert int((out["status"] == 0).sum()) == 0  # every pixel has a status
    disk = ns["reqs"][1]["out"]
    assert float(disk["g"].max()) > 0.0
    assert summary["p99_latency_s"] >= summary["p50_latency_s"] > 0.0
