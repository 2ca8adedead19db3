"""The Python usage example of README.md runs as written on a GPU."""
import os
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _example():
    lines = open(os.path.join(ROOT, "README.md")).read().splitlines()
    start = next(i for i, l in enumerate(lines) if l.startswith("Use from Python"))
    block, started = [], False
    for l in lines[start + 1:]:
        if l.startswith("    "):
            block.append(l)
            started = True
        elif started and l.strip():
            break
        elif started:
            block.append("")
    return textwrap.dedent("\n".join(block))


def test_readme_python_example_runs(lbmlib, cuda):
    code = _example()
    assert "lbm_step_gnn" in code and "lbm_step_bgk" in code
    exec(compile(code, "README.md", "exec"), {})
