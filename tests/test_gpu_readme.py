"""The Python quick start of README.md runs as written (the documentation stays true to the API)."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_quick_start_runs(tg):
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert len(blocks) == 1
    ns = {}
    exec(compile(blocks[0], "README.md", "exec"), ns)
    assert ns["iou"] > 0.95, ns["iou"]
    assert ns["n"] > 0 and ns["tris"].shape == (ns["n"], 3, 3)
    assert not ns["grad"].any()                      # Adam zeroed it
