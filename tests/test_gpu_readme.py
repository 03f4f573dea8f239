"""The usage example of README.md runs as written and gives the right
results: the inverse returns the input, and the learned path's output equals
the plain path's."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example(tmp_path, monkeypatch):
    import torch
    text = open(os.path.join(ROOT, "README.md")).read()
    code = re.search(r"```python\n(.*?)```", text, re.S).group(1)
    monkeypatch.chdir(tmp_path)  # the example writes its model file to the working directory
    env: dict = {}
    exec(compile(code, "README.md", "exec"), env)
    assert torch.equal(env["back"], env["d_in"])
    assert env["mtf"].numel() == env["chars"].numel()
    with env["Plan"](max_blocks=64, max_total_bytes=env["buf"].size, max_block_bytes=900_000,
                     flags=env["F_GRAPH"]) as plan:
        L_plain, p_plain = plan.forward(env["d_in"], env["off"])
    assert torch.equal(env["L"], L_plain) and torch.equal(env["primary"], p_plain)
