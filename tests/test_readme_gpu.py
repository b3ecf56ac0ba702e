"""The Python example in README.md runs as written and gives sane results."""
import os
import re

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_python_example_runs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_1658_gb300 import build
    build.build()
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert blocks, "no python example in README.md"
    env = {}
    cwd = os.getcwd()
    os.chdir(ROOT)
    try:
        exec(compile(blocks[0], "README.md", "exec"), env)
    finally:
        os.chdir(cwd)
    P, Pg, Pf, q, maxP = env["P"], env["Pg"], env["Pf"], env["q"], env["maxP"]
    k = int(np.argmax(P))
    f_peak = env["f0"] + k * env["df"]
    assert abs(f_peak - 0.37) < 2 * env["df"]
    assert int(np.argmax(Pg)) == k and abs(int(np.argmax(Pf)) - k) <= 1
    assert q.shape == (1, 9) and np.all(np.diff(q[0]) > 0)
    assert maxP.shape == (1000,) and np.all(maxP > 0)
    # the quantiles of the largest noise peak bracket the Monte-Carlo maxima
    assert q[0, 0] < np.median(maxP) < q[0, -1]
