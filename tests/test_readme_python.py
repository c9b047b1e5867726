"""The README's Python example parses and names only what the package
provides (module attributes and Plan methods); running it needs a GPU."""
import ast
import os
import re

import pytest

pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_python_example_names_exist():
    readme = open(os.path.join(ROOT, "README.md")).read()
    code = re.search(r"```python\n(.*?)```", readme, flags=re.S).group(1)
    tree = ast.parse(code)
    used_mod, used_plan = set(), set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Attribute) and isinstance(node.value, ast.Name):
            if node.value.id == "wmg":
                used_mod.add(node.attr)
            elif node.value.id in ("plan", "plan2"):
                used_plan.add(node.attr)
    assert used_mod and used_plan
    for name in used_mod:
        assert hasattr(wmg, name), name
    for name in used_plan:
        assert callable(getattr(wmg.Plan, name, None)), name
