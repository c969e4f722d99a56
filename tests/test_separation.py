"""The CUDA path and the oracle share no code: the product package never imports the
oracle, the oracle never imports the product, and the seeded input generators (synth)
import neither (CPU only, a static check of the sources)."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(folder):
    for dirpath, _, files in os.walk(os.path.join(ROOT, folder)):
        for f in files:
            if f.endswith(".py"):
                path = os.path.join(dirpath, f)
                tree = ast.parse(open(path, encoding="utf-8").read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        for a in node.names:
                            yield path, a.name
                    elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
                        yield path, node.module


def test_product_does_not_import_the_oracle():
    bad = [(p, m) for p, m in _imports("paper_2605_26347_gb300") if m.split(".")[0] in ("oracle", "synth")]
    assert not bad, bad
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2605_26347_gb300", "csrc")):
        for f in files:
            assert "oracle" not in open(os.path.join(dirpath, f), encoding="utf-8").read(), f


def test_oracle_and_inputs_do_not_import_the_product():
    for folder in ("oracle", "synth"):
        bad = [(p, m) for p, m in _imports(folder) if m.split(".")[0] == "paper_2605_26347_gb300"]
        assert not bad, bad
    assert not [(p, m) for p, m in _imports("synth") if m.split(".")[0] == "oracle"]
