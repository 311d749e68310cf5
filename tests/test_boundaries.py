"""Static checks of the code boundaries: the product (the package and its CUDA sources) never
imports, links or runs the oracle, and the oracle never touches the product."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def sources(top, exts):
    for d, _, files in os.walk(os.path.join(ROOT, top)):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_product_does_not_use_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)|liboracle|rb_oracle", re.M)
    for path in sources("paper_1807_11866_gb300", (".py", ".cu", ".cuh", ".h", ".c")):
        assert not pat.search(open(path).read()), path
    for path in sources("include", (".h",)):
        assert not pat.search(open(path).read()), path


def test_oracle_does_not_use_the_product():
    pat = re.compile(r"paper_1807_11866_gb300|librb|#include\s+\"rb", re.M)
    for path in sources("oracle", (".py", ".c", ".h")):
        assert not pat.search(open(path).read()), path


def test_inputs_module_is_shared_and_independent():
    """synth/ serves both sides and imports neither."""
    pat = re.compile(r"^\s*(import|from)\s+(oracle|paper_1807_11866_gb300)\b", re.M)
    for path in sources("synth", (".py",)):
        assert not pat.search(open(path).read()), path
