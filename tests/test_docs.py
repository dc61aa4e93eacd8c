"""The repository paths that README.md cite exist: test files,
oracle and package sources, the header, profiles and golden fixtures."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PATH = re.compile(r"(?:tests|oracle|include|profiles|paper_1302_1125_gb300)/[\w./-]+?"
                  r"\.(?:cuh|cu|cpp|py|md|txt|c|h)\b")
CSRC = re.compile(r"\b(rlb_\w+\.(?:cuh|cu|cpp))\b")


@pytest.mark.parametrize("doc", ["DESIGN.md", "README.md"])
def test_cited_paths_exist(doc):
    text = open(os.path.join(ROOT, doc)).read()
    paths = set(PATH.findall(text))
    assert paths, doc
    missing = [p for p in sorted(paths) if not os.path.exists(os.path.join(ROOT, p))]
    assert not missing, missing
    csrc = os.path.join(ROOT, "paper_1302_1125_gb300", "csrc")
    missing = [f for f in sorted(set(CSRC.findall(text))) if not os.path.exists(os.path.join(csrc, f))]
    assert not missing, missing
