"""The design notes and README name files that exist (tests, profiles, sources)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _refs(text):
    pats = [r"`(tests/[A-Za-z0-9_./]+\.(?:py|txt))`", r"`(profiles/[A-Za-z0-9_.\-]+)`",
            r"`(csrc/[A-Za-z0-9_.]+)`", r"`(paper_1906_04051_gb300/[A-Za-z0-9_./]+\.py)`",
            r"`(include/[A-Za-z0-9_.]+\.h)`", r"`(oracle/[A-Za-z0-9_.]+)`"]
    out = set()
    for p in pats:
        out.update(re.findall(p, text))
    return out


def test_named_files_exist():
    missing = []
    for doc in ("DESIGN.md", "README.md"):
        text = open(os.path.join(ROOT, doc)).read()
        for ref in _refs(text):
            path = ref
            if ref.startswith("csrc/"):
                path = os.path.join("paper_1906_04051_gb300", ref)
            if not os.path.exists(os.path.join(ROOT, path)):
                missing.append((doc, ref))
    assert not missing, missing
