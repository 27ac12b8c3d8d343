"""Every entry point declared in include/hydro.h carries a comment that cites the paper's passage
it serves (a section, table or figure) or says that it has no counterpart in the paper; a
declaration that directly follows another shares that one's comment."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_entry_point_cites_its_passage():
    with open(os.path.join(ROOT, "include", "hydro.h")) as f:
        text = f.read()
    # blank out comments but remember where each one ends
    comments = [(m.start(), m.end(), " ".join(m.group(0).replace("*", " ").split()))
                for m in re.finditer(r"/\*.*?\*/", text, re.S)]
    decls = [(m.start(), m.group(1)) for m in re.finditer(r"^\s*(?:int|void|const char\s*\*)\s+(hydro_\w+)\s*\(",
                                                              text, re.M)]
    assert len(decls) >= 30
    missing = []
    for pos, name in decls:
        before = [c for c in comments if c[1] <= pos]
        assert before, name
        doc = before[-1][2]
        ok = any(t in doc for t in ("Sec.", "Table", "Fig.", "no counterpart", "the paper has no"))
        if not ok:
            missing.append(name)
    assert not missing, missing
