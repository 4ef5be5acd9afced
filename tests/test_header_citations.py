"""Every entry point declared under include/ is documented where it is
declared: the comment nearest its declaration cites the passage of the paper
that defines the operation (a section, equation, table or remark), or says
that the paper has no counterpart (context management, measurement and the
forms outside the method)."""
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
CITE = re.compile(r"Sec\. |Eq\. |Eqs\. |Table |Tables |Remark |no counterpart|has no counterpart|The paper has no")


def declarations():
    for h in sorted((ROOT / "include").glob("*.h")):
        text = h.read_text()
        for m in re.finditer(r"^\s*(?:t7_status|const char \*)\s*(t7_\w+)\s*\(", text, re.M):
            before = text[:m.start()]
            end = before.rfind("*/")
            start = before.rfind("/*", 0, end)
            comment = re.sub(r"\s*\n\s*\*\s?", " ", before[start:end]) if 0 <= start < end else ""
            yield h.name, m.group(1), comment


def test_every_entry_point_cites_its_passage():
    decls = list(declarations())
    assert len(decls) >= 20
    uncited = [(h, name) for h, name, comment in decls if not CITE.search(comment)]
    assert not uncited, uncited
