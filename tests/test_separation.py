"""The CUDA path and the oracle share nothing: no source of the product package (the binding, its build step,
the CUDA sources and the C ABI header) names the oracle or includes, imports or links a file of it, and the
oracle includes nothing of the product.  Only the seeded input generators (synth/) serve both sides."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sources(*patterns):
    out = []
    for p in patterns:
        out += glob.glob(os.path.join(ROOT, p), recursive=True)
    return [f for f in out if "/_build/" not in f and "__pycache__" not in f]


def test_product_never_reaches_the_oracle():
    files = _sources("paper_2107_12330_b300/**/*.py", "paper_2107_12330_b300/csrc/*", "include/*.h")
    assert files
    for f in files:
        text = open(f, errors="replace").read()
        assert not re.search(r"\boracle\b", text, re.I), f"{f} names the oracle"


def test_oracle_includes_nothing_of_the_product():
    files = _sources("oracle/*.c", "oracle/*.py")
    assert files
    for f in files:
        text = open(f, errors="replace").read()
        assert "paper_2107_12330_b300" not in text, f
        assert "tripoll.h" not in text and "common.cuh" not in text, f
        for inc in re.findall(r'#include\s+"([^"]+)"', text):
            assert not inc.startswith(("../", "paper_", "include/")), (f, inc)


def _code_only(path, text):
    """The text without comments and string literals (docstrings included)."""
    if path.endswith(".py"):
        import io
        import tokenize
        keep = [t.string for t in tokenize.generate_tokens(io.StringIO(text).readline)
                if t.type not in (tokenize.COMMENT, tokenize.STRING)]
        return " ".join(keep)
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return re.sub(r'"(?:\\.|[^"\\])*"', " ", text)


def test_input_generators_hold_no_survey_arithmetic():
    """synth/ draws inputs only (it names the survey kinds of each workload, nothing more): it neither
    builds G+ nor counts triangles."""
    files = _sources("synth/*.py", "synth/*.c")
    assert files
    for f in files:
        code = _code_only(f, open(f, errors="replace").read())
        assert not re.search(r"triangle|wedge|ceil_log2|time_bin|sort3|intersect|orient|dedup", code, re.I), f
