"""Host logic of bench.py that needs no GPU: the hash tying the committed ncu
figures (profiles/traffic.json) to the kernel sources they were taken on."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_strip_comments_keeps_code_and_literals():
    b = _bench()
    src = ('int a = 1;  // note\n/* block\n comment */ asm("mov.u32 %0, %%smid; // not a comment" : "=r"(s));\n'
           "char q = '/'; char e = '\\''; const char* t = \"a /* b */ c\";")
    out = b.strip_comments(src)
    assert "note" not in out and "block" not in out
    assert 'asm("mov.u32 %0, %%smid; // not a comment" : "=r"(s));' in out
    assert "char q = '/';" in out and "char e = '\\'';" in out
    assert 'const char* t = "a /* b */ c";' in out


def test_hash_ignores_comments_and_layout_but_not_code():
    b = _bench()
    base = "double f(double x) {\n    return x * x;  // square\n}\n"
    same = "/* the square */\ndouble f(double x) { return x * x; }\n"
    other = "double f(double x) {\n    return x * x * x;\n}\n"
    assert b.strip_comments(base) == b.strip_comments(same)
    assert b.strip_comments(base) != b.strip_comments(other)

