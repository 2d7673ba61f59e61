"""Host-side logic of bench.py that needs no GPU: the fingerprint that ties the
reported DRAM traffic to one ncu capture of the kernel code."""
import importlib.util
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(HERE, "..", "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_code_only_ignores_comments_and_layout():
    b = _bench()
    src = 'int f(int a) { // add one\n  return a + 1; /* done */ }\nconst char* s = "// not a comment";\n'
    same = 'int f(int a)   {\n\n  return a + 1;   }\n// other words\nconst char* s = "// not a comment";'
    assert b._code_only(src) == b._code_only(same)
    # a code change, or a change inside a string literal, changes the code
    assert b._code_only(src) != b._code_only(src.replace("a + 1", "a + 2"))
    assert b._code_only(src) != b._code_only(src.replace('"// not a comment"', '"// not a Comment"'))


def test_fingerprint_covers_the_kernel_sources():
    b = _bench()
    fp = b.sources_fingerprint()
    assert len(fp) == 64 and int(fp, 16) >= 0
    assert fp == b.sources_fingerprint()  # deterministic
