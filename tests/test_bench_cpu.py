"""Host logic of the benchmark that needs no GPU: the digest that guards the profiled DRAM
traffic follows the kernels' code, not their comments or layout."""
import bench


def test_code_text_drops_comments_keeps_strings():
    src = 'int a = 1; // one\n/* block\n comment */ const char *s = "x // y /* z */";\n'
    assert bench.code_text(src) == 'int a = 1; const char *s = "x // y /* z */";'


def test_code_text_ignores_layout_only():
    a = "int f(int x) {\n  return x + 1;  // add\n}\n"
    b = "int f(int x) { return x + 1; }"
    c = "int f(int x) { return x + 2; }"
    assert bench.code_text(a) == bench.code_text(b) != bench.code_text(c)

