"""bench.py helpers that run without a GPU: the source digest that keys the
stored traffic record ignores comments and layout but not code."""
import bench


def test_code_tokens_drops_comments_keeps_literals():
    src = 'int a = 1; // note\n/* block\n comment */ char* s = "x // y /* z */"; char q = \'"\';\n\n  float b;'
    assert bench.code_tokens(src) == 'int a = 1; char* s = "x // y /* z */"; char q = \'"\'; float b;'
    assert bench.code_tokens('a = "esc \\" // still string"; // gone') == 'a = "esc \\" // still string";'


def test_comment_edits_keep_the_digest_code_edits_change_it():
    base = "__global__ void k(float* y) {\n    y[0] = 1.f;   // one\n}\n"
    reworded = "// a kernel\n__global__ void k(float* y) {\n    y[0] = 1.f;   /* the value one */\n}\n"
    changed = "__global__ void k(float* y) {\n    y[0] = 2.f;\n}\n"
    assert bench.code_tokens(base) == bench.code_tokens(reworded)
    assert bench.code_tokens(base) != bench.code_tokens(changed)
