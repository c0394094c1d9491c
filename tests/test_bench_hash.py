"""bench.py's fused-kernel source hash leaves comments and blank lines out (a change of comments
alone keeps a DRAM-traffic capture valid) and keeps everything else, string literals whole."""

import bench

def test_strip_c_comments_keeps_code_and_strings():
    src = ('int a = 1; // trailing\n'
           '/* block\n   comment */ int b = 2;\n'
           '\n'
           'const char* s = "not // a comment /* either */";\n'
           "char c = '/';  // slash\n"
           'asm volatile("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));\n')
    out = bench.strip_c_comments(src)
    assert out == ('int a = 1;\n'
                   ' int b = 2;\n'
                   'const char* s = "not // a comment /* either */";\n'
                   "char c = '/';\n"
                   'asm volatile("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));')

def test_comment_only_change_keeps_the_hash_and_code_change_does_not():
    a = "x = y + 1; // add one\nreturn x;\n"
    b = "// a new note\nx = y + 1;   // added one\n\nreturn x;\n"
    c = "x = y + 2; // add one\nreturn x;\n"
    assert bench.strip_c_comments(a) == bench.strip_c_comments(b)
    assert bench.strip_c_comments(a) != bench.strip_c_comments(c)
