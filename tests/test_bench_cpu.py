"""Host logic of bench.py that needs no GPU: the comment-insensitive kernel
code hash that decides whether the committed DRAM counters still apply."""
import bench


def test_strip_comments_keeps_code_and_literals():
    src = 'int a = 1; // gone\n/* gone\n too */ const char* s = "// kept /* kept */";\nchar c = \'/\';'
    assert bench.strip_comments(src) == 'inta=1;constchar*s="// kept /* kept */";charc=\'/\';'


def test_code_hash_ignores_comments_only(tmp_path):
    d = tmp_path / "a"
    d.mkdir()
    (d / "ks_market.cuh").write_text("// header\nint f() { return 1; }\n")
    h1 = bench.kernel_source_hash(str(d))
    (d / "ks_market.cuh").write_text("/* another header */\nint f() {\n  return 1;  // one\n}\n")
    assert bench.kernel_source_hash(str(d)) == h1
    (d / "ks_market.cuh").write_text("int f() { return 2; }\n")
    assert bench.kernel_source_hash(str(d)) != h1
