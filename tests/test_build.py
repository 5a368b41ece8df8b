"""The kernel-source fingerprint that ties a recorded DRAM-traffic figure to
the code it was measured on: comments do not count, code does."""

from paper_2605_25040_gb300 import build as B


def test_strip_comments_keeps_code_and_literals():
    src = (b'int a = 1; // one\n'
           b'/* block\n comment */ int b = 2;\n'
           b'const char* s = "not // a comment";\n'
           b"char c = '/'; char d = '\\'';\n"
           b'asm("mov.u32 %0, 1; /* kept */" : "=r"(a));\n')
    out = B.strip_comments(src)
    assert b'one' not in out and b'block' not in out
    assert b'int a = 1; \n' in out and b' int b = 2;' in out
    assert b'"not // a comment"' in out
    assert b"'/'" in out and b"'\\''" in out
    assert b'"mov.u32 %0, 1; /* kept */"' in out


def test_hash_ignores_comments_only():
    base = {"x.cu": b"__global__ void k() { int i = 0; }\n"}
    commented = {"x.cu": b"// header\n__global__ void k() { /* zero */ int i = 0; }\n"}
    reworded = {"x.cu": b"// another header\n__global__ void k() { /* still zero */ int i = 0; }\n"}
    changed = {"x.cu": b"__global__ void k() { int i = 1; }\n"}
    B.KERNEL_SOURCES["_test_kernel"] = ["x.cu"]
    try:
        h0 = B.kernel_source_hash("_test_kernel", read=lambda rel: base[rel])
        h1 = B.kernel_source_hash("_test_kernel", read=lambda rel: commented[rel])
        h2 = B.kernel_source_hash("_test_kernel", read=lambda rel: changed[rel])
        h3 = B.kernel_source_hash("_test_kernel", read=lambda rel: reworded[rel])
    finally:
        del B.KERNEL_SOURCES["_test_kernel"]
    assert h0 != h2
    # "//" and "/* */" leave their line breaks and surrounding spaces; the
    # fingerprint compares the text that remains
    assert B.strip_comments(commented["x.cu"]).replace(b"\n", b"").replace(b" ", b"") == \
        base["x.cu"].replace(b"\n", b"").replace(b" ", b"")
    assert h1 != h2
    assert h1 == h3   # a comment reworded in place leaves the fingerprint
