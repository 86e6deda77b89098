"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/bonsai.h (no GPU needed; no compute calls)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bonsai.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bonsai_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1204_2280_gb300 import builder
    return builder.build()


def test_header_and_binding_agree():
    import paper_1204_2280_gb300 as B
    assert declared() == sorted(B.EXPORTS)


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    syms = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [s for s in declared() if s not in syms]
    assert not missing, missing
    L = C.CDLL(libpath)
    for s in declared():
        assert hasattr(L, s)


def test_invalid_arguments_rejected_without_gpu(libpath):
    import paper_1204_2280_gb300 as B
    L = B.lib()
    assert L.bonsai_create(None, None, None) == -1
    ctx = C.c_void_p()
    bad = B.Config(ncrit=65)
    assert L.bonsai_create(C.byref(ctx), C.byref(bad), None) == -1
    assert b"ncrit" in L.bonsai_last_error(None)
    assert L.bonsai_build(None) == -1
    assert B.bonsai_version().startswith("bonsai-gb300")
    neg = B.Config(arena_limit_mib=-1)
    assert L.bonsai_create(C.byref(ctx), C.byref(neg), None) == -1
    assert b"arena_limit_mib" in L.bonsai_last_error(None)


def test_config_layout_matches_header(tmp_path):
    """The binding's bonsai_config has the C struct's size and field offsets
    (a probe compiled against include/bonsai.h by the host compiler)."""
    import paper_1204_2280_gb300 as B
    fields = [f[0] for f in B.Config._fields_]
    probe = tmp_path / "probe.c"
    probe.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "bonsai.h"\nint main(void) {\n'
        '  printf("%zu\\n", sizeof(bonsai_config));\n'
        + "".join(f'  printf("%zu\\n", offsetof(bonsai_config, {f}));\n' for f in fields)
        + "  return 0;\n}\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(probe), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[0] == C.sizeof(B.Config)
    assert got[1:] == [getattr(B.Config, f).offset for f in fields]


def test_create_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1204_2280_gb300 as B
    ctx = C.c_void_p()
    rc = B.lib().bonsai_create(C.byref(ctx), None, None)
    assert rc == -3 and not ctx.value


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the built library every entry point raises."""
    import paper_1204_2280_gb300 as B
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "libbonsai.so"))
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        B.lib()
    with pytest.raises(RuntimeError):
        B.Bonsai(B.Config())


def test_static_sort_binding_checks_before_any_launch():
    """bonsai_sort_keys_static's binding rejects wrong dtypes, short outputs,
    non-contiguous and non-CUDA tensors before it calls the library (the C
    side gets raw pointers and cannot check them)."""
    import torch
    import paper_1204_2280_gb300 as B
    n = 100
    k = torch.zeros(n, dtype=torch.int64)
    with pytest.raises(TypeError, match="perm must be torch.int32"):
        B.bonsai_sort_keys_static(k, k.clone(), torch.zeros(n, dtype=torch.int64))
    with pytest.raises(TypeError, match="sorted_keys must be torch.int64"):
        B.bonsai_sort_keys_static(k, torch.zeros(n, dtype=torch.int32), torch.zeros(n, dtype=torch.int32))
    with pytest.raises(ValueError, match="sorted_keys holds 99 elements, needs 100"):
        B.bonsai_sort_keys_static(k, k[:99].clone(), torch.zeros(n, dtype=torch.int32))
    with pytest.raises(ValueError, match="perm holds 50 elements"):
        B.bonsai_sort_keys_static(k, k.clone(), torch.zeros(50, dtype=torch.int32))
    with pytest.raises(ValueError, match="contiguous"):
        B.bonsai_sort_keys_static(k, torch.zeros(2 * n, dtype=torch.int64)[::2], torch.zeros(n, dtype=torch.int32))
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        B.bonsai_sort_keys_static(k, k.clone(), torch.zeros(n, dtype=torch.int32))


def test_bench_fma_and_hold_tile_reject_bad_arguments(libpath):
    import paper_1204_2280_gb300 as B
    L = B.lib()
    ms, fl = C.c_float(), C.c_double()
    assert L.bonsai_bench_fma(0, 256, 10, C.byref(ms), C.byref(fl)) == -1
    assert L.bonsai_bench_fma(4, 100, 10, C.byref(ms), C.byref(fl)) == -1
    assert b"bonsai_bench_fma" in L.bonsai_last_error(None)
    assert L.bonsai_debug_hold_sort_tile(None, 3) == -1
