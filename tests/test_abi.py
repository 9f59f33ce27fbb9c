"""The C-ABI library: it builds, loads without a GPU, exports every symbol the
header declares, the binding's structs, enum values and argument counts match
the header as a C compiler reads it, and the host-only layout helper agrees
with the oracle."""
import re
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2007_14822_gb300 import build, tnh
    build.build()
    return tnh.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "tnh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tnh_[a-z_0-9]+)\s*\(", src)))


def test_exports_match_header(lib):
    from paper_2007_14822_gb300 import tnh
    out = subprocess.run(["nm", "-D", "--defined-only", tnh.LIB_PATH], capture_output=True, text=True).stdout
    exported = sorted(set(re.findall(r" T (tnh_[a-z_0-9]+)$", out, flags=re.M)))
    declared = header_functions()
    assert declared == exported
    assert sorted(tnh.SYMBOLS) == declared
    for name in declared:
        assert hasattr(lib, name)


def test_layout_matches_oracle(lib):
    from oracle.blocksparse import QNIndex, allowed_blocks
    from paper_2007_14822_gb300 import tnh
    rng = np.random.default_rng(3)
    for trial in range(5):
        inds = []
        for r in range(4):
            ns = int(rng.integers(1, 5))
            inds.append(tnh.Index([((int(q), int(q) % 3), int(rng.integers(1, 4))) for q in range(-ns // 2, ns - ns // 2)],
                                  +1 if rng.random() < 0.5 else -1))
        flux = (int(rng.integers(-1, 2)), int(rng.integers(0, 2)))
        blocks, offs, total = tnh.layout(inds, flux)
        want = allowed_blocks([QNIndex(i.sectors, i.arrow) for i in inds], flux)
        assert blocks == want
        sizes = [int(np.prod([inds[i].sectors[s][1] for i, s in enumerate(b)])) for b in blocks]
        assert offs == list(np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int)) if blocks else offs == []
        assert total == sum(sizes)


def test_layout_matches_oracle_repeated_charges(lib):
    # ranks 1..5, sectors with repeated charges (the layout completes the
    # last index from the flux rule; its sectors must come in increasing order)
    from oracle.blocksparse import QNIndex, allowed_blocks
    from paper_2007_14822_gb300 import tnh
    rng = np.random.default_rng(11)
    for trial in range(40):
        rank = int(rng.integers(1, 6))
        inds = []
        for r in range(rank):
            ns = int(rng.integers(1, 6))
            inds.append(tnh.Index([((int(rng.integers(-2, 3)),), int(rng.integers(1, 3))) for _ in range(ns)],
                                  +1 if rng.random() < 0.5 else -1))
        flux = (int(rng.integers(-2, 3)),)
        blocks, offs, total = tnh.layout(inds, flux)
        assert blocks == allowed_blocks([QNIndex(i.sectors, i.arrow) for i in inds], flux)
        sizes = [int(np.prod([inds[i].sectors[s][1] for i, s in enumerate(b)])) for b in blocks]
        assert total == sum(sizes)


def test_layout_paper_block_sparse_example(lib):
    # Sec. 9.2 example: blockdims ([2,2],[2,3]), nonzero blocks (1,2),(2,1)
    from paper_2007_14822_gb300 import tnh
    i1 = tnh.Index([((0,), 2), ((1,), 2)])
    i2 = tnh.Index([((0,), 2), ((1,), 3)])
    blocks, offs, total = tnh.layout([i1, i2], (1,))
    assert [tuple(k + 1 for k in b) for b in blocks] == [(1, 2), (2, 1)]
    assert total == 10


def test_layout_rejects_bad_index(lib):
    from paper_2007_14822_gb300 import tnh
    with pytest.raises(tnh.TnhError):
        tnh.layout([tnh.Index([((0,), 0)])], (0,))


# ------------------------------------------- struct layouts and enum values
STRUCTS = ["tnh_index", "tnh_tensor", "tnh_sweep_params", "tnh_sweep_stat", "tnh_dmrg_problem"]
ENUMS = ["TNH_OK", "TNH_ERR_ARG", "TNH_ERR_LABEL", "TNH_ERR_ARROW", "TNH_ERR_FLUX", "TNH_ERR_SHAPE",
         "TNH_ERR_OOM", "TNH_ERR_CUDA", "TNH_ERR_TIMEOUT", "TNH_ERR_NUMERIC", "TNH_ERR_NOT_CONVERGED",
         "TNH_FP64", "TNH_BF16x6", "TNH_BF16x3", "TNH_BF16"]


def c_layouts(tmp_path):
    """sizeof / offsetof of the header's structs and the enum values, as a
    plain C compiler lays them out from include/tnh.h."""
    from paper_2007_14822_gb300 import tnh
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "tnh.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'    printf("sizeof {s} %zu\\n", sizeof({s}));')
        for f, _ in getattr(tnh, s)._fields_:
            lines.append(f'    printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    for e in ENUMS:
        lines.append(f'    printf("enum {e} %d\\n", (int){e});')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out.splitlines()}


def test_binding_structs_and_enums_match_header(tmp_path):
    import ctypes
    from paper_2007_14822_gb300 import tnh
    want = c_layouts(tmp_path)
    for s in STRUCTS:
        cls = getattr(tnh, s)
        assert ctypes.sizeof(cls) == want[("sizeof", s)], s
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == want[(s, f)], (s, f)
    for e in ENUMS:
        if e.startswith("TNH_ERR") or e == "TNH_OK":
            assert tnh.STATUS[want[("enum", e)]] == e
        else:
            assert tnh.PRECISION[e[4:].lower()] == want[("enum", e)]


def test_binding_argument_counts_match_header(lib):
    from paper_2007_14822_gb300 import tnh
    src = open(os.path.join(ROOT, "include", "tnh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = dict(re.findall(r"\b(tnh_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", src))
    assert sorted(protos) == sorted(tnh.SYMBOLS)
    for name, params in protos.items():
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(getattr(lib, name).argtypes) == n, name


# ------------------------------------------------------- error statuses
_NULL_CALLS = r'''
import ctypes as C, json, sys
sys.path.insert(0, sys.argv[1])
from paper_2007_14822_gb300 import tnh
L = tnh.lib()
out = {}
for name in tnh.SYMBOLS:
    f = getattr(L, name)
    args = [0 if t in (C.c_int32, C.c_int, C.c_int64, C.c_uint64) else 0.0 if t is C.c_double else None
            for t in f.argtypes]
    if name == "tnh_debug_fail_alloc":
        args = [-1]      # 0 is valid (it disarms the injection)
    r = f(*args)
    msg = L.tnh_last_error(None)
    out[name] = [r if isinstance(r, int) or r is None else "text", (msg or b"").decode()]
print(json.dumps(out))
'''


def test_null_handles_give_a_status_not_a_crash(lib):
    # every entry point called with NULL handles and zero sizes returns
    # TNH_ERR_ARG with a message (the free functions return nothing), in a
    # child process so that a crash would fail the test, not the run
    import json
    import sys
    from paper_2007_14822_gb300 import tnh
    p = subprocess.run([sys.executable, "-c", _NULL_CALLS, ROOT], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    got = json.loads(p.stdout.strip().splitlines()[-1])
    assert sorted(got) == sorted(tnh.SYMBOLS)
    for name, (code, msg) in got.items():
        if name in ("tnh_destroy", "tnh_heff_free", "tnh_svd_free"):
            assert code is None, name
        elif name == "tnh_last_error":
            assert code in ("text", None), name
        else:
            assert code == 1, (name, code, msg)
            assert msg, name


def test_create_without_a_device_fails_with_cuda_status(lib):
    # nothing falls back to the CPU: with no usable GPU, tnh_create returns
    # TNH_ERR_CUDA and names the failing CUDA call
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.tnh_create(ctypes.byref(h), 0, None) == 7
    assert not h.value
    assert b"cudaGetDeviceCount" in lib.tnh_last_error(None)
