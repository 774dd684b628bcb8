"""Host-side checks of the GPU library that need no GPU: it builds, loads,
exports every entry point the header declares, rejects bad parameters
before touching a device, and keeps the oracle out of the product path."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2410_06657_gb300 import lbm, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    L = lbm.load()
    declared = header_functions()
    assert declared, "no declarations found"
    assert sorted(lbm.EXPORTS) == declared
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lbm_\w+)", out))
    for name in declared:
        assert name in exported, name
        assert hasattr(L, name)


def test_struct_layouts_match_the_header():
    # lbm_params: 4 int32 then 25 doubles; lbm_obs: 17 eight-byte slots
    assert C.sizeof(lbm.Params) == 4 * 4 + 25 * 8
    assert C.sizeof(lbm.Obs) == 17 * 8
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    for struct, cls in (("lbm_params", lbm.Params), ("lbm_obs", lbm.Obs)):
        body = src[src.index("typedef struct " + struct):src.index("} " + struct + ";")]
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = re.findall(r"\b(?:int32_t|int64_t|double)\s+([^;]+);", body)
        fields = [n.strip() for group in names for n in group.split(",")]
        assert fields == [f for f, _ in cls._fields_], struct


@pytest.mark.parametrize("bad", [dict(nx=0), dict(ny=-3), dict(k_e=0), dict(precision=7),
                                 dict(theta_deg=180.0), dict(theta_deg=0.0), dict(M=0.0),
                                 dict(mu_l=-1.0), dict(Ste=0.0), dict(sigma_g=0.0),
                                 dict(T_w=1.0), dict(W=float("nan")), dict(alpha_sl=0.0),
                                 dict(nx=16384, ny=16384)])
def test_create_rejects_bad_parameters_without_a_device(bad):
    L = lbm.load()
    p = lbm.make_params(W.params(**bad))
    h = C.c_void_p()
    rc = L.lbm_create(C.byref(p), None, C.byref(h))
    assert rc == lbm.ERR_BADPARAM
    assert not h.value
    assert L.lbm_last_error()


def test_calls_on_null_handles_fail_cleanly():
    L = lbm.load()
    assert L.lbm_step(None, 1) == lbm.ERR_BADPARAM
    assert L.lbm_init_droplet(None, 5.0, 1.0, 1.0, 0) == lbm.ERR_BADPARAM
    assert L.lbm_observables(None, None) == lbm.ERR_BADPARAM
    assert L.lbm_observables_to_host(None, None) == lbm.ERR_BADPARAM
    assert L.lbm_sync(None) == lbm.ERR_BADPARAM
    assert L.lbm_observables_deferred(None, None) == lbm.ERR_BADPARAM
    assert L.lbm_presolve(None, 1e-10, 10, None, None) == lbm.ERR_BADPARAM
    assert L.lbm_batch_create(None, 0, None, 0, None) == lbm.ERR_BADPARAM
    L.lbm_destroy(None)


def test_product_path_never_uses_the_oracle():
    pkg = os.path.join(ROOT, "paper_2410_06657_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, re.M), f
                assert "lbm_oracle" not in text, f


def test_philox_matches_published_known_answers(tmp_path):
    """The stochastic rounding of half storage draws its bits from
    Philox4x32-10; the library's own header, compiled for the host, must
    reproduce the generator's published known-answer vectors, and the 13-bit
    fields must tile the 128-bit block in order."""
    import json
    kat = json.load(open(os.path.join(ROOT, "tests", "golden", "philox4x32_10_kat.json")))["vectors"]
    src = tmp_path / "kat.cpp"
    src.write_text(
        '#include <cstdio>\n#include <cstdlib>\n#include "philox.h"\n'
        "int main(int argc, char **argv) {\n"
        "  uint32_t c[4]; for (int i = 0; i < 4; i++) c[i] = (uint32_t)strtoul(argv[1 + i], 0, 16);\n"
        "  uint32_t k0 = (uint32_t)strtoul(argv[5], 0, 16), k1 = (uint32_t)strtoul(argv[6], 0, 16);\n"
        "  lbm::philox4x32_10(c, k0, k1);\n"
        '  printf("%08x %08x %08x %08x", c[0], c[1], c[2], c[3]);\n'
        "  for (int j = 0; j < 9; j++) printf(\" %u\", lbm::bits13(c, j));\n"
        "  return 0;\n}\n")
    exe = tmp_path / "kat"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2410_06657_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    for v in kat:
        out = subprocess.run([str(exe), *v["ctr"], *v["key"]], capture_output=True, text=True,
                             check=True).stdout.split()
        assert out[:4] == v["out"]
        words = [int(w, 16) for w in out[:4]]
        block = sum(w << (32 * i) for i, w in enumerate(words))
        assert [int(b) for b in out[4:]] == [(block >> (13 * j)) & 0x1fff for j in range(9)]


@pytest.mark.parametrize("prec,pop_off,aux_off,out_off", [
    (W.FP64, 4, 0, 0), (W.FP64, 0, 4, 0), (W.FP32, 2, 0, 0), (W.FP16S, 0, 2, 0), (W.FP32, 0, 0, 4)])
def test_noalloc_rejects_misaligned_pointers_without_a_device(prec, pop_off, aux_off, out_off):
    """The allocation-free observables read every plane element by element:
    a caller pointer that is not aligned to its element size is refused
    with LBM_ERR_BADPARAM before any device work (no GPU needed here)."""
    L = lbm.load()
    L.lbm_observables_noalloc.argtypes = [C.POINTER(lbm.Params), C.c_void_p, C.c_void_p, C.c_int32,
                                          C.c_int64, C.c_void_p, C.c_void_p]
    p = lbm.make_params(W.params(nx=64, ny=32, precision=prec))
    base = 1 << 20      # never dereferenced: the call must stop at the check
    rc = L.lbm_observables_noalloc(C.byref(p), C.c_void_p(base + pop_off), C.c_void_p(base + aux_off), 64, 0,
                                   C.c_void_p(base + out_off), None)
    assert rc == lbm.ERR_BADPARAM
    assert b"aligned" in L.lbm_last_error()


@pytest.mark.parametrize("v_off,r_off,out_off,n", [(2, 0, 0, 8), (0, 2, 0, 8), (0, 0, 1, 8), (0, 0, 0, -1)])
def test_half_rounding_entry_rejects_bad_arguments_without_a_device(v_off, r_off, out_off, n):
    """The half-rounding check entry refuses misaligned pointers and a
    negative count with LBM_ERR_BADPARAM before any device work; a count of
    zero enqueues nothing and succeeds."""
    L = lbm.load()
    base = 1 << 20      # never dereferenced
    rc = L.lbm_round_half_sr(C.c_void_p(base + v_off), C.c_void_p(base + r_off), C.c_void_p(base + out_off), n,
                             None)
    assert rc == lbm.ERR_BADPARAM
    assert L.lbm_round_half_sr(None, None, None, 0, None) == lbm.OK
