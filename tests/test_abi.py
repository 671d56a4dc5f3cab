"""The C-ABI library on the CPU: it loads, exports every symbol the header
declares, rejects bad input with the documented codes, and the emitter's
kernels compile with NVRTC for sm_103a (no GPU needed for either)."""
import ctypes
import os
import re

import pytest

from paper_2411_02640_gb300 import kx, synth
from tests import toys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "kx.h")).read()
    return sorted(set(re.findall(r"\b(kx_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = kx.lib()
    names = declared_symbols()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name


def test_status_strings():
    L = kx.lib()
    for s in range(11):
        assert L.kx_status_string(s)


def _load(path, **opts):
    o = kx.Options()
    for k, v in opts.items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    st = kx.lib().kx_load_mechanism(path.encode(), ctypes.byref(o), ctypes.byref(h))
    return st, h


def test_error_codes(tmp_path):
    assert _load(str(tmp_path / "missing.kxmech"))[0] == 1            # KX_ERR_IO
    bad = tmp_path / "bad.kxmech"
    bad.write_text("KXMECH 1\nspecies x\n")
    assert _load(str(bad))[0] == 2                                    # KX_ERR_PARSE
    m, path = toys.toy("unb", [toys.recomb("elementary")], str(tmp_path))
    text = open(path).read().replace("products 1 2 1", "products 1 0 1")
    unb = tmp_path / "unbalanced.kxmech"
    unb.write_text(text)
    assert _load(str(unb))[0] == 3                                    # KX_ERR_UNBALANCED
    assert _load(path, block=100)[0] == 4                             # KX_ERR_ARG
    assert b"multiple of 32" in kx.lib().kx_last_error()
    assert _load(path, kc_mode=7)[0] == 4
    assert _load(path, rates_negligible=2)[0] == 4


@pytest.mark.parametrize("name", ["h2o2_9_21"])
def test_emitted_kernels_compile_for_sm103a(name, tmp_path):
    path = synth.mechanism_file(name, str(tmp_path))
    m = kx.Mechanism(path, compile_only=1, cache_dir=str(tmp_path / "cache"))
    for k in ("wdot_fp64", "wdot_mixed", "rop_fp64", "rop_mixed", "thermo", "visc_fp64", "visc_mixed", "diff_fp64",
              "diff_mixed", "vjp", "vjp_wc", "wdot_fp64_wc", "wdot_fp64_noalloc"):
        info = m.kernel_info(k)
        assert 0 < info["registers"] <= 255, (k, info)
    # a compile-only handle refuses launches
    L = kx.lib()
    st = L.kx_production_rates(m.h, 1, 1, 1, 4, 1, 4, 0, None)
    assert st == 10                                                   # KX_ERR_UNSUPPORTED
    assert L.kx_production_rates(m.h, 1, 1, 1, 2, 1, 4, 0, None) == 4  # ld < n


def test_toy_mechanisms_compile(tmp_path):
    """Every reaction kind the file format has (three-body with a collider,
    Lindemann/Troe/SRI falloff, chemically activated, PLOG, irreversible)
    goes through the emitter and NVRTC."""
    from paper_2411_02640_gb300.synth import P_ATM, Reaction
    rx = [toys.recomb("elementary"), toys.recomb("three_body", efficiencies={3: 2.0}),
          toys.recomb("three_body", collider=3), toys.recomb("falloff", rate_low=(1e12, 0.1, 100.0)),
          toys.recomb("falloff", rate_low=(1e12, 0.1, 100.0), troe=(0.5, 100.0, 2000.0, 3000.0)),
          toys.recomb("falloff", rate_low=(1e12, 0.1, 100.0), sri=(0.5, 200.0, 1000.0, 1.2, 0.1)),
          toys.recomb("chem_act", rate_low=(1e12, 0.1, 100.0), troe=(0.5, 100.0, 2000.0, 3000.0)),
          Reaction(kind="plog", reversible=True, reactants=[(0, 1), (1, 1)], products=[(2, 1)], rate=(0, 0, 0),
                   plog=[(0.1 * P_ATM, 1e9, 0.2, 300.0), (10 * P_ATM, 1e11, -0.3, 900.0)]),
          Reaction(kind="elementary", reversible=False, reactants=[(2, 1)], products=[(0, 1), (1, 1)],
                   rate=(1e13, 0.0, 2e4))]
    _, path = toys.toy("allkinds", rx, str(tmp_path))
    m = kx.Mechanism(path, compile_only=1, cache_dir=str(tmp_path / "cache"))
    for k in ("wdot_fp64", "wdot_mixed", "rop_fp64", "rop_mixed"):
        assert m.kernel_info(k)["registers"] > 0


def test_transport_fit_keyword(tmp_path):
    """The file's transport_fit record: "direct" loads, anything but ln or
    direct is refused with KX_ERR_PARSE."""
    path = synth.mechanism_file("h2o2_9_21_direct", str(tmp_path))
    assert "transport_fit direct" in open(path).read()
    m = kx.Mechanism(path, compile_only=1, lazy=1, cache_dir=str(tmp_path / "c"))
    assert m.n_species == 9
    bad = tmp_path / "bad.kxmech"
    bad.write_text(open(path).read().replace("transport_fit direct", "transport_fit cubic"))
    with pytest.raises(kx.KxError) as e:
        kx.Mechanism(str(bad), compile_only=1, lazy=1, cache_dir=str(tmp_path / "c"))
    assert e.value.status == 2          # KX_ERR_PARSE


def test_host_side_argument_checks_of_the_status_and_no_alloc_calls(tmp_path):
    """kx_last_point_status and kx_production_rates_noalloc refuse a null
    handle or pointer and a handle that was only compiled (no device), before
    any CUDA call."""
    L = kx.lib()
    first = ctypes.c_int64(7)
    assert L.kx_last_point_status(None, None, ctypes.byref(first)) == 4            # KX_ERR_ARG
    _, path = toys.toy("st", [toys.recomb("elementary")], str(tmp_path))
    st, h = _load(path, compile_only=1, cache_dir=str(tmp_path / "c").encode())
    assert st == 0
    try:
        assert L.kx_last_point_status(h, None, None) == 4                             # null output
        assert L.kx_last_point_status(h, None, ctypes.byref(first)) == 10             # KX_ERR_UNSUPPORTED
        assert first.value == -1
        one = (ctypes.c_double * 8)()
        args = [h, one, one, one, ctypes.c_int64(1), one, ctypes.c_int64(1), None]
        assert L.kx_production_rates_noalloc(*args) == 10                             # compile-only handle
        args[6] = ctypes.c_int64(-1)
        assert L.kx_production_rates_noalloc(*args) == 4                              # negative count
        args[6] = ctypes.c_int64(0)
        assert L.kx_production_rates_noalloc(*args) == 0                              # n = 0: no-op
    finally:
        L.kx_free_mechanism(h)


def test_options_struct_matches_the_header():
    """The ctypes mirror of kx_options has the header's fields in the header's order and types
    (a field added on one side only would shift every later option)."""
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "kx.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} kx_options;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(const char\*|int)\s+(\w+);", body)
    want = [(n, ctypes.c_char_p if t == "const char*" else ctypes.c_int) for t, n in fields]
    assert [(n, t) for n, t in kx.Options._fields_] == want
