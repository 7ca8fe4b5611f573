"""The C-ABI library builds for sm_103a, loads, exports every symbol its
headers declare, and rejects malformed arguments on the host before any
device work (no GPU needed for these paths)."""
import ctypes as C
import math
import subprocess

import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W


def test_library_exports_every_declared_symbol():
    L = cz.lib()
    names = cz.exported_symbols()
    assert len(names) >= 17
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", cz._build.LIB], capture_output=True, text=True).stdout
    for n in names:
        assert f" T {n}" in out, n


def test_params_layout_and_defaults():
    p = cz.cosmica_params()
    cz.lib().cosmica_params_default(C.byref(p))
    assert p.struct_size == C.sizeof(cz.cosmica_params)
    assert p.version == cz.ABI_VERSION
    assert p.K0 == 11.5 and p.R_out_AU == 100.0 and p.max_steps == 100_000_000
    assert p.precision == cz.PREC_FP64 and p.polarity == 1


def _status(f, *a):
    return f(*a)


def test_invalid_arguments_are_rejected_on_the_host():
    L = cz.lib()
    h = C.c_void_p()
    assert L.cosmica_model_create(None, C.byref(h)) == cz.ERR_INVALID
    assert b"NULL" in L.cosmica_last_error()
    p = cz.make_params({})
    p.struct_size = 8
    assert L.cosmica_model_create(C.byref(p), C.byref(h)) == cz.ERR_INVALID
    assert b"struct_size" in L.cosmica_last_error()
    p = cz.make_params({"R_out": 0.5})
    assert L.cosmica_model_create(C.byref(p), C.byref(h)) == cz.ERR_INVALID
    p = cz.make_params({"polarity": 0})
    assert L.cosmica_model_create(C.byref(p), C.byref(h)) == cz.ERR_INVALID
    p = cz.make_params({}, precision=7)
    assert L.cosmica_model_create(C.byref(p), C.byref(h)) == cz.ERR_INVALID
    assert h.value is None
    # propagate / batch with NULL handles
    assert L.cosmica_propagate(None, None, None, 0, None, 1, None, None) == cz.ERR_INVALID
    assert L.cosmica_batch_create(None, 0, None, 0, C.byref(h)) == cz.ERR_INVALID
    assert L.cosmica_batch_run(None, None, 0, None, None, None, None) == cz.ERR_INVALID
    assert L.cosmica_batch_spectrum_hist(None, None, 0, None, None, None, None, None, None) == cz.ERR_INVALID
    assert b"batch is NULL" in L.cosmica_last_error()
    assert L.cosmica_debug_fn64(9, 0, None, None, None) == cz.ERR_INVALID
    assert L.cosmica_debug_normals32(1, 0, 4, 0, None, None, None) == cz.ERR_INVALID
    assert L.cosmica_debug_normals32(1, 0, 0, 0, None, None, None) == cz.OK   # n = 0: nothing to do


def test_invalid_model_extensions_are_rejected_on_the_host():
    """Validation of the radial shells, the squashed heliosphere, the energy form and the
    start point happens on the host, before any device work."""
    L = cz.lib()
    h = C.c_void_p()
    shells = W.shell_params(W.solar_cycle_series(), rotation=60)
    sq = W.params(R_ts=85.0, R_out=122.0, **W.SQUASHED)
    bad = [
        (dict(shells, n_shells=17.0), b"n_shells"),
        (dict(shells, shell_blend_AU=3.0), b"shell_blend"),
        (dict(shells, shell_K0=(0.0,) * 15), b"shell_K0"),
        (dict(shells, shell_tilt_deg=(95.0,) * 15), b"shell_tilt"),
        (dict(sq, squashed=2.0), b"squashed"),
        (dict(sq, hp_flank=-1.0), b"squashed"),
        (dict(sq, r0=125.0, th0=sq["nose_th"], ph0=sq["nose_ph"]), b"outside"),
        (W.params(formulation=2.0), b"formulation"),
        (W.params(th0=0.0), b"th0"),
        (W.params(ph0=math.nan), b"ph0"),
        (W.params(eps_adv=math.inf), b"eps_adv"),
        (W.params(dt_fixed=math.inf), b"dt_fixed"),
        (W.params(tilt_deg=math.nan), b"tilt"),
        (W.params(lat_fast_deg=math.inf), b"lat_fast"),
    ]
    for d, word in bad:
        p = cz.make_params(d)
        assert L.cosmica_model_create(C.byref(p), C.byref(h)) == cz.ERR_INVALID, d
        assert word in L.cosmica_last_error(), (word, L.cosmica_last_error())
        assert h.value is None
    # a start point toward the tail, inside the squashed boundary, passes validation
    # (creation then needs a GPU, so only the host check is exercised here)
    p = cz.make_params(dict(sq, r0=125.0, th0=math.pi - sq["nose_th"], ph0=(sq["nose_ph"] + math.pi) % (2 * math.pi)))
    st = L.cosmica_model_create(C.byref(p), C.byref(h))
    assert st != cz.ERR_INVALID or b"outside" not in L.cosmica_last_error()
    if h.value:
        L.cosmica_model_destroy(h)


def test_error_message_is_thread_local():
    import threading
    L = cz.lib()
    h = C.c_void_p()
    L.cosmica_model_create(None, C.byref(h))
    seen = {}

    def other():
        seen["msg"] = L.cosmica_last_error()

    t = threading.Thread(target=other)
    t.start(); t.join()
    assert seen["msg"] == b""
    assert L.cosmica_last_error() != b""


def test_oracle_and_library_share_no_code():
    """The oracle is C compiled by gcc; the library never includes or links it."""
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(root, "paper_2502_06319_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower(), f
    for f in ("cosmica.py", "_build.py", "__init__.py", "workloads.py"):
        txt = open(os.path.join(root, "paper_2502_06319_gb300", f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt, f


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding mirrors has the size and field offsets the C compiler gives
    the header's declaration (a plain C program compiled with gcc against include/)."""
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = {"cosmica_params": cz.cosmica_params, "cosmica_species": cz.cosmica_species,
               "cosmica_exit_states": cz.cosmica_exit_states, "cosmica_lis": cz.cosmica_lis,
               "cosmica_bins": cz.cosmica_bins, "cosmica_work_item": cz.cosmica_work_item,
               "cosmica_position": cz.cosmica_position, "cosmica_tuning": cz.cosmica_tuning,
               "cosmica_request": cz.cosmica_request, "cosmica_result": cz.cosmica_result,
               "cosmica_server_stats": cz.cosmica_server_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cosmica.h"', "int main(void) {"]
    for name, py in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(root, "include"), "-o", str(exe), str(src)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    for name, py in structs.items():
        assert got[(name, "size")] == C.sizeof(py), name
        for f, _ in py._fields_:
            assert got[(name, f)] == getattr(py, f).offset, (name, f)
