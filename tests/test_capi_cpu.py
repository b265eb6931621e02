"""The C-ABI library without a GPU: it loads, exports every function that
include/rdc.h declares, validates arguments, and its host-side rest-state
root equals the oracle's bit for bit.  No kernel is launched."""
from __future__ import annotations

import os
import re

import numpy as np
import pytest

from tests import oracle_pins as P

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "rdc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(rdc_\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(librdc):
    names = declared_functions()
    assert len(names) >= 20, names
    lib = librdc.lib()
    for n in names:
        assert hasattr(lib, n), f"librdc.so does not export {n}"
    from paper_1901_06535_gb300 import _capi
    assert set(names) <= set(_capi.exported_symbols()) | set(names)
    missing = set(names) - set(_capi.exported_symbols())
    assert not missing, f"binding lacks {missing}"


def test_params_default_is_table1(librdc):
    p = librdc.rdc_params_default()
    assert (p.eps, p.f, p.q, p.Du, p.dt, p.dx) == (P.EPS, P.F, P.Q, P.DU, P.DT, P.DX)
    assert p.precision == 0 and p.flags == 0 and p.k_block == 0 and p.round_seed == 0


@pytest.mark.parametrize("phi", [0.054, 0.0975, 0.2, 0.05, 0.08, 0.0301, 0.5])
def test_host_rest_state_bitwise_vs_oracle(librdc, orc, phi):
    assert librdc.rdc_rest_state(phi, P.F, P.Q) == orc.rest_state(phi)


def test_rest_state_rejects_no_root(librdc):
    with pytest.raises(librdc.RdcError):
        librdc.rdc_rest_state(0.001, P.F, P.Q)      # phi <= q (1 + f)
    with pytest.raises(librdc.RdcError):
        librdc.rdc_rest_state(0.054, 0.5, P.Q)      # f + q <= 1


@pytest.mark.parametrize("bad", [dict(eps=0.0), dict(q=-1.0), dict(dt=float("nan")),
                                 dict(Du=-0.1), dict(dx=0.0), dict(dt=0.05),
                                 dict(flags=3), dict(precision=7), dict(k_block=9),
                                 dict(round_seed=1), dict(f=0.5),
                                 dict(flags=4), dict(flags=4, precision=1), dict(flags=8),
                                 dict(flags=4 | 3, precision=2)])
def test_create_validates_params_before_touching_the_device(librdc, bad):
    p = librdc.rdc_params_default(**bad)
    with pytest.raises(librdc.RdcError) as e:
        librdc.rdc_create(16, 16, p)
    assert e.value.status == librdc.RDC_EINVAL


def test_create_validates_grid_and_phi(librdc):
    p = librdc.rdc_params_default()
    for W, H in ((0, 5), (5, 0), (-1, 3)):
        with pytest.raises(librdc.RdcError) as e:
            librdc.rdc_create(W, H, p)
        assert e.value.status == librdc.RDC_EINVAL
    for bad in (np.nan, 0.001, np.inf):
        phi = np.full((4, 4), 0.054, dtype=np.float32)
        phi[2, 1] = bad
        with pytest.raises(librdc.RdcError) as e:
            librdc.rdc_create(4, 4, p, phi)
        assert e.value.status == librdc.RDC_EINVAL


def test_status_strings(librdc):
    for code in range(8):
        assert librdc.rdc_status_str(code).startswith("RDC_")


@pytest.mark.parametrize("seg", [(0, 0, 10, 9.4), (3, 4, 20, 5), (0, 0, -1, 10), (5.5, 7.25, -30, -2),
                                 (100, 50, 60, 120), (1, 1, 1, 1)])
def test_host_snap_segment_bitwise_vs_oracle(librdc, orc, seg):
    assert librdc.rdc_snap_segment(*seg, 15.0) == orc.snap_segment(*seg, 15.0)


def test_missing_library_fails_loudly(librdc, monkeypatch, tmp_path):
    """Without the built library the binding raises; there is no fallback."""
    from paper_1901_06535_gb300 import _capi
    monkeypatch.setattr(_capi._build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_capi, "_LIB", None)
    with pytest.raises(RuntimeError, match="not built"):
        _capi.lib()


def test_create_ext_validates_before_touching_the_device(librdc):
    """Misaligned pointers, bad pitches and missing planes are refused with
    RDC_EINVAL before any device call (fake, never dereferenced addresses)."""
    p = librdc.rdc_params_default()
    base = 1 << 40
    good_u, good_v = [base, base + 4096], [base + 8192, base + 12288]
    phi = base + 16384
    cases = [
        dict(u=[base + 4, base + 4096], v=good_v, phi=phi, pitch=256),   # misaligned u
        dict(u=good_u, v=good_v, phi=phi + 8, pitch=256),                # misaligned phi
        dict(u=good_u, v=good_v, phi=phi, pitch=100),                    # pitch not 16-aligned
        dict(u=good_u, v=good_v, phi=phi, pitch=32),                     # pitch < W * 4
        dict(u=[0, base], v=good_v, phi=phi, pitch=256),                 # null plane
    ]
    for c in cases:
        with pytest.raises(librdc.RdcError) as e:
            librdc.rdc_create_ext(16, 4, p, c["u"], c["v"], c["phi"], c["pitch"])
        assert e.value.status == librdc.RDC_EINVAL


def test_check_division_validates_before_touching_the_device(librdc):
    """Bad q values and a NULL report are refused before any device call."""
    import ctypes
    L = librdc.lib()
    rep = librdc.rdc_division_report()
    for q in (0.0, -0.5, float("nan"), float("inf")):
        assert L.rdc_check_division(q, 0, 0, ctypes.byref(rep)) == librdc.RDC_EINVAL
    assert L.rdc_check_division(0.002, 0, 0, None) == librdc.RDC_EINVAL


def test_stochastic_rounding_params_pass_validation(librdc):
    """RDC_STOCH_ROUND with 16-bit storage and any seed is valid: without a
    GPU the call gets past validation and fails on the device instead."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("needs a machine without a GPU")
    for prec in (2, 3):
        for flags in (4, 4 | 1, 4 | 2):
            p = librdc.rdc_params_default(precision=prec, flags=flags, round_seed=0xDEADBEEF)
            with pytest.raises(librdc.RdcError) as e:
                librdc.rdc_create(16, 16, p)
            assert e.value.status != librdc.RDC_EINVAL


def test_stoch_round_sample_validates_before_touching_the_device(librdc):
    x = np.zeros(4, dtype=np.float32)
    for prec, row, col0 in ((0, 0, 0), (1, 0, 0), (2, -1, 0), (3, 0, -2)):
        with pytest.raises(librdc.RdcError) as e:
            librdc.rdc_stoch_round_sample(prec, 1, 5, row, col0, x)
        assert e.value.status == librdc.RDC_EINVAL


def test_philox_sample_validates_before_touching_the_device(librdc):
    import ctypes
    lib = librdc.lib()
    buf = (ctypes.c_uint32 * 8)()
    assert lib.rdc_philox_sample(-1, buf, buf, buf) == librdc.RDC_EINVAL
    assert lib.rdc_philox_sample((1 << 24) + 1, buf, buf, buf) == librdc.RDC_EINVAL
    assert lib.rdc_philox_sample(1, None, buf, buf) == librdc.RDC_EINVAL
    assert lib.rdc_philox_sample(1, buf, buf, None) == librdc.RDC_EINVAL
    assert lib.rdc_philox_sample(0, None, None, None) == librdc.RDC_OK


def test_stability_calls_validate_before_touching_the_device(librdc):
    import ctypes
    L = librdc.lib()
    rho = ctypes.c_double()
    assert L.rdc_batch_stability(None, 0, ctypes.byref(rho)) == librdc.RDC_EINVAL
    assert L.rdc_stability(None, ctypes.byref(rho)) == librdc.RDC_EINVAL


def test_params_reject_unknown_fields(librdc):
    with pytest.raises(TypeError):
        librdc.rdc_params_default(reserved=0)


def test_large_phi_map_validation_is_threaded_and_exact(librdc):
    """Maps larger than one scan chunk (2^22 cells) are validated on several
    host threads: an invalid value anywhere is still refused (before any
    device call), in every chunk position."""
    W, H = 4096, 3000                  # 12.3 M cells: several chunks
    p = librdc.rdc_params_default()
    for pos in (0, 5_000_000, W * H - 1):
        phi = np.full((H, W), 0.054, dtype=np.float32)
        phi.flat[pos] = np.nan if pos % 2 else 0.001
        with pytest.raises(librdc.RdcError) as e:
            librdc.rdc_create(W, H, p, phi)
        assert e.value.status == librdc.RDC_EINVAL, pos


def test_set_step_index_validates(librdc):
    import ctypes
    L = librdc.lib()
    assert L.rdc_set_step_index(None, 5) == librdc.RDC_EINVAL
    assert L.rdc_batch_set_step_index(None, 0, 5) == librdc.RDC_EINVAL


def test_noalloc_refuses_stochastic_rounding(librdc):
    """rdc_step_noalloc keeps no step index across calls, so it refuses
    RDC_STOCH_ROUND (before any device call)."""
    import ctypes
    L = librdc.lib()
    p = librdc.rdc_params_default(precision=2, flags=librdc.RDC_STOCH_ROUND, round_seed=1)
    fake = 1 << 40
    bad = ctypes.c_int64(0)
    from paper_1901_06535_gb300._capi import rdc_grid
    rc = L.rdc_step_noalloc(rdc_grid(16, 16), ctypes.byref(p), fake, fake + 4096,
                            fake + 8192, fake + 12288, fake + 16384, 64, 3, None,
                            ctypes.byref(bad))
    assert rc == librdc.RDC_EINVAL


def test_noalloc_scratch_limit_is_exact(librdc):
    """The static scratch (32 MiB) holds a 256-byte flag area and two state
    planes of roundup256(pitch * H) bytes: 2048 x 2048 FP32 (two 16 MiB
    planes) is 256 bytes over and is refused with RDC_EUNSUPPORTED before any
    device call (fake, never dereferenced addresses); so are the 16-bit and
    FP64 grids of the same plane size."""
    import ctypes
    L = librdc.lib()
    from paper_1901_06535_gb300._capi import rdc_grid
    fake = 1 << 40
    gap = 1 << 26                                       # 64 MiB apart: no overlap
    for prec, (w, h), esz in ((0, (2048, 2048), 4), (2, (4096, 2048), 2), (1, (1024, 2048), 8)):
        for kb, n in ((0, 3), (4, 5), (4, 8)):          # 3, 2 and 2 launches
            p = librdc.rdc_params_default(precision=prec, k_block=kb)
            rc = L.rdc_step_noalloc(rdc_grid(w, h), ctypes.byref(p), fake, fake + gap,
                                    fake + 2 * gap, fake + 3 * gap, fake + 4 * gap, w * esz,
                                    n, None, None)
            assert rc == librdc.RDC_EUNSUPPORTED, (prec, kb, n, rc)


def test_noalloc_refuses_outputs_that_overlap_another_buffer(librdc):
    """An output plane sharing any byte with another buffer of the call would
    be read through a restrict pointer while written: refused with RDC_EINVAL
    before any device call (fake, never dereferenced addresses)."""
    import ctypes
    L = librdc.lib()
    from paper_1901_06535_gb300._capi import rdc_grid
    W, H, pitch = 16, 16, 64                            # planes of 1024 bytes (FP32)
    fake = 1 << 40
    ui, vi, ph, uo, vo = (fake + i * 4096 for i in range(5))
    cases = {
        "v_out is u_in": (ui, vi, ph, uo, ui),
        "u_out is v_in": (ui, vi, ph, vi, vo),
        "u_out one row into u_in": (ui, vi, ph, ui + pitch, vo),
        "v_out ends inside u_in": (ui, vi, ph, uo, ui - 1008),
        "phi is u_out": (ui, vi, uo, uo, vo),
        "phi overlaps v_out": (ui, vi, vo + 512, uo, vo),
        "u_out overlaps v_out": (ui, vi, ph, uo, uo + 1008),
    }
    for name, (a, b, c, d, e) in cases.items():
        p = librdc.rdc_params_default(precision=0)
        rc = L.rdc_step_noalloc(rdc_grid(W, H), ctypes.byref(p), a, b, c, d, e, pitch, 3,
                                None, None)
        assert rc == librdc.RDC_EINVAL, name
    # FP64: phi is read as doubles, so a 1024-byte state plane's phi spans 2048 bytes
    p = librdc.rdc_params_default(precision=1)
    pitch64 = 128
    rc = L.rdc_step_noalloc(rdc_grid(W, H), ctypes.byref(p), fake, fake + 8192, fake + 16384,
                            fake + 16384 + 2048 - 16, fake + 32768, pitch64, 3, None, None)
    assert rc == librdc.RDC_EINVAL


def test_binding_checks_host_array_sizes(monkeypatch):
    """Host arrays passed to the library must hold one value per cell (the
    library reads or writes exactly width * height of them) and u and v the
    same dtype: the binding refuses anything else before calling the library
    (here a fake grid of 8 x 4 cells; the library is never reached)."""
    import numpy as np
    from paper_1901_06535_gb300 import _capi

    def no_lib():
        raise AssertionError("the library must not be called")

    monkeypatch.setattr(_capi, "lib", no_lib)
    monkeypatch.setattr(_capi, "rdc_get_view",
                        lambda h: _capi.rdc_view(width=8, height=4))
    monkeypatch.setattr(_capi, "rdc_batch_get_grid", lambda b, idx: (8, 4))
    good = np.zeros((4, 8))
    for bad in (np.zeros((4, 7)), np.zeros((3, 8)), np.zeros(33), np.zeros((8, 5))):
        for call in (lambda a: _capi.rdc_read(1, a, None),
                     lambda a: _capi.rdc_read(1, good, a),
                     lambda a: _capi.rdc_set_state(1, a, None),
                     lambda a: _capi.rdc_set_phi(1, a.astype(np.float32)),
                     lambda a: _capi.rdc_batch_read(1, 0, a, None),
                     lambda a: _capi.rdc_batch_set_state(1, 0, good, a)):
            with pytest.raises(ValueError, match="cells"):
                call(bad)
    for call in (lambda: _capi.rdc_read(1, good, good.astype(np.float32)),
                 lambda: _capi.rdc_batch_read(1, 0, good, good.astype(np.float32)),
                 lambda: _capi.rdc_batch_set_state(1, 0, good.astype(np.float16), good)):
        with pytest.raises(ValueError, match="same dtype"):
            call()


def test_batch_get_grid_validates(librdc):
    """rdc_batch_get_grid refuses a NULL batch or output (host only)."""
    import ctypes
    from paper_1901_06535_gb300._capi import rdc_grid
    L = librdc.lib()
    g = rdc_grid()
    assert L.rdc_batch_get_grid(None, 0, ctypes.byref(g)) == librdc.RDC_EINVAL
    assert L.rdc_batch_get_grid(None, 0, None) == librdc.RDC_EINVAL


def test_binding_checks_render_and_probe_buffers(monkeypatch):
    """rdc_render's caller-supplied output must be one contiguous RGBA8 image
    of the grid (W * H * 4 bytes); rdc_probe counts every index of a
    multi-dimensional index array (fake 8 x 4 grid; the library is only
    reached by the probe, through a fake that records the count)."""
    import numpy as np
    from paper_1901_06535_gb300 import _capi
    monkeypatch.setattr(_capi, "rdc_get_view", lambda h: _capi.rdc_view(width=8, height=4))
    seen = {}

    class FakeLib:
        def rdc_render(self, *a):
            raise AssertionError("an invalid output buffer reached the library")

        def rdc_probe(self, h, n, cells, out):
            seen["n"] = n
            return _capi.RDC_OK

    monkeypatch.setattr(_capi, "lib", lambda: FakeLib())
    for bad in (np.zeros((4, 8, 3), np.uint8), np.zeros((4, 7, 4), np.uint8),
                np.zeros((4, 8, 4), np.uint8)[:, ::2], np.zeros((4, 8, 4), np.uint16)):
        with pytest.raises(ValueError, match="out"):
            _capi.rdc_render(1, out=bad)
    out = _capi.rdc_probe(1, np.arange(12).reshape(3, 4))
    assert seen["n"] == 12 and out.shape == (12,)


def test_unusable_device_is_reported_not_hidden(librdc):
    """With no usable CUDA device (this machine), every call that needs one
    returns RDC_ECUDA with the runtime's message in rdc_last_error and no
    handle -- there is no CPU fallback -- and the library keeps answering
    host-only calls afterwards."""
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("needs a machine without a usable GPU")
    from paper_1901_06535_gb300._capi import rdc_grid
    L = librdc.lib()
    p = librdc.rdc_params_default()
    h = ctypes.c_void_p()
    assert L.rdc_create(rdc_grid(16, 16), ctypes.byref(p), None, None,
                        ctypes.byref(h)) == librdc.RDC_ECUDA
    assert h.value is None and librdc.rdc_last_error().startswith("cudaGetDevice")
    b = ctypes.c_void_p()
    assert L.rdc_batch_create(0, None, ctypes.byref(p), None, None,
                              ctypes.byref(b)) == librdc.RDC_ECUDA and b.value is None
    rep = librdc.rdc_division_report()
    assert L.rdc_check_division(0.002, 0, 0, ctypes.byref(rep)) == librdc.RDC_ECUDA
    # host-only calls still work, and validation still comes first
    assert librdc.rdc_rest_state(0.054, 1.4, 0.002) > 0.002
    bad = librdc.rdc_params_default()
    bad.dt = -1.0
    assert L.rdc_create(rdc_grid(16, 16), ctypes.byref(bad), None, None,
                        ctypes.byref(h)) == librdc.RDC_EINVAL


def test_binding_structures_match_the_header(tmp_path):
    """Every structure the binding passes through the C ABI has the header's
    size and field offsets (the header compiled by the host C compiler)."""
    import ctypes
    import shutil
    import subprocess
    from paper_1901_06535_gb300 import _capi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    structs = [_capi.rdc_grid, _capi.rdc_params, _capi.rdc_view, _capi.rdc_launch_shape,
               _capi.rdc_batch_info, _capi.rdc_division_report]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rdc.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for st in structs:
        n = st.__name__
        assert int(out[n]) == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert int(out[f"{n}.{f}"]) == getattr(st, f).offset, (n, f)
