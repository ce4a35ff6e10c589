"""CPU checks of the C-ABI library: it loads, exports every function include/chfpe.h declares,
and rejects invalid arguments before touching a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2509_25840_b300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(chfpe_\w+)\s*\(", text))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    lib = libbuild.build()
    declared = _declared()
    assert {"chfpe_create", "chfpe_response2", "chfpe_equilibrate"} <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (chfpe_\w+)", out))
    missing = declared - exported
    assert not missing, missing
    ctypes.CDLL(lib)       # loads without a GPU


def test_create_rejects_invalid_arguments_on_cpu():
    from paper_2509_25840_b300 import chfpe, inputs
    libbuild.build()
    wl = inputs.one_mode_64()
    bad = [
        dict(depth=9),                 # beyond the compiled range for one mode
        dict(dt=1.0),                  # above the RK4 stability bound
        dict(precision=16),
        dict(max_batch=-1),
        dict(bf16_tier=2),             # not a compiled (modes, depth, tier) combination
        dict(q_scheme=1),              # the compact q scheme needs Hermite momenta
        dict(p_basis=1, q_scheme=3),   # no such scheme
    ]
    for kw in bad:
        args = dict(depth=wl.depth, dt=wl.dt, precision=32, max_batch=1)
        args.update(kw)
        with pytest.raises(chfpe.ChfpeError) as e:
            chfpe.Handle(wl.model, wl.grid, **args)
        assert e.value.status == chfpe.EINVAL, (kw, str(e.value))
    small = inputs.Grid(nq=(6,), np=(64,), qmin=(-6,), qmax=(6,), pmin=(-6,), pmax=(6,))
    with pytest.raises(chfpe.ChfpeError):
        chfpe.Handle(wl.model, small, depth=2, dt=0.005)
    # the max-index truncation is declared but not built
    import ctypes
    m, g = chfpe.make_model(wl.model), chfpe.make_grid(wl.grid)
    o = chfpe.chfpe_options(depth=wl.depth, precision=32, dt=wl.dt, max_batch=1, truncation=1)
    h = ctypes.c_void_p()
    assert chfpe.load().chfpe_create(ctypes.byref(m), ctypes.byref(g), ctypes.byref(o),
                                     ctypes.byref(h)) == chfpe.EINVAL
    assert "truncation" in chfpe.last_error() and not h.value


def test_surrogate_host_entry_points_on_cpu():
    """Parameter count agrees with the oracle's layer list; create rejects bad sizes before
    touching a device."""
    import ctypes
    from oracle import surrogate_oracle as so
    from paper_2509_25840_b300 import chfpe
    lib = chfpe.load()
    assert lib.chfpe_surrogate_param_count() == so.param_count()
    h = ctypes.c_void_p()
    for bad in (0, -3, 4097):
        assert lib.chfpe_surrogate_create(bad, 1, None, ctypes.byref(h)) == chfpe.EINVAL
        assert not h.value
