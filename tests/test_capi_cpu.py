"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every entry point include/janc.h declares; the Python binding has a
function of the same name for each; argument validation fails cleanly."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2504_13750_gb300 import build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "janc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(janc_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libjanc():
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("no nvcc")
    path = build.build()
    return ctypes.CDLL(path)


def test_header_symbols_exported(libjanc):
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(libjanc, n), n


def test_binding_names_match_header():
    from paper_2504_13750_gb300 import janc

    for n in declared_symbols():
        assert callable(getattr(janc, n, None)), n


def test_workspace_and_validation_without_gpu(libjanc):
    from paper_2504_13750_gb300 import janc

    mech = janc.Mechanism(inputs.load_mechanism("h2air_synth"))
    d = janc.make_desc(4096, 512, 1e-5, 1e-5, [0, 0, 0, 0])
    nbytes = janc.janc_workspace_bytes(d, mech)
    n = 4096 * 512
    # 3 states of 16 planes + 2 face-flux arrays of 12 planes, plus small tables
    assert 3 * 16 * n * 8 + 2 * 12 * n * 8 <= nbytes < 3 * 16 * n * 8 + 2 * 12 * (n + 4096 + 512) * 8 + (1 << 20)
    bad = janc.make_desc(2, 4, 1e-5, 1e-5, [0, 0, 0, 0])  # walls need >= 3 cells
    with pytest.raises(janc.JancError) as e:
        janc.janc_workspace_bytes(bad, mech)
    assert e.value.rc == -1 and "nx >= 3" in str(e.value)
    m5 = inputs.load_mechanism("h2air_synth")
    m5 = dict(m5, ns=5)
    with pytest.raises(janc.JancError) as e:
        janc.janc_workspace_bytes(d, janc.Mechanism({**m5, "M": m5["M"][:5], "nasa": m5["nasa"][:5]}))
    assert e.value.rc == -2
    per = janc.make_desc(16, 16, 1e-5, 1e-5, [2, 0, 0, 0])
    with pytest.raises(janc.JancError):
        janc.janc_workspace_bytes(per, mech)


def test_oracle_and_product_share_no_code():
    """The oracle and the CUDA path import nothing from each other."""
    pkg = os.path.join(ROOT, "paper_2504_13750_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"^\s*(?:import|from)\s+(\w+)", text, flags=re.M), f
                assert "janc_oracle" not in text, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".cpp", ".hpp")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "csrc" not in text and "janc_device" not in text and "import janc" not in text, f


def test_new_entry_points_validate_without_gpu(libjanc):
    """Argument checks of the AMR, server-budget, source-step and chemistry
    modes return before any CUDA call."""
    from paper_2504_13750_gb300 import janc

    mech = janc.Mechanism(inputs.load_mechanism("h2air_synth"))
    d = janc.make_desc(64, 16, 1e-4, 1e-4, [0, 0, 0, 0])
    amr = janc.AmrDesc(2, 16, 1e6, 2, 10, 0)
    for bad, rc in ((janc.AmrDesc(2, 32, 1e6, 2, 10, 0), -2),     # block must be 16
                    (janc.AmrDesc(9, 16, 1e6, 2, 10, 0), -1),     # levels 0..6
                    (janc.AmrDesc(2, 16, 1e6, -1, 10, 0), -1),    # buffer >= 0
                    (janc.AmrDesc(2, 16, 1e6, 2, 0, 0), -1)):     # regrid period >= 1
        with pytest.raises(janc.JancError) as e:
            janc.janc_amr_create(d, mech, bad)
        assert e.value.rc == rc
    odd = janc.make_desc(60, 16, 1e-4, 1e-4, [0, 0, 0, 0])         # not a multiple of 8
    with pytest.raises(janc.JancError) as e:
        janc.janc_amr_create(odd, mech, amr)
    assert e.value.rc == -1
    for mode in (janc.CHEM_STRANG, janc.CHEM_EXPLICIT):           # AMR runs the Lie order
        with pytest.raises(janc.JancError) as e:
            janc.janc_amr_create(janc.make_desc(64, 16, 1e-4, 1e-4, [0, 0, 0, 0], chemistry=mode), mech, amr)
        assert e.value.rc == -2
    with pytest.raises(janc.JancError) as e:                         # chemistry mode out of range
        janc.janc_workspace_bytes(janc.make_desc(64, 16, 1e-4, 1e-4, [0, 0, 0, 0], chemistry=7), mech)
    assert e.value.rc == -1
    assert janc.janc_workspace_bytes(janc.make_desc(64, 16, 1e-4, 1e-4, [0, 0, 0, 0], chemistry=janc.CHEM_EXPLICIT),
                                     mech) > 0
    with pytest.raises(janc.JancError):                              # null server
        janc.janc_server_set_cell_budget(None, 1000)
    with pytest.raises(janc.JancError):                              # null grid
        janc.janc_source_step(None, 1, 1e-8)


def test_binding_marshals_host_arrays_and_rejects_the_rest():
    """The binding only marshals: C-contiguous float64 numpy arrays are host
    arguments, anything else is refused before the C call (there is no
    conversion or CPU path), and one call never mixes host and device."""
    from paper_2504_13750_gb300 import janc

    a = np.zeros((3, 4))
    ptr, where, keep = janc._arg(a, True)
    assert where == janc.JANC_HOST and keep is a and ptr.value == a.ctypes.data
    assert janc._arg(None) == (None, janc.JANC_HOST, None)
    for bad in (np.zeros((3, 4), dtype=np.float32), np.zeros((4, 3)).T, [0.0, 1.0]):
        with pytest.raises(ValueError):
            janc._arg(bad)
    ro = np.zeros(5)
    ro.flags.writeable = False
    janc._arg(ro)                       # read-only input is fine
    with pytest.raises(ValueError):
        janc._arg(ro, True)             # but not as an output
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        janc._arg(torch.zeros(4, dtype=torch.float64))   # a CPU tensor is not a device array
    host = janc._arg(a)
    fake_dev = (ctypes.c_void_p(1), janc.JANC_DEVICE, object())
    assert janc._where(host, janc._arg(None)) == janc.JANC_HOST
    with pytest.raises(ValueError):
        janc._where(host, fake_dev)
    assert janc.chem_mode(True) == janc.CHEM_LIE and janc.chem_mode(False) == janc.CHEM_OFF
    assert janc.chem_mode(janc.CHEM_EXPLICIT) == 3


def test_rhs_static_refuses_mismatched_buffers_before_the_call():
    """janc_rhs_static's binding checks every buffer's size against the grid
    and its device against the current one, so that an undersized or foreign
    tensor never reaches the kernels (checked on stand-ins: no GPU here)."""
    from paper_2504_13750_gb300 import janc

    class Buf:
        def __init__(self, n, dev=0):
            self.n, self.device = n, type("D", (), {"index": dev})()

        def numel(self):
            return self.n

    d = janc.make_desc(10, 4, 1e-4, 1e-4, [0, 0, 0, 0])
    ns, cells = 9, 40
    ok = dict(U=Buf(12 * cells), T=Buf(cells), L=Buf(12 * cells), alpha=Buf(2))
    janc._rhs_static_shapes(d, ns, device=0, **ok)
    janc._rhs_static_shapes(d, ns, device=0, **dict(ok, alpha=None))
    for bad in (dict(U=Buf(12 * cells - 1)), dict(T=Buf(cells + 1)), dict(L=Buf(11 * cells)), dict(alpha=Buf(1)),
                dict(L=Buf(12 * cells, dev=1)), dict(T=None)):
        with pytest.raises(ValueError):
            janc._rhs_static_shapes(d, ns, device=0, **dict(ok, **bad))


def test_fixed_structure_header_is_generated_from_the_mechanism():
    """csrc/janc_mech_fixed.cuh is exactly what mech_codegen writes from the
    shipped mechanism file, and encodes its structure: species and
    coefficients of every reaction side, third-body flags, and the species
    with a third-body coefficient other than one."""
    from paper_2504_13750_gb300 import mech_codegen

    with open(mech_codegen.HEADER) as f:
        assert f.read() == mech_codegen.render()
    m = inputs.load_mechanism("h2air_synth")
    sp, rx = mech_codegen.structure()
    assert sp == m["species"] and len(rx) == m["nr"]
    for i, r in enumerate(rx):
        assert r["nuf"] == list(m["nuf"][i]) and r["nub"] == list(m["nub"][i]) and r["tb"] == int(m["tb"][i])
        assert r["eff_ne1"] == [k for k in range(m["ns"]) if m["tb"][i] and m["eff"][i][k] != 1.0]


def test_adjoint_mode_refuses_a_null_grid(libjanc):
    from paper_2504_13750_gb300 import janc

    for mode in (janc.ADJ_RECOMPUTE, janc.ADJ_STORE_FACES, 7):
        with pytest.raises(janc.JancError) as e:
            janc.janc_set_adjoint_mode(None, mode)
        assert e.value.rc == -1
