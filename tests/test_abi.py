"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/lbm.h declares; host-only calls validate their
arguments. No compute call runs here."""
import ctypes
import os
import re

import pytest

from paper_2403_16122_gb300 import build as lbm_build
from paper_2403_16122_gb300 import inputs, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    lbm_build.build()
    return lbm.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_\w+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(lbm.SYMBOLS)


def test_params_struct_layout_matches_header():
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    body = txt[txt.index("typedef struct lbm_params"):txt.index("} lbm_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for typ, names in re.findall(r"(int32_t|double)\s+([^;]+);", body):
        for n in names.split(","):
            fields.append((n.strip(), typ))
    got = [(n, "int32_t" if t is ctypes.c_int32 else "double") for n, t in lbm.lbm_params._fields_]
    assert got == fields
    assert ctypes.sizeof(lbm.lbm_params) == 10 * 4 + 26 * 8


def test_workspace_size_host_only(lib):
    p, _, _ = inputs.stefan()
    n1 = lbm.lbm_workspace_size([p])
    # 2 buffers x (27 + 5) planes of 256 x 8 floats at least
    assert n1 >= 2 * 32 * 256 * 8 * 4
    n2 = lbm.lbm_workspace_size([p, p])
    assert n2 > 1.9 * n1 - 4096
    p16, _, _ = inputs.sessile(nx=64, ny=48, R=16.0)
    assert lbm.lbm_workspace_size([p16], lbm.LBM_STORE_FP16) < lbm.lbm_workspace_size([p16])


@pytest.mark.parametrize("bad", [dict(nx=2), dict(tau_h=0.5), dict(mobility=0.0),
                                 dict(theta_deg=0.0), dict(T_w=0.5), dict(Ste=-1.0),
                                 dict(pc_ramp=0.0), dict(periodic_x=2), dict(normal_eps=0.0),
                                 dict(k_ratio_sl=0.0), dict(Cp_ratio_gl=-1.0),
                                 dict(beta_T=float("inf"))])
def test_invalid_parameters_rejected(lib, bad):
    p = inputs.params(**bad)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_workspace_size([p])
    assert e.value.code == lbm.LBM_EINVAL


def test_unsupported_storage_rejected(lib):
    p = inputs.params()
    with pytest.raises(lbm.LbmError):
        lbm.lbm_workspace_size([p], storage=7)
    # BF16 takes the FP16 arrangement, and like it needs the strip layouts
    assert lbm.lbm_workspace_size([p], storage=lbm.LBM_STORE_BF16) == \
        lbm.lbm_workspace_size([p], storage=lbm.LBM_STORE_FP16)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_workspace_size([dict(p, periodic_x=0)], storage=lbm.LBM_STORE_BF16)


def test_error_strings(lib):
    for code in range(-6, 1):
        assert lbm.lbm_error_string(code)
    assert "unknown" in lbm.lbm_error_string(-99)


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_step_count(None) == -1
    lib.lbm_destroy(None)


def test_largest_lattice_accepted_and_one_row_more_refused(lib):
    """The state offsets are 32-bit: a lattice is accepted while 27 planes of
    it stay below 2^31 elements (8192 x 9709 is the last 8192-wide one; its
    two FP32 state buffers take 81 GB) and refused one row later."""
    ok = inputs.params(nx=8192, ny=9709, periodic_x=1, periodic_y=0)
    nbytes = lbm.lbm_workspace_size([ok])
    assert nbytes >= 2 * 8192 * 9709 * 32 * 4
    bad = inputs.params(nx=8192, ny=9710, periodic_x=1, periodic_y=0)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_workspace_size([bad])
    assert e.value.code == lbm.LBM_EINVAL


def test_step_kernels_keep_their_state_in_registers(lib):
    """The row-staged FP32 plain steps (128 and 168 registers), the 168-register
    observable step and the 168-register FP16 steps spill nothing: a spill in
    the step costs it several per cent. nvcc's code for a kernel depends on the
    rest of its file (the file is partitioned for parallel compilation), so an
    unrelated edit can change this; the report is that of the library's own
    build."""
    rep = lbm_build.ptxas_report()
    if not any("step_strip_staged" in k for k in rep):
        lbm_build.build(force=True)  # a library built before the report was kept
        rep = lbm_build.ptxas_report()
    want = ["ILi4ELi4ELi3ELb0EfE", "ILi4ELi3ELi3ELb0EfE", "ILi4ELi3ELi3ELb1EfE",
            "ILi4ELi3ELi3ELb0E6__halfE", "ILi4ELi3ELi3ELb1E6__halfE"]
    for tag in want:
        hits = [v for k, v in rep.items() if "step_strip_staged" + tag in k]
        assert len(hits) == 1, tag
        regs, spill = hits[0]
        assert spill == 0, (tag, regs, spill)
    # the 128-register variant really holds its budget
    assert [v for k, v in rep.items() if "step_strip_stagedILi4ELi4ELi3ELb0EfE" in k][0][0] <= 128
