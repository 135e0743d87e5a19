"""The C-ABI library loads and exports every symbol include/mpax.h declares; host-side
argument checks that return before any device work.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def C():
    from paper_2412_09734_gb300 import build
    build.build()
    from paper_2412_09734_gb300 import mpax
    return mpax


def declared_functions():
    with open(os.path.join(ROOT, "include", "mpax.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(mpax_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(C):
    lib = ctypes.CDLL(C.LIB_PATH)
    decl = declared_functions()
    assert len(decl) >= 17
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(C.EXPORTED) == decl


def test_version_and_defaults(C):
    assert "sm_103a" in C.mpax_version()
    o = C.mpax_options_default()
    # Appendix A defaults
    assert o.eps_abs == 1e-4 and o.eps_rel == 1e-4
    assert o.eps_primal_infeasible == 1e-8 and o.eps_dual_infeasible == 1e-8
    assert o.eps_feas_polish == 1e-6
    assert o.display_frequency == 10 and o.verbose == 0 and o.feasibility_polishing == 0
    assert o.iteration_limit == 2**63 - 1
    # rules fixed by this library
    assert o.check_every == 64 and o.ruiz_iters == 10 and o.pock_chambolle == 1
    assert o.reflection_gamma == 1.0 and o.step_safety == 0.998
    assert (o.restart_sufficient, o.restart_necessary, o.restart_artificial) == (0.2, 0.8, 0.36)


def test_struct_layout_matches_header(C, tmp_path):
    """Field offsets of the ctypes mirrors equal the C compiler's for mpax.h."""
    import subprocess
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mpax.h"', 'int main(void){']
    for cname, cls in (("mpax_options", C.Options), ("mpax_stats", C.Stats),
                       ("mpax_batch_stats", C.BatchStats)):
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for cname, cls in (("mpax_options", C.Options), ("mpax_stats", C.Stats),
                       ("mpax_batch_stats", C.BatchStats)):
        assert got[(cname, "size")] == ctypes.sizeof(cls)
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_invalid_sizes_rejected_before_device_work(C):
    h = ctypes.c_void_p()
    st = C._lib.mpax_lp_create(-1, 3, 0, None, None, None, None, None, None, None, None, 0,
                               None, ctypes.byref(h))
    assert st == 1 and "non-negative" in C.mpax_last_error()
    st = C._lib.mpax_lp_create(2, 3, 1 << 31, None, None, None, None, None, None, None, None,
                               0, None, ctypes.byref(h))
    assert st == 7
    rp = np.array([0, 1, 2], dtype=np.int64)
    st = C._lib.mpax_lp_create(2, 3, 2, rp.ctypes.data, None, None, None, None, None, None,
                               None, 0, None, ctypes.byref(h))
    assert st == 1 and "NULL" in C.mpax_last_error()
    st = C._lib.mpax_lp_create(2, 3, 2, rp.ctypes.data, None, None, None, None, None, None,
                               None, 5, None, ctypes.byref(h))
    assert st == 1
    assert C._lib.mpax_get_stats(None, None) == 1
    C.mpax_destroy(None)


def test_status_strings(C):
    for s in range(8):
        assert C._lib.mpax_status_string(s).decode() != "unknown status"


def test_new_entry_points_check_arguments_before_device_work(C):
    """mpax_qp_create, mpax_lp_create_f32, mpax_qp_unrolled_grad and
    mpax_get_reduced_cost reject bad arguments on the host."""
    h = ctypes.c_void_p()
    rp = np.array([0, 1, 2], dtype=np.int64)
    # general sparse Q without its row pointer
    st = C._lib.mpax_qp_create(2, 3, 0, rp.ctypes.data, None, None, None, None, None, None,
                               None, 0, None, None, None, 0, None, ctypes.byref(h))
    assert st == C.MPAX_ERR_INVALID_ARGUMENT and "q_row_ptr" in C.mpax_last_error()
    # Q with entries but no column indices
    st = C._lib.mpax_qp_create(2, 3, 0, rp.ctypes.data, None, None, None, None, None, None,
                               None, 4, rp.ctypes.data, None, None, 0, None, ctypes.byref(h))
    assert st == C.MPAX_ERR_INVALID_ARGUMENT
    # Q with 2^31 entries
    st = C._lib.mpax_qp_create(2, 3, 0, rp.ctypes.data, None, None, None, None, None, None,
                               None, 1 << 31, rp.ctypes.data, None, None, 0, None, ctypes.byref(h))
    assert st == C.MPAX_ERR_UNSUPPORTED
    # FP32 create: negative sizes, bad memory kind, NULL vectors
    st = C._lib.mpax_lp_create_f32(-1, 3, 0, None, None, None, None, None, None, None, None,
                                   0, None, ctypes.byref(h))
    assert st == C.MPAX_ERR_INVALID_ARGUMENT
    st = C._lib.mpax_lp_create_f32(2, 3, 0, rp.ctypes.data, None, None, None, None, None, None,
                                   None, 7, None, ctypes.byref(h))
    assert st == C.MPAX_ERR_INVALID_ARGUMENT and "kind" in C.mpax_last_error()
    st = C._lib.mpax_lp_create_f32(2, 3, 0, rp.ctypes.data, None, None, None, None, None, None,
                                   None, 0, None, ctypes.byref(h))
    assert st == C.MPAX_ERR_INVALID_ARGUMENT and "NULL" in C.mpax_last_error()
    # differentiation and getters on a NULL problem
    g = np.zeros(3)
    assert C._lib.mpax_qp_unrolled_grad(None, g.ctypes.data, None, None, None, None, None,
                                        None, None, 0) == C.MPAX_ERR_INVALID_ARGUMENT
    assert C._lib.mpax_get_reduced_cost(None, g.ctypes.data, 0) == C.MPAX_ERR_INVALID_ARGUMENT
    # record_tape is an FP64 option: the default leaves it off
    assert C.mpax_options_default().record_tape == 0


def test_qp_layers_free_their_handle_without_backward(C, monkeypatch):
    """Host logic of the QP layers: a forward whose inputs need no gradient (no_grad,
    constants) frees its handle at once, since no backward will free it."""
    from paper_2412_09734_gb300 import autograd as AG
    freed = []
    monkeypatch.setattr(AG.C, "mpax_destroy", lambda h: freed.append(h))

    class Ctx:
        pass

    ctx = Ctx()
    ctx.needs_input_grad = (False, False, False, False, False)
    assert AG._keep_if_needed(ctx, "h1") is None and freed == ["h1"]
    ctx.needs_input_grad = (False, True, False, False, False)
    k = AG._keep_if_needed(ctx, "h2")
    assert k.h == "h2" and freed == ["h1"]
    k.close()  # after backward: freed once
    k.close()
    assert freed == ["h1", "h2"]
    # a kept handle whose backward never comes is freed when dropped
    k3 = AG._keep_if_needed(ctx, "h3")
    del k3
    import gc
    gc.collect()
    assert freed == ["h1", "h2", "h3"]


def test_qp_layers_release_handles_on_every_path(C, monkeypatch):
    """With a fake library (no GPU): each QP layer frees its handle exactly once
    after backward, under no_grad, and when its graph is dropped unused."""
    import gc
    import types

    import torch

    from paper_2412_09734_gb300 import autograd as AG
    log = []
    f64 = torch.float64
    fake = types.SimpleNamespace(
        MPAX_PREC_FP64=0,
        mpax_qp_create_diag_lowrank=lambda *a, **k: "H",
        mpax_solve=lambda h, o: None,
        mpax_options_default=lambda **k: None,
        mpax_get_solution=lambda h, m, n, device=None: (torch.zeros(n, dtype=f64), None),
        mpax_destroy=lambda h: log.append(h),
        mpax_qp_adjoint=lambda h, g, m, n: (torch.ones(n, dtype=f64),) * 3 + ({},),
        mpax_qp_unrolled_grad=lambda h, g, m, n: {"c": torch.ones(n, dtype=f64),
                                                  "lc": torch.zeros(m, dtype=f64),
                                                  "uc": torch.zeros(m, dtype=f64),
                                                  "D": torch.ones(n, dtype=f64)})
    monkeypatch.setattr(AG, "C", fake)
    data = dict(m=2, n=3, row_ptr=None, col=None, val=None, l=None, u=None, f_row_ptr=None,
                f_col=None, f_val=None, r=1)
    for layer in (AG.QPLayer, AG.QPUnrolledLayer):
        c = torch.zeros(3, dtype=f64, requires_grad=True)
        b = torch.zeros(2, dtype=f64)
        D = torch.ones(3, dtype=f64)
        log.clear()
        layer.apply(c, b, D, data, {}).sum().backward()
        assert log == ["H"] and c.grad.tolist() == [1.0, 1.0, 1.0]
        log.clear()
        with torch.no_grad():
            layer.apply(c, b, D, data, {})
        gc.collect()
        assert log == ["H"]
        log.clear()
        x = layer.apply(c, b, D, data, {})
        del x
        gc.collect()
        assert log == ["H"]
