"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/fdf.h declares; the ctypes structures match the C layout; host-only
validation works without a device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fdf():
    from paper_2207_14256_gb300 import build
    from paper_2207_14256_gb300 import fdf as F

    build.build()
    F.lib()
    return F


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fdf.h")).read()
    return sorted(set(re.findall(r"^FDF_API [^(]*?\b(fdf_\w+)\(", src, re.M)))


def test_every_declared_symbol_is_exported(fdf):
    names = declared_symbols()
    assert len(names) >= 16
    L = C.CDLL(fdf.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", fdf.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (fdf_\w+)$", out, re.M))
    assert set(names) <= exported
    # nothing else of ours leaks out of the library
    assert {n for n in exported if n.startswith("fdf")} == set(names)


def _c_offsets():
    code = r'''
#include <stdio.h>
#include <stddef.h>
#include "fdf.h"
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("fdf_params %zu\n", sizeof(fdf_params));
  printf("fdf_tables %zu\n", sizeof(fdf_tables));
  O(fdf_params, box_mpc); O(fdf_params, n_part); O(fdf_params, n_grid); O(fdf_params, n_species);
  O(fdf_params, m_ev); O(fdf_params, T_nu_K); O(fdf_params, z_start); O(fdf_params, z_end);
  O(fdf_params, n_steps); O(fdf_params, precision); O(fdf_params, seed); O(fdf_params, h);
  O(fdf_params, omega_m); O(fdf_params, omega_r); O(fdf_params, A_s); O(fdf_params, n_s);
  O(fdf_params, k_pivot); O(fdf_params, flags); O(fdf_params, n_gl); O(fdf_params, sort_every); O(fdf_params, steps_per_pass);
  O(fdf_params, sort_tile); O(fdf_params, sort_cells); O(fdf_params, interp_order);
  O(fdf_params, superstep_tol); O(fdf_params, eom); O(fdf_params, pass_blocks); O(fdf_params, gather_tile); O(fdf_params, deposit_presum);
  O(fdf_tables, nk); O(fdf_tables, na); O(fdf_tables, lnk); O(fdf_tables, lna); O(fdf_tables, T_psi);
  O(fdf_tables, T_phi); O(fdf_tables, dTphi_dlna); O(fdf_tables, ncdf); O(fdf_tables, cdf_t);
  O(fdf_tables, cdf_F);
  printf("fdf_request_info %zu\n", sizeof(fdf_request_info));
  O(fdf_request_info, id); O(fdf_request_info, status); O(fdf_request_info, error); O(fdf_request_info, t_submit);
  O(fdf_request_info, t_admit); O(fdf_request_info, t_done); O(fdf_request_info, footprint);
  O(fdf_request_info, particle_steps); O(fdf_request_info, message);
  return 0;
}
'''
    tmp = os.path.join(ROOT, "_build_abi_check")
    os.makedirs(tmp, exist_ok=True)
    src = os.path.join(tmp, "layout.c")
    exe = os.path.join(tmp, "layout")
    open(src, "w").write(code)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return dict((l.split()[0], int(l.split()[1])) for l in out.strip().splitlines())


def test_struct_layout_matches_c(fdf):
    c = _c_offsets()
    assert c["fdf_params"] == C.sizeof(fdf.fdf_params)
    assert c["fdf_tables"] == C.sizeof(fdf.fdf_tables)
    assert c["fdf_request_info"] == C.sizeof(fdf.fdf_request_info)
    for name, cls in (("fdf_params", fdf.fdf_params), ("fdf_tables", fdf.fdf_tables),
                      ("fdf_request_info", fdf.fdf_request_info)):
        for f in cls._fields_:
            key = "%s.%s" % (name, f[0])
            if key in c:
                assert getattr(cls, f[0]).offset == c[key], key


def test_host_only_calls(fdf, inputs):
    assert fdf.fdf_error_string(0) == "ok"
    assert fdf.fdf_error_string(-4) == "call out of order"
    n = 3 * 256 ** 3
    # FP64 state (x, q FP64, q0 FP32, p, id, and the sampler's fixed-point positions) in
    # both halves of the sort's double buffer, plus 96-byte sort records
    b = fdf.fdf_footprint(fdf.make_params(inputs.config("c3_3x256")))
    assert b > n * 2 * (24 + 24 + 12 + 12 + 8 + 4)
    assert b < 24 * 2 ** 30
    # the split state: 36 bytes of positions and momenta per particle
    b = fdf.fdf_footprint(fdf.make_params(inputs.config("c3_3x256", precision=fdf.FDF_PREC_F32_FIXED)))
    assert b > n * (12 + 12 + 12 + 24 + 8 + 4)
    assert b < 16 * 2 ** 30
    bad = fdf.make_params(inputs.config("c1_32", n_grid=48))
    with pytest.raises(fdf.FdfError) as e:
        fdf.fdf_footprint(bad)
    assert e.value.code == fdf.FDF_EINVAL
    assert "power of two" in fdf.fdf_last_error()
    bad = fdf.make_params(inputs.config("c1_32", z_end=2e9))
    with pytest.raises(fdf.FdfError):
        fdf.fdf_footprint(bad)
    bad = fdf.make_params(inputs.config("c1_32", n_species=5, m_ev=[0.1] * 4))
    with pytest.raises(fdf.FdfError):
        fdf.fdf_footprint(bad)
    for knob in (dict(interp_order=3), dict(sort_tile=4), dict(sort_cells=-1), dict(steps_per_pass=9),
                 dict(superstep_tol=-0.1), dict(superstep_tol=float("nan")), dict(eom=6), dict(eom=-1),
                 dict(precision=0, eom=5, steps_per_pass=3), dict(precision=5), dict(precision=-1),
                 dict(flags=4), dict(pass_blocks=4), dict(pass_blocks=-1), dict(gather_tile=2), dict(deposit_presum=2)):
        with pytest.raises(fdf.FdfError) as e:
            fdf.fdf_footprint(fdf.make_params(inputs.config("c1_32", **knob)))
        assert e.value.code == fdf.FDF_EINVAL, knob
    # the comparison equations of motion exist in the plain FP64 form only
    with pytest.raises(fdf.FdfError) as e:
        fdf.fdf_footprint(fdf.make_params(inputs.config("c1_32", precision=1, eom=3)))
    assert e.value.code == fdf.FDF_ENOSYS
    assert fdf.fdf_footprint(fdf.make_params(inputs.config("c1_32", precision=0, eom=3))) > 0
    with pytest.raises(fdf.FdfError) as e:
        fdf.fdf_footprint(fdf.make_params(inputs.config("c1_32", precision=1, eom=fdf.FDF_EOM_EXACT)))
    assert e.value.code == fdf.FDF_ENOSYS
    # the exact form carries phi + psi per particle (both halves of the sort's double buffer)
    p = inputs.config("c1_32", precision=0)
    extra = fdf.fdf_footprint(fdf.make_params(dict(p, eom=fdf.FDF_EOM_EXACT))) - fdf.fdf_footprint(
        fdf.make_params(p))
    n = p["n_part"] * p["n_species"]
    assert abs(extra - 2 * n * 8) <= 4096, extra


def test_create_rejects_bad_tables_before_touching_the_device(fdf, inputs, c1_tables):
    p = inputs.config("c1_32")
    t = dict(c1_tables)
    t["lnk"] = t["lnk"].copy()
    t["lnk"][5] += 0.01  # not uniform
    P = fdf.make_params(p)
    T, keep = fdf.make_tables(t)
    with pytest.raises(fdf.FdfError) as e:
        fdf.fdf_create(P, T)
    assert e.value.code == fdf.FDF_EINVAL


def test_binding_constants_match_the_header(fdf):
    """Every integer #define of include/fdf.h that the binding defines has the same
    value there, and every entry point the header declares is bound with that name."""
    src = open(os.path.join(ROOT, "include", "fdf.h")).read()
    defines = {}
    for name, val in re.findall(r"^#define (FDF_\w+)\s+\(?(-?\d+)\)?", src, re.M):
        defines[name] = int(val)
    assert len(defines) >= 30
    checked = 0
    for name, val in defines.items():
        if hasattr(fdf, name):
            assert getattr(fdf, name) == val, name
            checked += 1
    # the codes, forms, quantities, equations of motion and kernel classes are all mirrored
    for prefix in ("FDF_E", "FDF_PREC_", "FDF_Q_", "FDF_EOM_", "FDF_K_PUSH", "FDF_REQ_"):
        names = [n for n in defines if n.startswith(prefix)]
        assert names and all(hasattr(fdf, n) for n in names), prefix
    assert checked >= 30
    for name in declared_symbols():
        assert hasattr(fdf, name), name


def test_noalloc_binding_refuses_bad_outputs_without_a_kernel(fdf, inputs, c1_tables):
    """The binding checks fdf_build_fields_noalloc's output tensor before the library is
    called: a wrong dtype, size or device would let the kernels write past it."""
    torch = pytest.importorskip("torch")
    p = inputs.config("c1_32", n_grid=16, precision=1)
    P = fdf.make_params(p)
    T, keep = fdf.make_tables(c1_tables)
    N = p["n_grid"]
    with pytest.raises(TypeError):
        fdf.fdf_build_fields_noalloc(P, T, -10.0, np.zeros(8 * N ** 3))
    with pytest.raises(ValueError, match="float64"):
        fdf.fdf_build_fields_noalloc(P, T, -10.0, torch.zeros(8 * N ** 3, dtype=torch.float32))
    with pytest.raises(ValueError, match="8 n_grid"):
        fdf.fdf_build_fields_noalloc(P, T, -10.0, torch.zeros(8, dtype=torch.float64))
    with pytest.raises(ValueError, match="contiguous"):
        fdf.fdf_build_fields_noalloc(P, T, -10.0, torch.zeros(16 * N ** 3, dtype=torch.float64)[::2])
    with pytest.raises(ValueError, match="device memory"):
        fdf.fdf_build_fields_noalloc(P, T, -10.0, torch.zeros(8 * N ** 3, dtype=torch.float64))
