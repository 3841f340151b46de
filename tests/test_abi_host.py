"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point that include/sfp.h declares, and its parameter derivation
reproduces the constants printed in the paper."""
import ctypes as ct
import os
import re

import pytest

import paper_1411_3487_gb300 as sfp
from golden_values import PAPER
from paper_1411_3487_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "sfp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sfp_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = _lib.load()
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s
    assert set(syms) == set(_lib.EXPORTS)


def test_derive_dsdna_matches_printed_constants():
    d = sfp.derive()
    assert d["Tstar"] == PAPER["Tstar"] and d["nu"] == PAPER["nu"]
    assert round(d["b"], 1) == PAPER["b_approx"]                       # Sec. 2A
    assert round(d["d_nm"], 1) == PAPER["d_nm_approx"]                 # Sec. 2A
    assert round(d["lp_over_a"]) == PAPER["lp_bp_approx"]              # Eq. a3, Sec. 7B
    assert round(d["c_ps"], 2) == PAPER["c_ps_approx"]                 # Eq. relat
    # Table 2: dtau_max -> dt_max in ps
    for n in (64, 128, 256, 512):
        assert round(PAPER[f"dtau_max_{n}"] * d["c_ps"], 2) == pytest.approx(PAPER[f"dt_max_ps_{n}"], abs=0.011)
    # l_p in nm (Table 0 caption / Sec. 8: 37.6-37.7 nm)
    assert d["lp_over_a"] * PAPER["a_nm"] == pytest.approx(PAPER["lp_nm"], abs=0.2)


def test_derive_from_physical_stiffnesses_round_trips():
    d = sfp.derive()
    p = sfp.params_dsdna()
    p.lambda_pN_per_nm = d["lambda_pN_per_nm"]
    p.kappa_pN_per_nm = d["kappa_pN_per_nm"]
    p.T_star = 0.0
    p.nu = 0.0
    e = sfp.derive(p)
    assert e["Tstar"] == pytest.approx(PAPER["Tstar"], rel=1e-12)
    assert e["nu"] == pytest.approx(PAPER["nu"], rel=1e-12)
    # a^2 xi / kT recomputed from a, xi, kT instead of the printed 52.0 ps
    p.a2xi_over_kT_ps = 0.0
    f = sfp.derive(p)
    a2xi = PAPER["a_nm"] ** 2 * PAPER["xi_kg_per_s"] / PAPER["kT_pN_nm"] * 1e15
    assert f["c_ps"] == pytest.approx(PAPER["Tstar"] * (1 - 2 * PAPER["nu"]) ** 2 * a2xi, rel=1e-12)
    # t = xi tau / lambda  (Sec. 3)
    assert f["c_ps"] == pytest.approx(PAPER["xi_kg_per_s"] / (d["lambda_pN_per_nm"] * 1e-3) * 1e12, rel=1e-9)


@pytest.mark.parametrize("nu", [0.0, 0.5, 0.7, -0.1])
def test_derive_rejects_unstable_nu(nu):
    """Sec. 2: stability of Eq. a2 needs 0 < nu < 1/2."""
    p = sfp.params_dsdna()
    p.nu = nu
    with pytest.raises(sfp.SfpError) as e:
        sfp.derive(p)
    assert e.value.code == _lib.SFP_EINVAL
    assert "nu" in _lib.load().sfp_last_error().decode()


def test_create_rejects_bad_arguments_before_touching_the_gpu():
    L = _lib.load()
    p = sfp.params_dsdna()
    h = ct.c_void_p()
    d = (_lib.SfpChainDesc * 1)()
    d[0].n_beads = 2
    d[0].dtau = 1.0
    assert L.sfp_create(ct.byref(p), d, 1, 1, sfp.SFP_FP32, None, 0, ct.byref(h)) == _lib.SFP_EINVAL
    d[0].n_beads = 64
    d[0].dtau = 0.0
    d[0].dt_ps = -1.0
    assert L.sfp_create(ct.byref(p), d, 1, 1, sfp.SFP_FP32, None, 0, ct.byref(h)) == _lib.SFP_EINVAL
    d[0].dtau = 1.0
    d[0].job_id = 1 << 32
    assert L.sfp_create(ct.byref(p), d, 1, 1, sfp.SFP_FP32, None, 0, ct.byref(h)) == _lib.SFP_EINVAL
    d[0].job_id = 0
    assert L.sfp_create(ct.byref(p), d, 1, 1 << 33, sfp.SFP_FP32, None, 0, ct.byref(h)) == _lib.SFP_EINVAL
    assert L.sfp_create(ct.byref(p), d, 1, 1, 99, None, 0, ct.byref(h)) == _lib.SFP_EINVAL
    assert h.value is None


def test_product_path_has_no_oracle_dependency():
    """The CUDA path and its binding never import or link the oracle."""
    pkg = os.path.join(ROOT, "paper_1411_3487_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower(), f
