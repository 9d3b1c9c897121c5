"""Row patterns (a one- or two-byte form index per row instead of the CSR offsets and columns)
give exactly the CSR results: the exchange sum adds the same terms in the same order.  Checked bit for bit on
the workload lattices, in both precisions and every step kind that reads rows."""
import numpy as np
import pytest

from paper_1310_6143_gb300 import lattice as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SS():
    from paper_1310_6143_gb300.system import SpinSystem

    return SpinSystem


def _run(SS, lats, patterns, precision, kw, steps=12, mc=0):
    with SS(lats, precision=precision, **kw) as s:
        s.set_row_patterns(patterns)
        info = s.info()
        s.step(steps)
        rec = s.record(0, steps)
        if mc:
            s.mc_step(mc)
        S = s.spins()
        m, e = s.magnetisation(), s.energy()
    return info, S, rec, m, e


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name", ["film", "sc_open", "fcc", "core_shell", "grains"])
def test_patterns_bitwise_equal_to_csr(SS, name, precision):
    kw = dict(alpha=0.05, dt=1e-16, T=600.0, seed=3)
    if name == "film":  # in-plane periodic, free z surfaces: rows of 5 and 6
        lats, forms = L.film(48, 40, 16), True
    elif name == "sc_open":  # one free axis, a field, anisotropy
        lats, forms = L.simple_cubic(9, 7, 11, periodic=(True, False, True), k_u=1e-24), True
        kw["H"] = (0.3, 0.0, 0.1)
    elif name == "fcc":  # rows of 12
        lats, forms = L.fcc(6, 5, 7), True
    elif name == "core_shell":  # irregular surface rows, three J values
        lats, forms = L.core_shell_sphere(diameter=4e-9, r_core=1.5e-9), None
    else:  # a batch of grains (each system's own rows)
        g, temps = L.grain_ensemble(count=6, n_min=300, n_max=900, layers=4, seed=7)
        lats, forms = g, None
        kw.update(T=[float(t) for t in temps], seed=[11 + k for k in range(6)])
    on = _run(SS, lats, True, precision, kw, mc=3)
    off = _run(SS, lats, False, precision, kw, mc=3)
    assert off[0]["row_patterns"] == 0
    if forms:
        assert 0 < on[0]["row_patterns"] <= 256
    for a, b in zip(on[1:], off[1:]):
        np.testing.assert_array_equal(a, b)


def test_film_form_count(SS):
    """The film's rows come in 27 forms (bulk, top and bottom surface, times the in-plane wraps)."""
    with SS(L.film(32, 24, 16), precision="fp32") as s:
        assert s.info()["row_patterns"] == 27


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_two_byte_forms_bitwise_equal_to_csr(SS, precision):
    """A batch whose rows take more than 256 forms (40 grains of ragged shapes) stores two-byte
    form indices; the results are still the CSR's bit for bit."""
    g, temps = L.grain_ensemble(count=40, n_min=2000, n_max=6000, layers=5, seed=21)
    kw = dict(alpha=0.05, dt=1e-16, T=[float(t) for t in temps], seed=[5 + k for k in range(40)],
              sys_id=list(range(40)))
    on = _run(SS, g, True, precision, kw, mc=2)
    off = _run(SS, g, False, precision, kw, mc=2)
    assert 256 < on[0]["row_patterns"] <= 65536 and off[0]["row_patterns"] == 0
    for a, b in zip(on[1:], off[1:]):
        np.testing.assert_array_equal(a, b)


def test_more_forms_than_two_bytes_keep_the_csr(SS):
    """The 20 nm core-shell sphere's rows take 76,795 forms (offsets that follow the sphere's
    ragged atom rows, three J values), more than a two-byte index holds: the handle reads the
    CSR."""
    with SS(L.core_shell_sphere(), precision="fp32", alpha=0.1, dt=1e-16, T=10.0) as s:
        assert s.info()["row_patterns"] == 0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name", ["sc_open", "fcc64"])
def test_tensor_forms_bitwise_equal_to_csr(SS, name, precision):
    """Tensor bonds with an interface Dzyaloshinskii-Moriya term and cubic anisotropy: the forms
    hold each bond's tensor entry in place of J, and the results are the CSR's bit for bit, in
    the Heun steps, the records and Monte Carlo.  sc with a free axis (rows of up to 6 bonds, 27
    forms); fcc 64^3 as benchmarked (rows of 12, 17,959 forms: the DM vectors' last bits follow
    the positions, two-byte indices)."""
    if name == "sc_open":
        lat = L.with_dm(L.simple_cubic(9, 7, 11, periodic=(True, False, True), k_u=1e-24, with_pos=True), D=1e-21)
        steps, mc = 12, 3
    else:
        lat = L.with_dm(L.fcc(64, 64, 64, J=11.2e-21, k_u=6.69e-24, with_pos=True), D=1.12e-21)
        steps, mc = 4, 1
    lat.k_c = np.full(lat.n, 5e-24)
    kw = dict(alpha=0.05, dt=1e-16, T=300.0, seed=4, H=(0.1, 0.0, 0.2))
    on = _run(SS, lat, True, precision, kw, steps=steps, mc=mc)
    off = _run(SS, lat, False, precision, kw, steps=steps, mc=mc)
    assert on[0]["row_patterns"] > 0 and off[0]["row_patterns"] == 0
    for a, b in zip(on[1:], off[1:]):
        np.testing.assert_array_equal(a, b)
