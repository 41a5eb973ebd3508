"""Anisotropic (P_L) scattering on the GPU against the oracle. The library carries angular
moments against real harmonics (addition theorem); the oracle evaluates the scattering source
of every direction by a direct double sum over directions with P_l of the scattering cosine --
two different computations of the same discrete method."""
import numpy as np
import pytest

import oracle
from paper_2607_01591_gb300 import moc
from paper_2607_01591_gb300 import workloads as W
from paper_2607_01591_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


@pytest.mark.parametrize("L,precision,tol", [(1, "fp64", 1e-10), (2, "fp64", 1e-10), (3, "fp64", 1e-10),
                                             (1, "fp32", 2e-5), (3, "fp32", 2e-5)])
def test_aniso_outers_match_oracle(L, precision, tol):
    prob = W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=16, ray_spacing=0.05)
    ssl = W.anisotropic_moments(prob.xs, L, [0.05, 0.1, 0.4])
    o = oracle.Oracle.from_problem(prob, threads=8)
    o.set_scattering(ssl)
    m = moc.Moc.from_problem(prob, precision=precision)
    m.set_scattering(ssl)
    T, _ = m.track_counts()
    G = prob.xs.n_groups
    rng = np.random.default_rng(31)
    phi0 = rng.uniform(0.5, 1.5, (prob.mesh.n_tri, G))
    psi0 = rng.uniform(0.0, 0.2, (T, 2, 3, G))
    o.set_state(phi0, 1.1, psi0)
    o.normalise()
    m.set_state(phi0, 1.1, psi0)
    for it in range(4):
        o.outer(True)
        kg, _ = m.outer(1)
        phio, ko = o.get_state()
        assert abs(kg - ko) <= tol * ko, (it, kg, ko)
        assert _rel(m.get_state()[0], phio) <= 10 * tol, (it, _rel(m.get_state()[0], phio))


def test_p1_bare_square_converges_to_the_oracle():
    mesh = W.grid_mesh(8, 8, 4.0, 4.0, bc=(0, 0, 0, 0))
    xs = W.CrossSections(np.array([[1.0]]), np.array([[0.25]]), np.array([[1.0]]), np.array([[[0.9]]]))
    prob = W.Problem(mesh, xs, 16, 0.05)
    ssl = W.anisotropic_moments(xs, 1, [0.4])
    o = oracle.Oracle.from_problem(prob)
    o.set_scattering(ssl)
    ko, _, _, co = o.iterate(True, 1e-11, 1e-10, 5000)
    m = moc.Moc.from_problem(prob, precision="fp64")
    m.set_scattering(ssl)
    k, n, r, c = m.power_iterate(1e-11, 1e-10, 5000, check_every=1)
    assert co and c
    assert abs(k - ko) <= 1e-9 * ko
    assert _rel(m.get_state()[0], o.get_state()[0]) <= 1e-7


def test_aniso_and_cmfd_are_exclusive():
    prob = W.small_lattice_problem(3)
    m = moc.Moc.from_problem(prob, precision="fp64")
    m.set_scattering(W.anisotropic_moments(prob.xs, 1, [0.1, 0.1, 0.1]))
    cell, nc = W.grid_cells(prob.mesh, 1.26)
    with pytest.raises(moc.MocError):
        m.set_cmfd(cell, nc, 4, 4)


def test_p1_full_assembly_outers_match_oracle():
    """The bench's full-size assembly (9.1M segments) with P1 scattering: 3 outers from the same
    state, GPU FP64 vs oracle after each."""
    prob = W.assembly_problem()
    ssl = W.anisotropic_moments(prob.xs, 1, [0.05, 0.05, 0.4])
    o = oracle.Oracle.from_problem(prob, threads=8)
    o.set_scattering(ssl)
    o.normalise()
    m = moc.Moc.from_problem(prob, precision="fp64")
    m.set_scattering(ssl)
    for it in range(3):
        o.outer(True)
        kg, _ = m.outer(1)
        phio, ko = o.get_state()
        assert abs(kg - ko) <= 1e-10 * ko, (it, kg, ko)
        assert _rel(m.get_state()[0], phio) <= 1e-9, (it, _rel(m.get_state()[0], phio))
