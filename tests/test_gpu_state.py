"""State transfer through the C ABI: set_state/get_state with pageable numpy arrays and with
pinned arrays (read and written in place by one kernel each way) against the definition:
phi and psi scaled by 1/F with F = sum_i A_i sum_g nuSigma_f phi, zero inflow on track ends no
link feeds, k unchanged."""
import numpy as np
import pytest

from paper_2607_01591_gb300 import moc
from paper_2607_01591_gb300 import workloads as W
from paper_2607_01591_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _pinned(a):
    import torch
    out = torch.empty(a.shape, dtype=torch.float64, pin_memory=True).numpy()
    out[...] = a
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("memory", ["pageable", "pinned"])
def test_state_round_trip(precision, memory):
    prob = W.small_lattice_problem(3, bc=(1, 0, 1, 0), n_azim=24, ray_spacing=0.03)
    m = moc.Moc.from_problem(prob, precision=precision)
    T, _ = m.track_counts()
    R, G = prob.mesh.n_tri, prob.xs.n_groups
    rng = np.random.default_rng(5)
    phi = rng.uniform(0.5, 1.5, (R, G))
    psi = rng.uniform(0.0, 0.3, (T, 2, 3, G))
    if memory == "pinned":
        phi, psi = _pinned(phi), _pinned(psi)
    m.set_state(phi, 1.234, psi)
    if memory == "pinned":
        phi2, psi2 = _pinned(np.zeros((R, G))), _pinned(np.zeros((T, 2, 3, G)))
        _, k2, _ = m.get_state(out=(phi2, psi2))
    else:
        phi2, k2, psi2 = m.get_state(with_psi=True)
    A = m.areas()
    F = float((A[:, None] * prob.xs.nu_sigma_f[prob.mesh.mat] * phi).sum())
    link = m.tracks()["link"].ravel()
    fed = np.zeros(2 * T, bool)
    fed[link[link >= 0]] = True
    psi_exp = np.where(fed.reshape(T, 2)[:, :, None, None], psi, 0.0) / F
    tol = 1e-14 if precision == "fp64" else 1e-7
    assert k2 == 1.234
    np.testing.assert_allclose(phi2, phi / F, rtol=tol)
    np.testing.assert_allclose(psi2, psi_exp, rtol=tol, atol=0)
    # the same outers from pinned and from pageable copies of one state agree up to the order
    # of the sweep's atomic additions: in FP64 that order moves k by rounding only; in FP32 the
    # compensated tally (one Fast2Sum step per addition) is exact only while the running sum
    # outweighs the addend, so a different order leaves a residue near 2^-24 per region tally,
    # about 1e-10 of k after two outers
    m.set_state(phi, 1.234, psi)
    k_a, _ = m.outer(2)
    m.set_state(np.array(phi), 1.234, np.array(psi))
    k_b, _ = m.outer(2)
    rep = 1e-13 if precision == "fp64" else 1e-8
    assert abs(k_a - k_b) <= rep * k_a
