"""The small dense hermitian eigensolver of the Rayleigh-Ritz step (Algorithm 2's
HEEVD call), through chase_bse_eigh: scalar FP64 Jacobi, the mixed-precision solver
of a mixed solve (FP32 block Jacobi, Ogita-Aishima refinement, FP64 on what stays
coupled) and FP64 block Jacobi, against numpy's eigvalsh on planted spectra shaped
like the Rayleigh-Ritz problem's (+-theta pairs, a dense band near the top)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2601_10557_gb300 as p
    return p


def planted(k, seed, band=0.3):
    """G = U diag(theta) U^* with theta = +-1/lambda, lambda ~ U[1, 40] with a fraction
    `band` of them in [1, 1.2] (nearly equal pairs), U Haar unitary."""
    rng = np.random.default_rng(seed)
    h = k // 2
    lam = rng.uniform(1.0, 40.0, size=h)
    nb = int(band * h)
    lam[:nb] = rng.uniform(1.0, 1.2, size=nb)
    th = np.concatenate([1.0 / lam, -1.0 / lam])
    Z = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
    Q, R = np.linalg.qr(Z)
    Q = Q * (np.diag(R) / np.abs(np.diag(R)))[None, :]
    G = (Q * th[None, :]) @ Q.conj().T
    return 0.5 * (G + G.conj().T)


@pytest.mark.parametrize("method", ["jacobi", "mixed", "block"])
@pytest.mark.parametrize("k", [96, 520, 1040])
def test_eigh_matches_numpy(pkg, method, k):
    if method == "mixed" and not pkg.has_mixed():
        pytest.fail("tensor-core path not available on this device")
    G = planted(k, k)
    theta, V = pkg.eigh(torch.from_numpy(G).cuda(), method=method, thr=2e-16)
    theta = theta.cpu().numpy()
    V = V.cpu().numpy()
    ref = np.linalg.eigvalsh(G)
    nrm = np.linalg.norm(G, 2)
    assert np.abs(np.sort(theta) - ref).max() <= 1e-12 * nrm
    # residual of a column: the couplings left below the solver's threshold (at most
    # 1e-13 of the diagonal in the mixed solver) summed over the column, plus rounding
    assert np.linalg.norm(G @ V - V * theta, axis=0).max() <= (1e-12 + 1e-13 * np.sqrt(k)) * nrm
    assert np.abs(V.conj().T @ V - np.eye(k)).max() <= 1e-12
