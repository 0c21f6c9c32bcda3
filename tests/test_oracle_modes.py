"""Small-amplitude eigenmodes: a sine perturbation along one right eigenvector of the x
Jacobian (computed numerically from complex-step derivatives of the Gaussian-moment flux,
independent of the oracle's closed-form eigen-system) travels at that eigenvalue.  For the
slow and fast acoustic waves, the shear waves and the contact, in every scheme of the
oracle, the L1 error against the translated linear wave falls at second order (>= 1.9
between 128 and 256 cells, the MC limiter clipping the extrema) and is small."""
import numpy as np
import pytest

from tests import bruteforce as BF

W0 = np.array([1.0, 0.3, 0.1, -0.2, 1.0, 0.2, 0.1, 0.8, 0.05, 0.6])
EPS = 1e-6
MODES = {"fast-": 0, "shear-": 1, "contact": 3, "shear+": 8, "fast+": 9}
SCHEMES = {"hll": 0, "kt": 1, "roe": 2, "hllc": 3}


@pytest.fixture(scope="module")
def eig():
    _, lam, R = BF.eigen(W0, 0)
    return lam, R


def _error(oracle, lam, R, k, n, scheme, travel=0.5):
    x = (np.arange(n) + 0.5) / n
    r = R[:, k] / np.abs(R[:, k]).max()
    W = W0[:, None] + EPS * np.sin(2 * np.pi * x)[None, :] * r[:, None]
    g = oracle.Grid((n,), (0.0,), (1.0,), ((0, 0),), 0.5, scheme=scheme)
    U, ns, t, rc, _ = oracle.run(g, oracle.prim_to_cons(W.reshape(10, 1, 1, n)), travel / abs(lam[k]))
    assert rc == 0
    Wn = oracle.cons_to_prim(U).reshape(10, n)
    exact = W0[:, None] + EPS * np.sin(2 * np.pi * (x - lam[k] * t))[None, :] * r[:, None]
    return np.abs(Wn - exact).sum() / n / EPS


@pytest.mark.parametrize("scheme", list(SCHEMES))
@pytest.mark.parametrize("mode", list(MODES))
def test_eigenmode_second_order(oracle, eig, scheme, mode):
    lam, R = eig
    k = MODES[mode]
    e = [_error(oracle, lam, R, k, n, SCHEMES[scheme]) for n in (64, 128, 256)]
    order = np.log2(e[1] / e[2])
    assert order >= 1.9 and e[2] <= 1e-3, (e, order)
