"""Gradient of the disc's m = 2 Fourier amplitude through the autograd binding of the
forward run and msh_adjoint_run: FP64 against central finite differences of the forward
run, FP32 against FP64."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_5246_gb300 import disc, msh
    msh.load()
    return disc, msh


def test_disc_gradient_fp64_matches_central_fd(mods):
    disc, msh = mods
    D = disc.DiscProblem(n=48, nsteps=40, precision=msh.FP64, K=7)
    L0, gd, gb = D.value_and_grad(beta=0.05)
    assert 0 < L0 < 1
    with torch.no_grad():
        h = 1e-5
        fd_b = (float(D.loss(D.delta0, torch.tensor(0.05 + h, dtype=torch.float64, device="cuda")))
                - float(D.loss(D.delta0, torch.tensor(0.05 - h, dtype=torch.float64, device="cuda")))) / (2 * h)
        assert abs(fd_b - gb) <= 1e-4 * abs(fd_b) + 1e-9, (fd_b, gb)
        rng = np.random.default_rng(3)
        v = torch.tensor(rng.normal(size=D.delta0.shape), device="cuda") * 0.01
        b = torch.tensor(0.05, dtype=torch.float64, device="cuda")
        h = 1e-4
        fd_d = (float(D.loss(D.delta0 + h * v, b)) - float(D.loss(D.delta0 - h * v, b))) / (2 * h)
        ad_d = float((gd * v).sum())
        assert abs(fd_d - ad_d) <= 1e-3 * abs(fd_d) + 1e-9, (fd_d, ad_d)
    D.close()


def test_disc_gradient_fp32_close_to_fp64(mods):
    disc, msh = mods
    out = {}
    for prec in (msh.FP32, msh.FP64):
        D = disc.DiscProblem(n=128, nsteps=200, precision=prec, K=50)
        out[prec] = D.value_and_grad(beta=0.0)
        D.close()
    L32, gd32, gb32 = out[msh.FP32]
    L64, gd64, gb64 = out[msh.FP64]
    assert abs(L32 - L64) <= 1e-3 * L64
    assert abs(gb32 - gb64) <= 1e-2 * abs(gb64)
    rel = float(torch.linalg.norm(gd32 - gd64) / torch.linalg.norm(gd64))
    assert rel <= 1e-2, rel
