"""GPU forward mode (JVPs of the DKD run and of P(k)) through the C ABI, against
the FP64 oracle's forward mode, and against the GPU reverse mode through the
dot-product identity <u, J t> = <J^T u, t>.

Tolerances: with TSC/PCS (smooth kernels) max |t_gpu - t_oracle| <= 2e-4 of the
rms tangent; with CIC a float32 position on the other side of a cell face
changes that particle's kernel derivative by O(1), so the relative L2 error is
used (<= 2e-3), as for the CIC adjoint.
"""
import numpy as np
import pytest
import torch

from oracle import nbody
from paper_2510_05206_gb300 import PM, Config, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV)


def _np(t):
    return t.double().cpu().numpy()


def _rms(a):
    return np.sqrt(np.mean(np.sum(a ** 2, axis=0)))


@pytest.mark.parametrize("order", [3, 2, 4])
def test_jvp_run_matches_oracle(order):
    n, L = 32, 200.0
    kw = dict(n_part=n, n_mesh=n, box=L, order=order, n_steps=3)
    pm = PM(Config(**kw), device=DEV)
    w = inputs.white_noise(n, seed=41)
    wt = inputs.white_noise(n, seed=42)
    d, v = pm.ic_zeldovich(_t(w.reshape(1, -1)))
    td, tv = pm.ic_zeldovich(_t(wt.reshape(1, -1)))      # the ICs are linear in the noise
    pm.jvp(d, v, td, tv)
    ocfg = nbody.Config(**kw)
    P0, V0 = nbody.zeldovich_ic(ocfg, w)
    Pt0, Vt0 = nbody.zeldovich_ic(ocfg, wt)
    P, V, Pt, Vt = nbody.run_jvp(ocfg, P0, V0, Pt0, Vt0)
    assert np.max(np.abs(_np(d)[0] - P)) / _rms(P) < 1e-4
    for got, ref in ((_np(td)[0], Pt), (_np(tv)[0], Vt)):
        if order >= 3:
            assert np.max(np.abs(got - ref)) / _rms(ref) < 2e-4
        else:
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-3


def test_power_spectrum_jvp_matches_oracle():
    n, L = 32, 150.0
    pm = PM(Config(n_part=n, n_mesh=n, box=L), device=DEV)
    Psi = inputs.random_displacements(n, scale=3.0, seed=43)
    T = inputs.random_displacements(n, scale=1.0, seed=44)
    k, pk, dpk, cnt = pm.power_spectrum_jvp(_t(Psi[None]), _t(T[None]), n, 16)
    kr, dr, cr = nbody.power_spectrum_jvp(Psi, T, n, L, 16, order=2)
    np.testing.assert_array_equal(cnt[0], cr)
    assert np.max(np.abs(dpk[0] - dr)) / np.max(np.abs(dr)) < 2e-3


@pytest.mark.parametrize("order", [3, 2])
def test_jvp_and_adjoint_dot_product(order):
    # <u, J t> from the forward mode equals <J^T u, t> from the reverse mode
    n, L = 32, 200.0
    pm = PM(Config(n_part=n, n_mesh=n, box=L, order=order, n_steps=4), device=DEV)
    d0, v0 = pm.ic_zeldovich(_t(inputs.white_noise(n, seed=45).reshape(1, -1)))
    t0d, t0v = pm.ic_zeldovich(_t(inputs.white_noise(n, seed=46).reshape(1, -1)))
    d, v, td, tv = d0.clone(), v0.clone(), t0d.clone(), t0v.clone()
    pm.jvp(d, v, td, tv)
    ud = _t(inputs.random_displacements(n, 1.0, seed=47)[None])
    uv = _t(inputs.random_displacements(n, 1.0, seed=48)[None])
    lhs = float((ud.double() * td.double()).sum() + (uv.double() * tv.double()).sum())
    ad, av = ud.clone(), uv.clone()
    pm.adjoint(d, v, ad, av)
    rhs = float((ad.double() * t0d.double()).sum() + (av.double() * t0v.double()).sum())
    assert lhs == pytest.approx(rhs, rel=(2e-4 if order == 3 else 2e-3))
