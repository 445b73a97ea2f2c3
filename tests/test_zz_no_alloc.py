"""pm_power_spectrum_static: the power spectrum for callers that cannot call
cudaMalloc (the scratch is a fixed file-scope device array inside libpmgb).
Its output must match the handle-based pm_power_spectrum within the P(k)
tolerance of the parity tests (1e-4 relative per bin), on two calls in a row
(the array keeps the previous call's contents, so each call must clear it).
This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_2510_05206_gb300 import PM, Config, inputs
from paper_2510_05206_gb300.pm import power_spectrum_static

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_static_power_spectrum_matches_handle_api_twice():
    n_part, L = 64, 300.0
    pm = PM(Config(n_part=n_part, n_mesh=64, box=L), device=DEV)
    for seed, n_mesh, n_bins in ((41, 64, 32), (42, 32, 12)):
        psi = inputs.random_displacements(n_part, scale=5.0, seed=seed)
        disp = torch.tensor(psi[None], dtype=torch.float32, device=DEV).contiguous()
        k_ref, p_ref, c_ref = pm.power_spectrum(disp, n_mesh, n_bins)
        k, p, c = power_spectrum_static(disp[0], n_part, L, n_mesh, n_bins)
        np.testing.assert_array_equal(c, c_ref[0])
        np.testing.assert_allclose(k, k_ref[0], rtol=1e-12)
        ok = c > 0
        assert np.max(np.abs(p[ok] / p_ref[0][ok] - 1)) < 1e-4


def test_static_power_spectrum_rejects_large_mesh():
    disp = torch.zeros((3, 32 ** 3), dtype=torch.float32, device=DEV)
    with pytest.raises(RuntimeError):
        power_spectrum_static(disp, 32, 100.0, 128, 8)
