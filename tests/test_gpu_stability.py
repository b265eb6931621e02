"""The instability record of forward Euler at the rest state (§2's scheme with
Table 1's dt): every simulation and batch grid records, when it is created
and whenever its phi map changes, whether the homogeneous rest state of the
map's largest phi is linearly unstable under forward Euler.  phi = 0.054
(Table 1's phi_active) is stable; phi = 0.2 (the workloads' passive
background) is not.

The recorded rho = max |1 + dt lambda| is checked against an independent
evaluation: the eigenvalues (numpy) of the hand-derived Jacobian of Eq. 1's
reaction term at the oracle's rest state, shifted by the discrete Laplacian's
spectrum from 0 to -8 Du / dx^2."""
from __future__ import annotations

import numpy as np
import pytest

from tests.oracle_pins import DT, DU, DX, analytic_jacobian

pytestmark = pytest.mark.gpu

W, H = 96, 64


def _rho(orc, phi):
    us = orc.rest_state(phi)
    J = analytic_jacobian(us, us, phi)
    rho = 0.0
    for shift in np.linspace(-8.0 * DU / DX ** 2, 0.0, 65):
        lam = np.linalg.eigvals(J + np.diag([shift, 0.0]))
        rho = max(rho, float(np.max(np.abs(1.0 + DT * lam))))
    return rho


def _map(background, band=None):
    phi = np.full((H, W), background, dtype=np.float32)
    if band is not None:
        phi[20:30, :] = band
    return phi


@pytest.mark.parametrize("background,band,unstable", [(0.054, None, False), (0.054, 0.2, True),
                                                      (0.2, None, True), (0.0975, None, False)])
def test_create_records_stability(gpu, orc, background, band, unstable):
    h = gpu.rdc_create(W, H, gpu.rdc_params_default(), _map(background, band))
    try:
        view = gpu.rdc_get_view(h)
        rc, rho = gpu.rdc_stability(h)
    finally:
        gpu.rdc_destroy(h)
    assert bool(view.unstable) == unstable
    assert rc == (gpu.RDC_EUNSTABLE_WARN if unstable else gpu.RDC_OK)
    assert view.stability_rho == rho
    phimax = float(np.float32(band if band is not None else background))
    assert rho == pytest.approx(_rho(orc, phimax), rel=1e-12)
    assert (rho > 1.0) == unstable


def test_record_follows_phi_changes(gpu):
    h = gpu.rdc_create(W, H, gpu.rdc_params_default())
    try:
        assert gpu.rdc_get_view(h).unstable == 0
        gpu.rdc_draw_line(h, 10, 10, 80, 10, 3, 0.2)
        assert gpu.rdc_get_view(h).unstable == 1
        gpu.rdc_fill_phi(h, 0.054)
        assert gpu.rdc_get_view(h).unstable == 0
        gpu.rdc_set_phi(h, _map(0.2))
        assert gpu.rdc_get_view(h).unstable == 1
        gpu.rdc_set_phi(h, _map(0.054))
        assert gpu.rdc_get_view(h).unstable == 0
    finally:
        gpu.rdc_destroy(h)


@pytest.mark.parametrize("band", [None, 0.2, 0.0975])
def test_caller_owned_map_is_scanned_on_the_device(gpu, band):
    """rdc_create_ext finds the largest phi of a device map: the record equals
    that of the same map created from the host, bit for bit."""
    import torch
    pitch = 128
    phi = _map(0.054, band)
    dphi = torch.zeros((H, pitch), dtype=torch.float32, device="cuda")
    dphi[:, :W] = torch.from_numpy(phi).cuda()
    dphi[:, W:] = 0.3            # padding beyond the grid's columns is not part of the map
    planes = [torch.zeros((H, pitch), dtype=torch.float32, device="cuda") for _ in range(4)]
    p = gpu.rdc_params_default()
    he = gpu.rdc_create_ext(W, H, p, [planes[0].data_ptr(), planes[1].data_ptr()],
                            [planes[2].data_ptr(), planes[3].data_ptr()], dphi.data_ptr(),
                            pitch * 4)
    hh = gpu.rdc_create(W, H, p, phi)
    try:
        ve, vh = gpu.rdc_get_view(he), gpu.rdc_get_view(hh)
    finally:
        gpu.rdc_destroy(he)
        gpu.rdc_destroy(hh)
    assert ve.unstable == vh.unstable == (1 if band == 0.2 else 0)
    assert ve.stability_rho == vh.stability_rho


def test_batch_grids_record_stability(gpu, orc):
    p = gpu.rdc_params_default()
    b = gpu.rdc_batch_create([(W, H), (40, 30)], [p, p], [_map(0.054), None])
    try:
        i = gpu.rdc_batch_add(b, W, H, p, _map(0.054, 0.2))
        assert gpu.rdc_batch_stability(b, 0)[0] == gpu.RDC_OK
        assert gpu.rdc_batch_stability(b, 1)[0] == gpu.RDC_OK
        rc, rho = gpu.rdc_batch_stability(b, i)
        assert rc == gpu.RDC_EUNSTABLE_WARN
        assert rho == pytest.approx(_rho(orc, float(np.float32(0.2))), rel=1e-12)
    finally:
        gpu.rdc_batch_destroy(b)
