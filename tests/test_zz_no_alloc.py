"""GPU test of pm_mse_loss_noalloc, the allocation-free entry point for
callers that cannot call cudaMalloc (memory fully reserved by another
allocator, or loops that cannot take cudaMalloc's device-wide
synchronisation).  It is called through the C ABI and must agree with the
existing pm_mse_loss on two calls in a row (the second with different
inputs, so leftovers of the first call in the shared scratch would show).
Kept in a file that pytest collects last."""

import ctypes

import numpy as np
import pytest
import torch

from paper_2211_09958_gb300 import _pmgb, inputs

pytestmark = pytest.mark.gpu


def _noalloc(lib, n_p, n_m, box, s, target, want_grad=True):
    loss = torch.zeros(s.shape[0], dtype=torch.float64, device=s.device)
    dlds = torch.empty_like(s) if want_grad else None
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.pm_mse_loss_noalloc(n_p, n_m, s.shape[0], box, ctypes.c_void_p(s.data_ptr()),
                                 ctypes.c_void_p(target.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                 ctypes.c_void_p(dlds.data_ptr()) if dlds is not None else None,
                                 ctypes.c_void_p(stream))
    assert rc == 0, rc
    torch.cuda.synchronize()
    return loss.cpu().numpy(), dlds


def test_noalloc_matches_pm_mse_loss_twice():
    from paper_2211_09958_gb300.pm import ParticleMesh
    lib = _pmgb.load()
    n_p, n_m, box = 16, 32, 64.0
    pm = ParticleMesh(n_p, n_m, box, 0.3, 0.8, 2)
    for call in range(2):
        s = torch.from_numpy(inputs.random_displacements(n_p, box, seed=40 + call, scale=0.7 + 0.3 * call))[None].cuda()
        target = torch.from_numpy(inputs.target_field(n_m, 50 + call))[None].cuda()
        ref_loss, ref_g = pm.mse_loss(s, target)
        loss, g = _noalloc(lib, n_p, n_m, box, s, target)
        assert abs(loss[0] - ref_loss[0]) <= 1e-5 * abs(ref_loss[0]), (call, loss, ref_loss)
        scale = torch.max(torch.abs(ref_g)).item()
        assert torch.max(torch.abs(g - ref_g)).item() <= 1e-4 * scale, call
    pm.close()


def test_noalloc_batched_and_limits():
    lib = _pmgb.load()
    n_p, n_m, box, nb = 8, 16, 32.0, 3
    s = torch.from_numpy(np.stack([inputs.random_displacements(n_p, box, seed=60 + b) for b in range(nb)])).cuda()
    target = torch.from_numpy(np.stack([inputs.target_field(n_m, 70 + b) for b in range(nb)])).cuda()
    loss, _ = _noalloc(lib, n_p, n_m, box, s, target, want_grad=False)
    from paper_2211_09958_gb300.pm import ParticleMesh
    pm = ParticleMesh(n_p, n_m, box, [0.3] * nb, [0.8] * nb, 2)
    ref, _ = pm.mse_loss(s, target, want_grad=False)
    np.testing.assert_allclose(loss, ref, rtol=1e-5)
    pm.close()
    # 256^3 cells exceed the fixed scratch: rejected before any device work
    big = lib.pm_mse_loss_noalloc(128, 256, 1, 256.0, ctypes.c_void_p(s.data_ptr()),
                                  ctypes.c_void_p(target.data_ptr()), ctypes.c_void_p(s.data_ptr()), None, None)
    assert big == -5
