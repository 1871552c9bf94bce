"""Host uploads through the C ABI: lbm_set_fields and lbm_set_state give the
same state from pageable host memory (staged through a device buffer),
page-locked host memory (read by the upload kernel in place) and device
memory."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _solver():
    from paper_2607_07432_b300 import lbmib
    return lbmib.Solver("D3Q19", "fp32", (24, 20, 16), mach=0.2, reynolds=50.0, ref_length=6.0,
                        bc=[lbmib.BC_PERIODIC] * 6)


def _fields(s, seed):
    rng = np.random.default_rng(seed)
    th = s.constants()["theta_inf"]
    N = s.N
    rho = 1.0 + 0.05 * rng.standard_normal(N)
    u = 0.05 * rng.standard_normal(3 * N)
    T = th * (1.0 + 0.05 * rng.standard_normal(N))
    return rho, u, T


def test_set_fields_pinned_pageable_device_agree():
    import torch
    s = _solver()
    rho, u, T = _fields(s, 11)
    states = []
    # pageable numpy arrays
    s.set_fields(rho, u, T)
    states.append(s.state())
    # page-locked host tensors (numpy views of them reach the C ABI)
    pins = [torch.from_numpy(a).pin_memory() for a in (rho, u, T)]
    s.set_fields(*[p.numpy() for p in pins])
    states.append(s.state())
    # device tensors
    devs = [torch.from_numpy(a).cuda() for a in (rho, u, T)]
    s.set_fields(*devs, device=True)
    states.append(s.state())
    for f, E in states[1:]:
        assert np.array_equal(f, states[0][0])
        assert np.array_equal(E, states[0][1])
    # the uploaded state steps like any other
    s.step(3)
    s.check()
    s.close()


def test_set_state_pinned_equals_pageable():
    import torch
    s = _solver()
    rho, u, T = _fields(s, 12)
    s.set_fields(rho, u, T)
    s.step(2)
    f, E = s.state()
    f2 = f * (1.0 + 1e-3 * np.random.default_rng(3).standard_normal(f.shape))
    s.set_state(f2, E)
    a = s.state()
    fp, Ep = torch.from_numpy(np.ascontiguousarray(f2)).pin_memory(), torch.from_numpy(E).pin_memory()
    s.set_state(fp.numpy(), Ep.numpy())
    b = s.state()
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    s.close()
