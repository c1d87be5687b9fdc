"""Allocation-free RDP entry point (pet_rdp_static), for callers that cannot allocate
device memory while running: its gradient, Hessian diagonal and FP64 value must match
pet_rdp's, on two calls in a row (the second call reuses the shared partial-sum array
that the first one left behind).  Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_rdp_static_matches_rdp_twice():
    from paper_2506_04976_gb300 import binding as pet
    lib = pet._lib
    lib.pet_rdp_static.restype = C.c_int
    lib.pet_rdp_static.argtypes = [C.POINTER(pet.RdpParams), C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_int, C.c_void_p]
    dev = "cuda:0"
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, shape in enumerate([(23, 37, 70), (9, 64, 45)]):
        gen = torch.Generator(device=dev).manual_seed(11 + call)
        x = torch.rand(shape, device=dev, generator=gen) * 3.0
        x[x < 0.3] = 0.0
        p = pet.rdp_params(shape, (2.0, 2.0, 2.8), 2.0, 1e-3, 0.7)
        ref_v, ref_g, ref_h = pet.rdp(x, (2.0, 2.0, 2.8), 2.0, 1e-3, 0.7)
        g = torch.empty_like(x)
        h = torch.empty_like(x)
        v = torch.full((), -1.0, device=dev, dtype=torch.float64)
        st = lib.pet_rdp_static(C.byref(p), C.c_void_p(x.data_ptr()), C.c_void_p(g.data_ptr()),
                                C.c_void_p(h.data_ptr()), C.c_void_p(v.data_ptr()), 0, stream)
        assert st == 0, pet.STATUS.get(st, st)
        torch.cuda.synchronize()
        rg, rh = ref_g.cpu().numpy(), ref_h.cpu().numpy()
        assert np.abs(g.cpu().numpy() - rg).max() <= 1e-5 * np.abs(rg).max()
        assert np.all(np.abs(h.cpu().numpy() - rh) <= 1e-5 * np.abs(rh) + 1e-7 * np.abs(rh).max())
        assert abs(float(v) - float(ref_v)) <= 1e-5 * abs(float(ref_v))
