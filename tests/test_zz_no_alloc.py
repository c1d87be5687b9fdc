"""Allocation-free RDP entry point (pet_rdp_static), for callers that cannot allocate
device memory while running (a service whose device memory is reserved at start-up, a
host framework that forbids allocations outside its own allocator).

Its gradient, Hessian diagonal and FP64 value must match pet_rdp's on two calls in a
row; the second call covers fewer stencil blocks than the first, so the shared partial-
sum array still holds the first call's extra partials, which the second must not read.
The stream-ordered allocator's high-water mark must not move during a call (pet_rdp's
own call moves it, which shows that the check can see an allocation).  Oversized images
are rejected before any launch, and val = NULL and value accumulation work.  Collected
last on purpose."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SPACING = (2.0, 2.0, 2.8)
# driver-API attributes of a memory pool (cuda.h): bytes in use now / highest since reset
_USED_MEM_CURRENT, _USED_MEM_HIGH = 7, 8


def _lib():
    from paper_2506_04976_gb300 import binding as pet
    lib = pet._lib
    lib.pet_rdp_static.restype = C.c_int
    lib.pet_rdp_static.argtypes = [C.POINTER(pet.RdpParams), C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_int, C.c_void_p]
    return pet, lib


class _Pool:
    """Default stream-ordered memory pool of device 0 (the pool cudaMallocAsync draws from)."""

    def __init__(self):
        self.cu = C.CDLL("libcuda.so.1")
        dev = C.c_int()
        assert self.cu.cuDeviceGet(C.byref(dev), 0) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def get(self, attr):
        v = C.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, C.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = C.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, _USED_MEM_HIGH, C.byref(zero)) == 0

    def peak_above_current(self):
        """Bytes by which the pool's use rose above its present level since reset_high."""
        return max(0, self.get(_USED_MEM_HIGH) - self.get(_USED_MEM_CURRENT))


def _static(lib, p, x, g, h, v, flags=0):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    return lib.pet_rdp_static(C.byref(p), ptr(x), ptr(g), ptr(h), ptr(v), flags, stream)


def _image(shape, seed):
    gen = torch.Generator(device=DEV).manual_seed(seed)
    x = torch.rand(shape, device=DEV, generator=gen) * 3.0
    x[x < 0.3] = 0.0
    return x


def test_rdp_static_matches_rdp_twice_without_allocating():
    pet, lib = _lib()
    pool = _Pool()
    # 240 stencil blocks of 32x8x4 voxels, then 30: the second call leaves 210 stale partials
    for call, shape in enumerate([(40, 64, 96), (9, 37, 45)]):
        x = _image(shape, 11 + call)
        p = pet.rdp_params(shape, SPACING, 2.0, 1e-3, 0.7)
        torch.cuda.synchronize()
        pool.reset_high()
        ref_v, ref_g, ref_h = pet.rdp(x, SPACING, 2.0, 1e-3, 0.7)
        torch.cuda.synchronize()
        assert pool.peak_above_current() > 0  # pet_rdp's partials came from the pool
        g = torch.empty_like(x)
        h = torch.empty_like(x)
        v = torch.full((), -1.0, device=DEV, dtype=torch.float64)
        torch.cuda.synchronize()
        pool.reset_high()
        st = _static(lib, p, x, g, h, v)
        torch.cuda.synchronize()
        assert st == 0, pet.STATUS.get(st, st)
        assert pool.peak_above_current() == 0
        rg, rh = ref_g.cpu().numpy(), ref_h.cpu().numpy()
        assert np.abs(g.cpu().numpy() - rg).max() <= 1e-5 * np.abs(rg).max()
        assert np.all(np.abs(h.cpu().numpy() - rh) <= 1e-5 * np.abs(rh) + 1e-7 * np.abs(rh).max())
        assert abs(float(v) - float(ref_v)) <= 1e-5 * abs(float(ref_v))


def test_rdp_static_without_value_and_with_value_accumulation():
    pet, lib = _lib()
    shape = (13, 30, 41)
    x = _image(shape, 5)
    p = pet.rdp_params(shape, SPACING, 2.0, 1e-3, 0.25)
    ref_v, ref_g, ref_h = pet.rdp(x, SPACING, 2.0, 1e-3, 0.25)
    g = torch.empty_like(x)
    h = torch.empty_like(x)
    assert _static(lib, p, x, g, h, None) == 0
    v = torch.full((), 2.5, device=DEV, dtype=torch.float64)
    assert _static(lib, p, x, None, None, v, pet.RDP_ACC_VAL) == 0  # v = 2.5 + 0.25 S
    torch.cuda.synchronize()
    rg, rh = ref_g.cpu().numpy(), ref_h.cpu().numpy()
    assert np.abs(g.cpu().numpy() - rg).max() <= 1e-5 * np.abs(rg).max()
    assert np.all(np.abs(h.cpu().numpy() - rh) <= 1e-5 * np.abs(rh) + 1e-7 * np.abs(rh).max())
    assert abs(float(v) - 2.5 - float(ref_v)) <= 1e-5 * abs(float(ref_v))


def test_rdp_static_rejects_images_beyond_its_partial_array():
    pet, lib = _lib()
    # 32 x 8 x (4 x 65537) voxels need 65537 stencil blocks, one more than the array holds;
    # the call returns before any launch, so the small buffers are never touched
    p = pet.rdp_params((4 * 65537, 8, 32), SPACING, 2.0, 1e-3, 1.0)
    x = torch.zeros(16, device=DEV)
    v = torch.zeros((), device=DEV, dtype=torch.float64)
    assert _static(lib, p, x, None, None, v) == 6  # PET_ERR_UNSUPPORTED
