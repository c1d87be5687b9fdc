"""Small scanner geometries for the oracle pins and the GPU parity tests."""
import numpy as np

from paper_2506_04976_gb300 import synth


def geom2d(n=8, nrad=12, nview=10, d=2.0, drad=2.0, rdet=100.0):
    g = dict(nx=n, ny=n, nz=1, dx=d, dy=d, dz=d, nrad=nrad, nview=nview, drad=drad,
             rdet=rdet, ntof=1, tof_sigma=1.0, tof_bin=1.0)
    g["z1"], g["z2"] = synth.planes_2d()
    return g


def geom3d(n=8, nz=5, nrad=12, nview=10, d=2.0, dz=2.5, drad=2.0, rdet=100.0, ntof=1,
           tof_sigma=8.0, tof_bin=10.0, oblique=True):
    nrings = (nz + 1) // 2
    pitch = 2 * dz
    g = dict(nx=n, ny=n, nz=nz, dx=d, dy=d, dz=dz, nrad=nrad, nview=nview, drad=drad,
             rdet=rdet, ntof=ntof, tof_sigma=tof_sigma, tof_bin=tof_bin)
    z1, z2 = synth.planes_span1(nrings, pitch)
    if not oblique:
        keep = z1 == z2
        z1, z2 = z1[keep], z2[keep]
    g["z1"], g["z2"] = z1, z2
    return g


def rand_img(g, seed, lo=0.0, hi=1.0):
    return synth.random_image_like(g, seed, lo, hi)


def rand_sino(g, seed, lo=0.5, hi=1.5):
    return synth.random_sinogram_like(g, seed, lo, hi)


def make_spec_problem(args):
    """(seed, spec) -> synth.make_problem(spec name, seed, **rest of spec); a module-level
    function so that spawned worker processes can build batch instances in parallel."""
    seed, spec = args
    sp = dict(spec)
    name = sp.pop("name")
    return synth.make_problem(name, seed, **sp)
