"""lbm_flags_noalloc: node flags for callers that cannot allocate device
memory, checked through the C ABI against the flags of the ordinary entry
points (lbm_init / lbm_set_particles / lbm_step / lbm_get_fields) and against
the FP64 oracle's classification (Eq. (26), owner = argmax), on two calls in
a row with different particle sets.  Flags are integers, so the tolerance of
the flag tests applies: bit-exact.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

from tests import _helpers as H

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def pkg():
    from paper_2206_11634_gb300 import build as b
    b.build()
    import paper_2206_11634_gb300 as p
    return p


def _workloads():
    from paper_2206_11634_gb300 import workloads as W
    a = W.multi_particle(10, n=64, nz=64, storage="f32", seed_offset=7)
    rng = np.random.default_rng(5)
    cp, K = W.random_metaball(rng, 3, 3.0)
    b = W.empty_box(8, "f32", (1, 1, 0))
    b.update(nx=32, ny=24, nz=20)
    b["particles"] = [W._particle(cp, K, (0.4, 23.3, 9.8), q=(0.6, 0.2, 0.7, 0.33))]
    for wl in (a, b):
        H.fixed_mass(wl)
        for p in wl["particles"]:
            p["fixed"] = 1
    return [a, b]


def _oracle_flags(oracle_mod, wl):
    orc = H.make_oracle(oracle_mod, wl, n_sub=0)
    orc.set_particles(H.oracle_particles(oracle_mod, wl))
    return orc.classify() + 1


def _existing_flags(pkg, wl):
    lat = H.make_gpu(pkg, wl, n_sub=0)
    lat.set_particles(H.gpu_particles(pkg, wl))
    lat.step(1)
    return lat.flags().cpu().numpy(), lat.cfg


def _noalloc_flags(pkg, cfg, wl, out, stream):
    parts = H.gpu_particles(pkg, wl)
    arr = (pkg.LbmParticle * len(parts))(*parts)
    lib = pkg.load_library()
    rc = lib.lbm_flags_noalloc(C.byref(cfg), arr, len(parts), C.c_void_p(out.data_ptr()),
                               C.c_void_p(stream.cuda_stream))
    assert rc == 0, rc
    return (out.to(torch.int32) & 0xFFFF).cpu().numpy()


def test_noalloc_flags_match_existing_path_two_calls(pkg, oracle_mod):
    wls = [H.with_margin(oracle_mod, wl) for wl in _workloads()]
    expected = [_existing_flags(pkg, wl) for wl in wls]
    stream = torch.cuda.current_stream()
    outs = [torch.empty(tuple(reversed((wl["nx"], wl["ny"], wl["nz"]))), dtype=torch.int16, device="cuda")
            for wl in wls]
    torch.cuda.synchronize()
    # first call on the device: looks up the scratch array's address
    got0 = _noalloc_flags(pkg, expected[0][1], wls[0], outs[0], stream)
    assert np.array_equal(got0, expected[0][0])
    assert np.array_equal(got0, _oracle_flags(oracle_mod, wls[0]))
    assert (got0 > 0).sum() > 100
    # second call, another lattice and particle set: nothing of the first call
    # may leak through the shared scratch, and no device memory is taken
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    got1 = _noalloc_flags(pkg, expected[1][1], wls[1], outs[1], stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    assert np.array_equal(got1, expected[1][0])
    assert np.array_equal(got1, _oracle_flags(oracle_mod, wls[1]))
    assert (got1 > 0).sum() > 20


def test_noalloc_rejects_oversized_inputs(pkg):
    lib = pkg.load_library()
    out = torch.empty(8, dtype=torch.int16, device="cuda")
    big = pkg.make_config(512, 512, 512)
    p = pkg.make_particle([[0, 0, 0]], [4.0], (3.0, 3.0, 3.0))
    arr = (pkg.LbmParticle * 1)(p)
    assert lib.lbm_flags_noalloc(C.byref(big), arr, 1, C.c_void_p(out.data_ptr()), None) == -3
    small = pkg.make_config(16, 16, 16)
    many = (pkg.LbmParticle * 257)(*([p] * 257))
    assert lib.lbm_flags_noalloc(C.byref(small), many, 257, C.c_void_p(out.data_ptr()), None) == -3


def test_noalloc_brick_overflow_after_launch(pkg):
    """Twenty small particles inside one 32x4x2 brick: the binning finds more
    than 16 particles meeting it, which only the device can see, and the
    call reports LBM_ERR_CAPACITY after its kernels ran."""
    lib = pkg.load_library()
    cfg = pkg.make_config(64, 16, 8)
    out = torch.empty((8, 16, 64), dtype=torch.int16, device="cuda")
    parts = [pkg.make_particle([[0, 0, 0]], [0.3], (1.3 + 1.5 * k, 1.6, 0.4), fixed=1, mass=1.0,
                               inertia=np.eye(3)) for k in range(20)]
    arr = (pkg.LbmParticle * 20)(*parts)
    assert lib.lbm_flags_noalloc(C.byref(cfg), arr, 20, C.c_void_p(out.data_ptr()), None) == -3
    # the next call on the shared scratch starts clean
    one = (pkg.LbmParticle * 1)(pkg.make_particle([[0, 0, 0]], [4.0], (30.2, 8.3, 4.1), fixed=1, mass=1.0,
                                                  inertia=np.eye(3)))
    assert lib.lbm_flags_noalloc(C.byref(cfg), one, 1, C.c_void_p(out.data_ptr()), None) == 0
    assert int((out > 0).sum().item()) > 10
