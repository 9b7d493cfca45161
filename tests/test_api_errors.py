"""Host-side checks of the C ABI that need no GPU: the library loads and exports every
function include/iugkp.h declares, and invalid input is rejected with IUGKP_EINVAL and a
message before any CUDA call (failure detection without a device fault)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_09465_gb300 import build as B
    B.build()
    from paper_2506_09465_gb300 import _lib as L
    return L


def test_library_exports_every_declared_symbol(lib):
    header = open(os.path.join(ROOT, "include", "iugkp.h")).read()
    declared = set(re.findall(r"\b(iugkp_[a-z0-9_]+)\s*\(", header))
    assert "iugkp_sweep" in declared and "iugkp_diffusion_solve_noalloc" in declared
    L = lib.load()
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared == set(lib.SIGNATURES), declared ^ set(lib.SIGNATURES)


def _create(lib, dim=2, n=(4, 3), tau=None, wall=None, src=None, nb=1, **opt):
    L = lib.load()
    nc = int(np.prod(n))
    tau = np.full((nb, nc), 0.5) if tau is None else np.asarray(tau, dtype=np.float64)
    wall = np.zeros(2 * dim) if wall is None else np.asarray(wall, dtype=np.float64)
    C = np.ones(nb)
    v = np.ones(nb)
    nn = list(n) + [1] * (3 - len(n))
    grid = lib.Grid(dim, nn[0], nn[1], nn[2], 1.0, 1.0, 1.0)
    bands = lib.Bands(nb, C.ctypes.data, v.ctypes.data)
    o = lib.default_options(**opt)
    ctx = ctypes.c_void_p()
    st = L.iugkp_create(ctypes.byref(grid), tau.ctypes.data, ctypes.byref(bands), wall.ctypes.data,
                        None if src is None else np.asarray(src, dtype=np.float64).ctypes.data, ctypes.byref(o),
                        ctypes.byref(ctx))
    return st, L.iugkp_last_error(None).decode()


@pytest.mark.parametrize("case,kw,needle", [
    ("tau_zero", dict(tau=np.zeros((1, 12))), "tau"),
    ("tau_nan", dict(tau=np.full((1, 12), np.nan)), "tau"),
    ("wall_inf", dict(wall=[0, 0, np.inf, 0]), "wall"),
    ("source_nan", dict(src=np.full(12, np.nan)), "source"),
    ("bad_dim", dict(dim=4), "grid"),
    ("zero_cells", dict(n=(0, 3)), "grid"),
    ("too_few_particles", dict(nb=2, tau=np.full((2, 12), 0.5), particles_per_cell=1), "particles"),
    ("bad_precision", dict(precision=7), "precision"),
    ("bad_tally", dict(tally=3), "tally"),
    ("k32_needs_fp32", dict(tally=2, precision=0), "tally"),
    ("bad_refill", dict(refill_lanes=40), "refill"),
    ("bad_grab", dict(warp_grab=-1), "warp_grab"),
    ("bad_walk", dict(walk_k=5000), "walk_k"),
    ("bad_cg", dict(cg_rtol=0.0), "cg"),
])
def test_create_rejects_invalid_input(lib, case, kw, needle):
    st, msg = _create(lib, **kw)
    assert st == 1, (case, st, msg)
    assert needle in msg, (case, msg)


def test_null_arguments_rejected(lib):
    L = lib.load()
    assert L.iugkp_create(None, None, None, None, None, None, None) == 1
    assert L.iugkp_sweep(None, None, 0, None, None, None, None, None, None) == 1
    assert L.iugkp_solve_steady(None, None, 1e-8, 10, None, None, None) == 1
    assert L.iugkp_adjoint(None, None, None, 1e-8, 10, None, None, None, None) == 1
    assert L.iugkp_autotune(None, None, 0, 0, None, None) == 1
    assert L.iugkp_average(None, None, 1, 0, None, None, None, None) == 1
    assert L.iugkp_persistent_reset(None, None) == 1
    assert L.iugkp_persistent_step(None, None, 0, None, None, None, None, None, None) == 1
    L.iugkp_destroy(None)  # no-op


def test_noalloc_rejects_before_any_device_work(lib):
    L = lib.load()
    g = lib.Grid(3, 64, 64, 32, 1.0, 1.0, 1.0)  # 131072 cells > the static limit
    st = L.iugkp_diffusion_solve_noalloc(ctypes.byref(g), 8, 1.0, 8, 8, 1e-6, 10, None, None)
    assert st == 1
    assert "IUGKP_NOALLOC_MAX_CELLS" in L.iugkp_last_error(None).decode()


def test_default_options(lib):
    o = lib.default_options()
    assert o.precision == lib.TRACK_FP32 and o.tally == lib.TALLY_STAGED and o.draws == lib.DRAWS_FROZEN
    assert o.newton == 1 and o.use_graphs == 1 and o.particles_per_cell == 1024
    assert o.warp_grab == 0 and o.walk_k == 0 and o.refill_lanes == 0
    with pytest.raises(AttributeError):
        lib.default_options(no_such_option=1)


def test_fp32_uniform_from_mantissa_bits_is_exact():
    # The fast path forms its FP32 uniforms as (1 + m 2^-23) - (1 - 2^-24) from the top 23
    # bits m of a Philox word; this equals (2m + 1) 2^-24, the value the oracle and the FP64
    # path use, for every m (IEEE round-to-nearest FP32, as on the GPU).
    m = np.arange(1 << 23, dtype=np.uint32)
    fast = (0x3F800000 | m).view(np.float32) - np.float32(0.99999994)
    ref = ((2 * m.astype(np.float64) + 1) / 16777216.0).astype(np.float32)
    assert np.float32(0.99999994) == np.float32(1.0 - 2.0 ** -24)
    assert np.array_equal(fast, ref) and np.array_equal(ref.astype(np.float64), (2 * m.astype(np.float64) + 1) / 16777216.0)


def test_integer_division_by_multiply_high_is_exact():
    # The fast path divides particle and cell indices n < 2^31 by d >= 1 as
    # q = umulhi(n, M) + [n - q d >= d] with M = floor((2^32 - 1) / d); checked here with
    # exact integers on divisors and indices that include the extremes and exact multiples.
    rng = np.random.default_rng(0)
    ds = [1, 2, 3, 7, 100, 101, 128, 255, 256, 1023, 16384, 65535, 65536, 1000003, 2 ** 30, 2 ** 31 - 1]
    ds += [int(x) for x in rng.integers(1, 2 ** 31, 40)]
    for d in ds:
        M = (2 ** 32 - 1) // d
        ns = {0, 1, d - 1, d, d + 1, 2 ** 31 - 1, (2 ** 31 - 1) // d * d, (2 ** 31 - 1) // d * d - 1}
        ns |= {int(x) for x in rng.integers(0, 2 ** 31, 200)}
        for n in ns:
            if n < 0 or n >= 2 ** 31:
                continue
            q = (n * M) >> 32
            q += 1 if n - q * d >= d else 0
            assert q == n // d, (n, d)
