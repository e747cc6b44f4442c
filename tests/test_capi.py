"""CPU-side checks of the C ABI: the library loads, exports every function that
include/sch.h declares, and rejects invalid arguments on the host before any
CUDA call (these tests need no GPU)."""
import ctypes as ct
import os
import re

import pytest

from tests.helpers import noise_poly_expected

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:int|size_t)\s+(\w+)\s*\(", src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2402_06927_gb300 import build
    build.build()
    from paper_2402_06927_gb300 import _lib
    return _lib.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2402_06927_gb300 import _lib
    bound = set(_lib.SIGNATURES) | set(_lib.RESTYPES)
    assert set(declared_functions()) <= bound


def _params(**kw):
    from paper_2402_06927_gb300._lib import SchParams, SCH_F64
    p = SchParams()
    p.L, p.n, p.alpha, p.mu, p.dt, p.K = 40.0, 256, 1.0, 0.02, 0.025, 4
    p.amps[0] = p.amps[1] = 0.05
    p.M, p.sigma, p.tol, p.max_iter, p.dtype = 32, 0.05, 1e-13, 50, SCH_F64
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("kw,rc", [({}, 0), ({"n": 100, "M": 25}, -6), ({"n": 256 * 4}, 0), ({"K": 3}, -1),
                                   ({"K": 66}, -1), ({"M": 33}, -1), ({"sigma": 0.0}, -1), ({"dt": -1.0}, -1),
                                   ({"dtype": 5}, -1), ({"n": 8192}, -6), ({"max_iter": 0}, -1),
                                   # kernel layouts: the warp-per-particle layout takes float fields, the
                                   # explicit-advection solver and n = 256, 512 or 1024 only; the warp-group
                                   # layouts float fields, explicit advection, the mode expansion and
                                   # n = 2048 or 4096, and n = 1024 with 16 nodes a lane
                                   ({"layout": 5}, -1), ({"layout": 2}, -6), ({"layout": 1}, 0),
                                   ({"layout": 2, "dtype": 1}, 0), ({"layout": 2, "dtype": 1, "n": 1024, "M": 64}, 0),
                                   ({"layout": 2, "dtype": 1, "solver": 1}, -6),
                                   ({"layout": 2, "dtype": 1, "n": 2048, "M": 64}, -6),
                                   ({"layout": 3}, -6), ({"layout": 3, "dtype": 1}, -6),
                                   ({"layout": 3, "dtype": 1, "n": 4096, "M": 128}, 0),
                                   ({"layout": 4, "dtype": 1, "n": 4096, "M": 128}, 0),
                                   ({"layout": 4, "dtype": 1, "n": 2048, "M": 64}, 0),
                                   ({"layout": 4, "dtype": 1, "n": 1024, "M": 64}, 0),
                                   ({"layout": 3, "dtype": 1, "n": 1024, "M": 64}, -6),
                                   ({"layout": 4, "dtype": 1, "n": 512, "M": 64}, -6),
                                   ({"dtype": 1, "n": 2048, "M": 64}, 0), ({"dtype": 1, "n": 4096, "M": 128}, 0),
                                   ({"layout": 3, "dtype": 1, "n": 4096, "M": 128, "solver": 1}, -6),
                                   ({"layout": 3, "dtype": 1, "n": 4096, "M": 128, "noise": 1, "kappa": 1.0, "eta": 1.0,
                                     "matern_k": 3}, -6)])
def test_create_validates(lib, kw, rc):
    p = _params(**kw)
    h = ct.c_void_p()
    got = lib.sch_create(ct.byref(p), ct.byref(h))
    assert got == rc
    if got == 0:
        ea32 = p.dtype == 1 and p.solver != 1
        auto = 2 if (ea32 and p.n in (256, 512, 1024)) else 3 if (ea32 and p.n in (2048, 4096)) else 1
        want = kw.get("layout", 0) or auto
        assert lib.sch_layout(h) == want
        assert lib.sch_destroy(h) == 0


def test_host_argument_errors_need_no_gpu(lib):
    p = _params()
    h = ct.c_void_p()
    assert lib.sch_create(ct.byref(p), ct.byref(h)) == 0
    # missing pointers are rejected before any launch
    assert lib.sch_ensemble_step(h, 4, 5, None, None, None, None, None, None, None, None, None, None, None) == -1
    assert lib.sch_ensemble_step(h, -1, 5, None, None, None, None, None, None, None, None, None, None, None) == -1
    # empty ensembles are a no-op
    assert lib.sch_ensemble_step(h, 0, 5, None, None, None, None, None, None, None, None, None, None, None) == 0
    assert lib.pf_temper(0, None, None, 0.0, 1.0, None, None, None) == -1
    assert lib.pf_temper_halving(0, None, None, 0.0, 1.0, None, None, None) == -1
    # device-gated stage entry points: missing device scalars are argument errors
    assert lib.pf_temper_dev(4, ct.c_void_p(16), None, None, 1.0, 0, ct.c_void_p(16), ct.c_void_p(16), None) == -1
    assert lib.pf_temper_dev(4, ct.c_void_p(16), None, ct.c_void_p(16), 1.0, 7, ct.c_void_p(16), ct.c_void_p(16),
                             None) == -1
    assert lib.pf_resample_gated(4, ct.c_void_p(16), 0, 0, None, ct.c_void_p(16), None) == -1
    assert lib.pf_temper(4, ct.c_void_p(16), None, 1.0, 1.0, ct.c_void_p(16), ct.c_void_p(16), None) == -1
    assert lib.pf_resample(9000, ct.c_void_p(16), 0, 0, ct.c_void_p(16), 0, None, None, None, 0, None) == -1
    arr = (ct.c_void_p * 1)(16)
    rows = (ct.c_size_t * 1)(32)
    assert lib.pf_resample(4, ct.c_void_p(16), 0, 0, ct.c_void_p(16), 1, arr, rows, None, 0, None) == -5
    assert lib.pf_gather_rows(4, ct.c_void_p(16), ct.c_void_p(16), ct.c_void_p(32), 6, None) == -1
    assert lib.pf_jitter(h, 4, 5, 1, 0.5, 1.5, 0, 0, *([None] * 12)) == -1
    assert lib.pf_resample_workspace_bytes(10, 48) == 480
    # MALA: step size, temperature and pointers checked on the host; an empty ensemble is a no-op
    P16 = ct.c_void_p(16)
    assert lib.pf_mala_propose(h, 4, 5, 0.5, 0.0, 0, 0, 0, P16, None, P16, P16, None) == -1
    assert lib.pf_mala_propose(h, 4, 5, 1.5, 0.1, 0, 0, 0, P16, None, P16, P16, None) == -1
    assert lib.pf_mala_propose(h, 4, 5, 0.5, 0.1, 0, 0, -1, P16, None, P16, P16, None) == -1
    assert lib.pf_mala_propose(h, 4, 5, 0.5, 0.1, 0, 0, 0, None, None, P16, P16, None) == -1
    assert lib.pf_mala_propose(h, 0, 5, 0.5, 0.1, 0, 0, 0, None, None, None, None, None) == 0
    assert lib.pf_mala_accept(h, 4, 5, 0.5, 0.1, 0, 0, 0, P16, P16, None, P16, None, P16, P16, None, None) == -1
    assert lib.pf_mala_accept(h, 0, 5, 0.5, 0.1, 0, 0, 0, *([None] * 9)) == 0
    # the Exp 1 ensemble
    assert lib.sch_prior_exp1(h, 4, 0, -1, P16, P16, None) == -1
    assert lib.sch_prior_exp1(h, 4, 0, 0, None, P16, None) == -1
    assert lib.sch_prior_exp1(h, 0, 0, 0, None, None, None) == 0
    assert lib.sch_prior_exp1(None, 4, 0, 0, P16, P16, None) == -1
    # gated stages: a negative jitter count is an argument error (zero jitters nothing)
    bufs = (ct.c_void_p * 7)(*([16] * 6 + [None]))
    assert lib.pf_gated_stages(h, 4, 5, 1, 0, 1.0, 0, 0.9, -1, 0, 0, P16, bufs, bufs, P16, P16, P16, P16, None, None,
                               None, None, None) == -1
    assert lib.sch_destroy(h) == 0


@pytest.mark.parametrize("kw,rc", [({"noise": 1}, 0), ({"noise": 1, "dtype": 1}, 0),
                                   ({"noise": 2}, -1), ({"noise": 1, "kappa": 0.0}, -1),
                                   ({"noise": 1, "eta": -1.0}, -1), ({"noise": 1, "matern_k": 0}, -1),
                                   ({"noise": 1, "matern_k": 9}, -1),
                                   # Matern noise: each precision's default solver only; the warp
                                   # layout where it fits (FP32, n = 256, 512 or 1024)
                                   ({"noise": 1, "dtype": 1, "layout": 2}, 0), ({"noise": 1, "layout": 2}, -6),
                                   ({"noise": 1, "solver": 2}, -6), ({"noise": 1, "dtype": 1, "solver": 1}, -6)])
def test_create_validates_matern(lib, kw, rc):
    base = {"kappa": 1.0, "eta": 0.2, "matern_k": 3}
    base.update(kw)
    p = _params(**base)
    h = ct.c_void_p()
    got = lib.sch_create(ct.byref(p), ct.byref(h))
    assert got == rc
    if got == 0:
        # one Brownian motion per cell; the warp layout wherever it fits (FP32 here, n = 256)
        assert lib.sch_noise_dim(h) == p.n
        assert lib.sch_layout(h) == (2 if p.layout == 2 or (p.layout == 0 and p.dtype == 1) else 1)
        # the entry points built on the adjoint check their arguments; the nudging workspace holds
        # the optimiser's vectors, 17 of nsteps x n doubles, besides the adjoint's region
        assert lib.pf_nudge(h, 1, 5, 0, 10, 1e-6, 1, 0, 0, None, None, None, None, None, None, None, None, 0,
                            None) == -1
        assert lib.pf_nudge_workspace_bytes(h, 1, 5, 1) >= 17 * 5 * p.n * 8 + lib.sch_adjoint_workspace_bytes(h, 1, 5, 1)
        assert lib.sch_adjoint_window(h, 1, 5, 1, None, None, None, None, None, None, None, None, None, None, None,
                                      0, None) == -1
        assert lib.pf_mala_propose(h, 1, 5, 0.5, 0.1, 0, 0, 0, None, None, None, None, None) == -1
        assert lib.sch_destroy(h) == 0


def test_noise_dim_of_the_mode_expansion(lib):
    p = _params()
    h = ct.c_void_p()
    assert lib.sch_create(ct.byref(p), ct.byref(h)) == 0
    assert lib.sch_noise_dim(h) == 4
    assert lib.sch_noise_dim(None) == -1
    assert lib.sch_destroy(h) == 0


def test_adjoint_workspace_sizes(lib):
    # per particle: ceil(nsteps / ckpt) checkpoints and 2 (ckpt + 1) segment states of n reals;
    # the binding's default interval is the whole window (one checkpoint, every state kept)
    from paper_2402_06927_gb300.api import _ckpt
    p = _params()          # FP64, n = 256
    h = ct.c_void_p()
    assert lib.sch_create(ct.byref(p), ct.byref(h)) == 0
    assert lib.sch_adjoint_workspace_bytes(h, 3, 20, 5) == 3 * (4 + 12) * 256 * 8
    assert lib.sch_adjoint_workspace_bytes(h, 3, 20, 20) == 3 * (1 + 42) * 256 * 8
    assert lib.sch_adjoint_workspace_bytes(h, 3, 20, 0) == 0
    assert lib.sch_adjoint_workspace_bytes(h, 0, 20, 5) == 0
    assert _ckpt(None, 20) == 20 and _ckpt(5, 20) == 5
    assert lib.sch_destroy(h) == 0


def test_jitter_workspace_size_and_checks(lib):
    # the warm-start workspace: N Ns n floats for the warp-group layouts, none elsewhere;
    # a misaligned pointer is refused, NULL clears it (no device memory is touched here)
    from paper_2402_06927_gb300._lib import SCH_F32
    for kw, per in [({"layout": 3, "dtype": SCH_F32, "n": 4096, "M": 128}, 4096),
                    ({"layout": 4, "dtype": SCH_F32, "n": 1024, "M": 64}, 1024),
                    ({"layout": 2, "dtype": SCH_F32, "n": 1024, "M": 64}, 0),
                    ({"layout": 1}, 0)]:
        p = _params(**kw)
        h = ct.c_void_p()
        assert lib.sch_create(ct.byref(p), ct.byref(h)) == 0
        assert lib.sch_jitter_workspace_bytes(h, 64, 10) == 64 * 10 * per * 4
        assert lib.sch_jitter_workspace_bytes(h, 0, 10) == 0
        assert lib.sch_set_jitter_workspace(h, ct.c_void_p(0x1000008), 1 << 20) == -1   # 8-byte aligned only
        assert lib.sch_set_jitter_workspace(h, None, 0) == 0
        assert lib.sch_destroy(h) == 0
    assert lib.sch_set_jitter_workspace(None, None, 0) == -1


def test_noise_form_choice(lib):
    # the lane-centred noise sums: in the warp-group layouts polynomial fits where they are
    # accurate to 2^-30 and cheaper, the tables elsewhere; the one-warp layout always takes the
    # tables (at K = 10, n = 1024 the fits would qualify); neither for the CTA layout or the
    # Matern noise
    from paper_2402_06927_gb300._lib import SCH_F32
    cases = [(4096, 32, 3, 16, True), (4096, 64, 3, 16, False), (4096, 48, 3, 16, False),
             (2048, 32, 3, 16, False), (2048, 32, 4, 8, True), (1024, 32, 4, 8, False),
             (1024, 8, 2, 16, False), (1024, 10, 2, 16, True), (1024, 32, 2, 16, False),
             (4096, 4, 3, 16, False), (256, 4, 2, 4, False)]
    for n, K, layout, H, fits in cases:
        assert fits == noise_poly_expected(n, H, K // 2), (n, K, layout)
        want = 2 if (fits and layout != 2) else 1
        p = _params(n=n, M=64, K=K, dtype=SCH_F32, layout=layout, tol=1e-6)
        for j in range(K // 2):
            p.amps[j] = 0.05
        h = ct.c_void_p()
        assert lib.sch_create(ct.byref(p), ct.byref(h)) == 0, (n, K, layout)
        assert lib.sch_noise_form(h) == want, (n, K, layout)
        assert lib.sch_destroy(h) == 0
    for kw in [{"layout": 1}, {"noise": 1, "kappa": 1.0, "eta": 0.2, "matern_k": 3, "n": 1024, "M": 64,
                                "dtype": SCH_F32, "layout": 2}]:
        p = _params(**kw)
        h = ct.c_void_p()
        assert lib.sch_create(ct.byref(p), ct.byref(h)) == 0
        assert lib.sch_noise_form(h) == 0
        assert lib.sch_destroy(h) == 0
    assert lib.sch_noise_form(None) == -1


def test_matern_layout_choice(lib):
    # SCH_LAYOUT_AUTO: one warp per particle for FP32 fields at n = 256, 512, 1024 with either
    # noise model, the CTA layout at other sizes and for FP64; SCH_LAYOUT_CTA always honoured
    for n, dtype, layout, want in [(512, 1, 0, 2), (1024, 1, 0, 2), (2048, 1, 0, 1), (1024, 0, 0, 1),
                                   (1024, 1, 1, 1), (1024, 1, 2, 2)]:
        p = _params(noise=1, kappa=1.0, eta=0.2, matern_k=3, n=n, M=64, dtype=dtype, layout=layout)
        h = ct.c_void_p()
        assert lib.sch_create(ct.byref(p), ct.byref(h)) == 0, (n, dtype, layout)
        assert lib.sch_layout(h) == want, (n, dtype, layout)
        assert lib.sch_noise_dim(h) == n
        assert lib.sch_destroy(h) == 0
