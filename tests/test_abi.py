"""The C-ABI library builds, loads and exports every entry point that
include/sigk.h declares; host-side argument checks reject bad calls before any
CUDA work (so these run without a GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sigk.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="needs nvcc to build libsigk.so")


def declared_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sigk_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libsigk():
    from paper_2006_14794_gb300 import sigk
    return sigk.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("sigk_pairs", "sigk_gram", "sigk_pairs_varlen", "sigk_pairs_backward",
                 "sigk_gram_backward", "sigk_workspace_bytes", "sigk_stream_status",
                 "sigk_strerror", "sigk_mmd2", "sigk_mmd2_backward"):
        assert must in names


def test_library_exports_every_declared_symbol(libsigk):
    from paper_2006_14794_gb300 import sigk
    for name in declared_symbols():
        assert hasattr(libsigk, name), name
    bound = {n for n, _, _ in sigk.SIGNATURES}
    assert set(declared_symbols()) == bound


def test_exported_symbols_are_c_linkage():
    from paper_2006_14794_gb300 import build
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sigk_[a-z0-9_]+)\b", out))
    assert set(declared_symbols()) <= exported


def test_version_and_strerror(libsigk):
    assert b"sm_103a" in libsigk.sigk_version()
    for s in range(6):
        assert libsigk.sigk_strerror(s)
    assert libsigk.sigk_strerror(99) == b"unknown status"


def test_argument_checks_need_no_gpu(libsigk):
    from paper_2006_14794_gb300 import sigk
    o = sigk.SigkOpts()
    P = ctypes.c_void_p(16)   # never dereferenced: the checks fail first
    # negative batch, zero channels, bad dtype, too-high dyadic order, reserved opts
    assert libsigk.sigk_pairs(P, P, -1, 4, 4, 2, 0, 0, ctypes.byref(o), P, None, 0, None) == sigk.SIGK_EINVAL
    assert libsigk.sigk_pairs(P, P, 3, 4, 4, 0, 0, 0, ctypes.byref(o), P, None, 0, None) == sigk.SIGK_EINVAL
    assert libsigk.sigk_pairs(P, P, 3, 4, 4, 2, 0, 7, ctypes.byref(o), P, None, 0, None) == sigk.SIGK_EINVAL
    assert libsigk.sigk_pairs(P, P, 3, 4, 4, 2, 9, 0, ctypes.byref(o), P, None, 0, None) == sigk.SIGK_EUNSUPPORTED
    assert libsigk.sigk_pairs(P, P, 3, 4, 4, 2, -1, 0, ctypes.byref(o), P, None, 0, None) == sigk.SIGK_EINVAL
    assert libsigk.sigk_pairs(None, P, 3, 4, 4, 2, 1, 0, None, P, None, 0, None) == sigk.SIGK_EINVAL
    o.reserved[0] = 1
    assert libsigk.sigk_gram(P, P, 2, 2, 4, 4, 2, 0, 0, ctypes.byref(o), P, None, 0, None) == sigk.SIGK_EINVAL
    o.reserved[0] = 0
    o.accumulate = 2
    assert libsigk.sigk_gram(P, P, 2, 2, 4, 4, 2, 0, 0, ctypes.byref(o), P, None, 0, None) == sigk.SIGK_EINVAL
    o.accumulate = 0
    # the scalar chain rule: sizes and dtype checked before any launch
    assert libsigk.sigk_scale_grad(P, P, P, -1, 0, None) == sigk.SIGK_EINVAL
    assert libsigk.sigk_scale_grad(P, P, P, 4, 5, None) == sigk.SIGK_EINVAL
    assert libsigk.sigk_scale_grad(None, P, P, 4, 0, None) == sigk.SIGK_EINVAL
    assert libsigk.sigk_scale_grad(None, None, None, 0, 0, None) == sigk.SIGK_OK
    o2 = sigk.SigkOpts(); o2.symmetric = 1
    assert libsigk.sigk_gram(P, P, 2, 3, 4, 4, 2, 0, 0, ctypes.byref(o2), P, None, 0, None) == sigk.SIGK_EINVAL
    # empty batches are valid and launch nothing
    assert libsigk.sigk_pairs(None, None, 0, 4, 4, 2, 0, 0, None, None, None, 0, None) == sigk.SIGK_OK
    assert libsigk.sigk_gram(None, None, 0, 5, 4, 4, 2, 0, 0, None, None, None, 0, None) == sigk.SIGK_OK


def test_value_and_grad_checks_need_no_gpu(libsigk):
    """sigk_gram_value_and_grad refuses, before any CUDA work, what only the
    two separate calls can do."""
    from paper_2006_14794_gb300 import sigk
    P = ctypes.c_void_p(16)   # never dereferenced: the checks fail first
    f = libsigk.sigk_gram_value_and_grad

    def call(Bx=2, By=2, L=4, M=4, d=2, lam=0, dtype=0, out=P, dY=P, **kw):
        o = sigk.SigkOpts()
        for k, v in kw.items():
            setattr(o, k, v)
        return f(P, P, P, Bx, By, L, M, d, lam, dtype, ctypes.byref(o), out, P, dY, None, 0, None)

    assert call(out=None) == sigk.SIGK_EINVAL
    assert call(symmetric=1) == sigk.SIGK_EINVAL              # symmetric: dY must be NULL
    assert call(symmetric=1, By=3, dY=None) == sigk.SIGK_EINVAL
    assert call(Bx=0) == sigk.SIGK_OK
    # outside the band form: the caller makes the two calls
    assert call(L=1) == sigk.SIGK_EUNSUPPORTED
    assert call(dtype=1) == sigk.SIGK_EUNSUPPORTED
    assert call(rec=sigk.REC_STRIP) == sigk.SIGK_EUNSUPPORTED
    assert call(static_kernel=sigk.KERNEL_RBF, sigma=1.0) == sigk.SIGK_EUNSUPPORTED
    assert call(L=600, M=600) == sigk.SIGK_EUNSUPPORTED        # 599 rows: no band


def test_schedule_options_are_checked(libsigk):
    from paper_2006_14794_gb300 import sigk
    P = ctypes.c_void_p(16)

    def call(dtype=0, **kw):
        o = sigk.SigkOpts()
        for k, v in kw.items():
            setattr(o, k, v)
        return libsigk.sigk_pairs(P, P, 3, 4, 4, 2, 0, dtype, ctypes.byref(o), P, None, 0, None)

    assert call(rows_per_lane=3) == sigk.SIGK_EINVAL
    assert call(rows_per_lane=32) == sigk.SIGK_EINVAL
    assert call(coef_path=4) == sigk.SIGK_EINVAL
    assert call(coef_path=-1) == sigk.SIGK_EINVAL
    assert call(rec=5) == sigk.SIGK_EINVAL
    # the tensor-core coefficient kernels are f32 only; the tcgen05 one takes d <= 64
    assert call(dtype=1, coef_path=2) == sigk.SIGK_EUNSUPPORTED
    assert call(dtype=1, coef_path=3) == sigk.SIGK_EUNSUPPORTED
    o = sigk.SigkOpts()
    o.coef_path = 3
    assert libsigk.sigk_pairs(P, P, 3, 4, 4, 65, 0, 0, ctypes.byref(o), P, None, 0, None) == sigk.SIGK_EUNSUPPORTED


def test_variant_options_are_checked(libsigk):
    from paper_2006_14794_gb300 import sigk
    P = ctypes.c_void_p(16)

    def call(**kw):
        o = sigk.SigkOpts()
        for k, v in kw.items():
            setattr(o, k, v)
        return libsigk.sigk_pairs(P, P, 3, 4, 4, 2, 0, 0, ctypes.byref(o), P, None, 0, None)

    assert call(scheme=2) == sigk.SIGK_EINVAL
    assert call(scheme=-1) == sigk.SIGK_EINVAL
    assert call(static_kernel=2) == sigk.SIGK_EINVAL
    # the RBF bandwidth must be positive and finite
    assert call(static_kernel=sigk.KERNEL_RBF, sigma=0.0) == sigk.SIGK_EINVAL
    assert call(static_kernel=sigk.KERNEL_RBF, sigma=-1.0) == sigk.SIGK_EINVAL
    assert call(static_kernel=sigk.KERNEL_RBF, sigma=float("nan")) == sigk.SIGK_EINVAL
    assert call(static_kernel=sigk.KERNEL_RBF, sigma=float("inf")) == sigk.SIGK_EINVAL
    # sigma is ignored for the linear kernel
    o = sigk.SigkOpts()
    o.scheme = sigk.SCHEME_IMPLICIT
    o.sigma = -3.0
    assert libsigk.sigk_pairs(None, None, 0, 4, 4, 2, 0, 0, ctypes.byref(o), None, None, 0, None) == sigk.SIGK_OK


def test_opts_layout_matches_the_header():
    from paper_2006_14794_gb300 import sigk
    txt = open(HEADER).read()
    body = txt[txt.index("typedef struct {"):txt.index("} sigk_opts;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(int|double)\s+([a-z_]+)(\[\d+\])?;", body)
    assert [f[1] for f in fields] == [f[0] for f in sigk.SigkOpts._fields_]
    assert ctypes.sizeof(sigk.SigkOpts) == 48


def test_forced_strip_schedule_asks_for_workspace(libsigk):
    from paper_2006_14794_gb300 import sigk
    auto, strip = sigk.SigkOpts(), sigk.SigkOpts()
    strip.rec = sigk.REC_STRIP
    # 64 pairs of 33-point paths in f64: the default one-block-per-pair sweep
    # needs no workspace, the strip path does
    n_auto = libsigk.sigk_workspace_bytes(sigk.OP_PAIRS, 64, 0, 33, 33, 4, 1, 1, ctypes.byref(auto))
    n_strip = libsigk.sigk_workspace_bytes(sigk.OP_PAIRS, 64, 0, 33, 33, 4, 1, 1, ctypes.byref(strip))
    assert n_auto == 0 and n_strip > 0
    # no strip instance above dyadic order 3: nothing to size
    assert libsigk.sigk_workspace_bytes(sigk.OP_PAIRS, 64, 0, 33, 33, 4, 4, 1, ctypes.byref(strip)) == 0


def test_band_schedule_is_f32_only(libsigk):
    from paper_2006_14794_gb300 import sigk
    o = sigk.SigkOpts()
    o.rec = sigk.REC_BAND
    P = ctypes.c_void_p(16)
    # f64 has no band form, for equal or uneven lengths
    assert libsigk.sigk_pairs(P, P, 3, 40, 40, 32, 1, 1, ctypes.byref(o), P, P, 1 << 30, None) == \
        sigk.SIGK_EUNSUPPORTED
    assert libsigk.sigk_pairs_varlen(P, P, P, P, 3, 32, 40, 1, 1, ctypes.byref(o), P, P, 1 << 30, None) == \
        sigk.SIGK_EUNSUPPORTED
    # uneven f32 lengths take the band form when the longest path fits its
    # largest band (1024 refined rows at dyadic order 1): a workspace, and the
    # refusal beyond
    assert libsigk.sigk_workspace_bytes(sigk.OP_PAIRS_VARLEN, 3, 0, 513, 513, 16, 1, 0, ctypes.byref(o)) > 0
    assert libsigk.sigk_workspace_bytes(sigk.OP_PAIRS_VARLEN, 3, 0, 514, 514, 16, 1, 0, ctypes.byref(o)) == 0
    assert libsigk.sigk_pairs_varlen(P, P, P, P, 3, 16, 514, 1, 0, ctypes.byref(o), P, P, 1 << 30, None) == \
        sigk.SIGK_EUNSUPPORTED
    # rec CHAIN (and AUTO) on uneven f32 lengths with d <= 16: the warp
    # stacks, whose workspace holds the increments of both sides (2 x pairs x
    # max_len rows of 16-byte channel quads) and the plan
    o.rec = sigk.REC_CHAIN
    ws_chain = libsigk.sigk_workspace_bytes(sigk.OP_PAIRS_VARLEN, 3, 0, 513, 513, 16, 1, 0, ctypes.byref(o))
    assert ws_chain > 2 * 3 * 513 * 64
    # AUTO takes the stacks for d <= 8 (the band form's contraction wins at d = 16)
    o.rec = sigk.REC_CHAIN
    ws8 = libsigk.sigk_workspace_bytes(sigk.OP_PAIRS_VARLEN, 3, 0, 513, 513, 8, 1, 0, ctypes.byref(o))
    o.rec = sigk.REC_AUTO
    assert libsigk.sigk_workspace_bytes(sigk.OP_PAIRS_VARLEN, 3, 0, 513, 513, 8, 1, 0, ctypes.byref(o)) == ws8
    assert libsigk.sigk_workspace_bytes(sigk.OP_PAIRS_VARLEN, 3, 0, 513, 513, 16, 1, 0, ctypes.byref(o)) != ws_chain
    o.rec = sigk.REC_BAND
    # the band workspace: a 256-byte header, then (pairs x macro-steps + 1)
    # slot rows of 32 x NG^2 floats.
    # 256-point paths at dyadic order 1: 510 refined rows -> 16 rows per lane,
    # NG = 8 coarse rows per lane, 512 padded columns -> 32 macro-steps per pair
    n = libsigk.sigk_workspace_bytes(sigk.OP_GRAM, 4, 5, 256, 256, 32, 1, 0, ctypes.byref(o))
    assert n == 256 + 4 * (20 * 32 + 1) * 32 * 64


def test_strip_backward_workspace_holds_no_per_cell_values(libsigk):
    """The strip adjoint reruns the forward backwards between checkpoints:
    its workspace for 8 long pairs (L = M = 4096, d = 64, dyadic order 1) is
    the coarse coefficient blocks and dk/dG (0.57 + 0.54 GB) and the strips'
    bottom rows and checkpoints (under 0.1 GB), not a value per refined cell
    (2.15 GB of sums on their own)."""
    from paper_2006_14794_gb300 import sigk
    o = sigk.SigkOpts()
    o.rec = sigk.REC_STRIP
    n = libsigk.sigk_workspace_bytes(sigk.OP_PAIRS_BACKWARD, 8, 0, 4096, 4096, 64, 1, 0, ctypes.byref(o))
    per_cell = 8 * 8190 * 8190 * 4
    assert 0 < n < 1.25e9 < per_cell


def test_surface_workspace_follows_the_schedule(libsigk):
    """The solution surface's workspace (no device needed): the chained sweep
    (f32, explicit scheme, linear kernel, d <= 16) keeps only the nodes' band
    layout, Tper/R + 1 slots of 32 NG^2 floats a pair; the band form adds the
    coefficient band before it."""
    from paper_2006_14794_gb300 import sigk
    o = sigk.SigkOpts()
    B, L, M, d, lam = 3, 128, 128, 8, 2
    # 127 coarse rows at order 2: 508 refined rows -> 16 rows a lane, NG = 4
    # coarse rows a lane; 508 refined columns padded to 512: Tper/R = 32
    chain = libsigk.sigk_workspace_bytes(sigk.OP_PAIRS_SURFACE, B, 0, L, M, d, lam, 0, ctypes.byref(o))
    assert chain == 256 + 4 * B * (32 + 1) * 32 * 4 * 4
    o.rec = sigk.REC_BAND
    band = libsigk.sigk_workspace_bytes(sigk.OP_PAIRS_SURFACE, B, 0, L, M, d, lam, 0, ctypes.byref(o))
    assert band > chain
    # the implicit scheme and d > 16 take the band form under AUTO too
    o.rec = sigk.REC_AUTO
    o.scheme = sigk.SCHEMES["implicit"]
    assert libsigk.sigk_workspace_bytes(sigk.OP_PAIRS_SURFACE, B, 0, L, M, d, lam, 0, ctypes.byref(o)) == band
    o.scheme = 0
    wide = libsigk.sigk_workspace_bytes(sigk.OP_PAIRS_SURFACE, B, 0, L, M, 17, lam, 0, ctypes.byref(o))
    o.rec = sigk.REC_BAND
    assert wide == libsigk.sigk_workspace_bytes(sigk.OP_PAIRS_SURFACE, B, 0, L, M, 17, lam, 0, ctypes.byref(o))
