"""Pairs of uneven lengths in warp stacks (sigk_pairs_varlen, f32, rec CHAIN
and AUTO): the device plans pairs by the number of 64-coarse-row bands their
shorter path needs and deals them to chains; each chain's block sweeps its
pairs with one warp a band, the coefficients formed inside the sweep from
increments staged in shared memory.  Checked against the oracle element by
element: every stack height of each dyadic order, the largest height, single-
point paths, both orientations, chains of several pairs of different lengths,
pairs shorter than a warp's lane skew, channel counts of every instance, the
implicit scheme and a CUDA-graph replay on other lengths."""
import numpy as np
import pytest
import torch

import oracle
from paper_2006_14794_gb300 import inputs
from tests.gpu_util import need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    from paper_2006_14794_gb300 import sigk
    sigk.lib()


def S():
    from paper_2006_14794_gb300 import sigk
    return sigk


def _packed(seed, Ls, Ms, d, scale=1.0):
    rng = np.random.default_rng(seed)
    xs = [inputs.random_paths(int(rng.integers(1 << 30)), 1, int(L), d, scale=scale, time_channel=d > 1)[0]
          for L in Ls]
    ys = [inputs.random_paths(int(rng.integers(1 << 30)), 1, int(M), d, scale=scale, time_channel=d > 1)[0]
          for M in Ms]
    xo = np.concatenate([[0], np.cumsum(Ls)]).astype(np.int64)
    yo = np.concatenate([[0], np.cumsum(Ms)]).astype(np.int64)
    X32, X64 = inputs.f32(np.concatenate(xs))
    Y32, Y64 = inputs.f32(np.concatenate(ys))
    return X32, X64, xo, Y32, Y64, yo


def _run(X32, xo, Y32, yo, lam, max_len, rec=None, **kw):
    if rec is None:
        rec = S().REC_CHAIN
    return S().pairs_varlen(to_dev(X32), torch.as_tensor(xo).cuda(), to_dev(Y32), torch.as_tensor(yo).cuda(),
                            lam, max_len=max_len, rec=rec, check_status=True, **kw).cpu().numpy()


def _ref(X64, xo, Y64, yo, lam, **kw):
    return oracle.pairs_varlen(X64, xo, Y64, yo, lam, **kw)


TOP = 513   # longest shorter path a stack holds: 8 bands of 64 coarse rows


@pytest.mark.parametrize("lam", [0, 1, 2])
def test_every_stack_height_against_the_oracle(lam):
    rng = np.random.default_rng(300 + lam)
    # shorter paths in every band count 1..8, the band edges included
    edges = [2, 65, 66, 129, 130, 257, 258, 449, 450, TOP]
    Ls = list(rng.integers(2, TOP + 1, size=36)) + edges + [1, 2, 5, 3]
    Ms = list(rng.integers(2, TOP + 1, size=36)) + [TOP] * len(edges) + [7, 1, TOP, 2]
    Ls, Ms = np.array(Ls), np.array(Ms)
    # half the pairs with the longer path first (the rows refine the shorter one)
    sw = rng.random(len(Ls)) < 0.5
    Ls2, Ms2 = np.where(sw, Ms, Ls), np.where(sw, Ls, Ms)
    X32, X64, xo, Y32, Y64, yo = _packed(400 + lam, Ls2, Ms2, 3, scale=1.0)
    max_len = int(max(Ls2.max(), Ms2.max()))
    got = _run(X32, xo, Y32, yo, lam, max_len)
    ref = _ref(X64, xo, Y64, yo, lam)
    assert np.isfinite(got).all()
    assert rel_err(got, ref) <= 1e-5
    one = (Ls2 < 2) | (Ms2 < 2)
    assert np.all(got[one] == 1.0)


def test_auto_takes_the_stacks():
    # d <= 8: AUTO takes the stacks
    rng = np.random.default_rng(11)
    Ls = rng.integers(2, 300, size=40)
    Ms = rng.integers(2, 300, size=40)
    X32, X64, xo, Y32, Y64, yo = _packed(12, Ls, Ms, 8)
    a = _run(X32, xo, Y32, yo, 1, 300, rec=S().REC_AUTO)
    c = _run(X32, xo, Y32, yo, 1, 300)
    assert np.array_equal(a, c)
    assert rel_err(c, _ref(X64, xo, Y64, yo, 1)) <= 1e-5


def test_chains_of_several_pairs_of_different_lengths():
    # far more pairs of one height than the GPU holds chains: chains of many
    # pairs whose macro-step counts differ
    rng = np.random.default_rng(17)
    n = 6000
    Ls = rng.integers(130, 190, size=n)
    Ms = rng.integers(130, 330, size=n)
    X32, X64, xo, Y32, Y64, yo = _packed(18, Ls, Ms, 3, scale=1.0)
    got = _run(X32, xo, Y32, yo, 1, 330)
    # chaining adds nothing to a pair's arithmetic: the stacks and the band
    # form (coefficients from a separate contraction, its dot products summed
    # in another order) agree within the FP32 bar
    band = _run(X32, xo, Y32, yo, 1, 330, rec=S().REC_BAND)
    assert rel_err(got, band) <= 1e-5
    ref = _ref(X64, xo, Y64, yo, 1)
    # relative error with a floor of 0.25: 6000 random draws include kernels
    # far below 1, whose error is the absolute rounding of O(1) intermediates
    assert rel_err(got, ref, floor=0.25) <= 1e-5


@pytest.mark.parametrize("lam", [0, 1, 2])
def test_sixteen_channels_every_dyadic_order(lam):
    # the widest instance (four channel quads a column) at every dyadic order:
    # at order 0 a barrier period fills twice as many ring columns as the
    # producer warp has lanes
    rng = np.random.default_rng(80 + lam)
    Ls = rng.integers(2, 300, size=48)
    Ms = rng.integers(2, 300, size=48)
    X32, X64, xo, Y32, Y64, yo = _packed(90 + lam, Ls, Ms, 16)
    got = _run(X32, xo, Y32, yo, lam, 300)
    assert rel_err(got, _ref(X64, xo, Y64, yo, lam)) <= 1e-5


def test_pairs_shorter_than_the_lane_skew():
    # 2 .. 20 points: a pair lasts fewer macro-steps than the 32 lanes of a
    # warp are apart, so a warp holds several pairs at once
    rng = np.random.default_rng(21)
    Ls = rng.integers(2, 21, size=500)
    Ms = rng.integers(2, 21, size=500)
    X32, X64, xo, Y32, Y64, yo = _packed(22, Ls, Ms, 4)
    for lam in (0, 1, 2):
        got = _run(X32, xo, Y32, yo, lam, 20)
        assert rel_err(got, _ref(X64, xo, Y64, yo, lam)) <= 1e-5


@pytest.mark.parametrize("d", [1, 3, 5, 8, 13, 16])
def test_channel_counts(d):
    # every channel-quad instance (1, 2, 4 quads), d not a multiple of 4 too
    rng = np.random.default_rng(30 + d)
    Ls = rng.integers(2, 400, size=24)
    Ms = rng.integers(2, 400, size=24)
    X32, X64, xo, Y32, Y64, yo = _packed(40 + d, Ls, Ms, d)
    got = _run(X32, xo, Y32, yo, 1, 400)
    assert rel_err(got, _ref(X64, xo, Y64, yo, 1)) <= 1e-5


def test_wide_paths_take_the_other_forms():
    # d > 16 has no stack instance: CHAIN takes the strip path, AUTO the band form
    rng = np.random.default_rng(50)
    Ls = rng.integers(2, 50, size=4)
    X32, X64, xo, Y32, Y64, yo = _packed(51, Ls, Ls, 17)
    ref = _ref(X64, xo, Y64, yo, 1)
    for rec in (S().REC_CHAIN, S().REC_AUTO):
        assert rel_err(_run(X32, xo, Y32, yo, 1, 50, rec=rec), ref) <= 1e-5


def test_implicit_scheme():
    rng = np.random.default_rng(55)
    Ls = rng.integers(2, 300, size=30)
    Ms = rng.integers(2, 300, size=30)
    X32, X64, xo, Y32, Y64, yo = _packed(56, Ls, Ms, 4)
    v = S().Variant(scheme="implicit")
    got = _run(X32, xo, Y32, yo, 1, 300, variant=v)
    assert rel_err(got, _ref(X64, xo, Y64, yo, 1, scheme="implicit")) <= 1e-5


def test_graph_replay_with_other_lengths():
    rng = np.random.default_rng(70)
    n = 300
    Ls = rng.integers(2, 513, size=n)
    Ms = rng.integers(2, 513, size=n)
    a = _packed(71, Ls, Ms, 16)
    # the second batch: the lengths dealt to other pairs, so the point rows,
    # and with them the static buffers' shapes, stay the same
    b = _packed(72, rng.permutation(Ls), rng.permutation(Ms), 16)
    dev = [to_dev(a[0]), torch.as_tensor(a[2]).cuda(), to_dev(a[3]), torch.as_tensor(a[5]).cuda()]
    g = S().graphed(S().pairs_varlen, *dev, 1, max_len=512, rec=S().REC_CHAIN)
    for X32, X64, xo, Y32, Y64, yo in (a, b, a):
        out = g(to_dev(X32), torch.as_tensor(xo).cuda(), to_dev(Y32), torch.as_tensor(yo).cuda())
        torch.cuda.synchronize()
        assert rel_err(out.cpu().numpy(), _ref(X64, xo, Y64, yo, 1)) <= 1e-5
