"""The gather / permute kernel (TTGT reshaping and slice-gather) against
numpy index arithmetic: the result is a data movement, compared bit-exactly."""
import numpy as np
import pytest

from gpu_helpers import lib, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    need_gpu()
    hd = lib().Handle()
    yield hd
    hd.close()


def _ref_gather(src, dims, strides, offset):
    total = int(np.prod(dims)) if len(dims) else 1
    t = np.arange(total, dtype=np.int64)
    off = np.full(total, offset, dtype=np.int64)
    for d, s in zip(dims, strides):
        off += (t % d) * s
        t //= d
    return src[off]


@pytest.mark.parametrize("shape,perm", [((2,) * 10, None), ((4, 8, 16, 32), (3, 1, 0, 2)),
                                        ((33, 7, 65), (2, 0, 1)), ((2,) * 22, None),
                                        ((1024, 3, 130), (1, 2, 0)), ((5,), (0,))])
def test_permute_matches_numpy(h, shape, perm):
    q = lib()
    g = np.random.default_rng(len(shape))
    if perm is None:
        perm = tuple(g.permutation(len(shape)))
    src = (g.standard_normal(int(np.prod(shape))) + 1j * g.standard_normal(int(np.prod(shape)))).astype(np.complex64)
    fstr = np.cumprod((1,) + tuple(shape[:-1]))  # first-index-fastest strides of the source
    dims = [shape[p] for p in perm]
    strides = [int(fstr[p]) for p in perm]
    out = q.permute(h, torch.from_numpy(src).cuda(), dims, strides).cpu().numpy()
    assert np.array_equal(out, _ref_gather(src, dims, strides, 0))


def test_slice_gather_with_offset(h):
    """Fix one index of a (2, 8, 2, 16) tensor to 1 (a slice) while permuting."""
    q = lib()
    shape = (2, 8, 2, 16)
    g = np.random.default_rng(3)
    src = (g.standard_normal(512) + 1j * g.standard_normal(512)).astype(np.complex64)
    fstr = [1, 2, 16, 32]
    dims = [16, 2, 8]            # dims 3, 0, 1 of the source; dim 2 fixed to 1
    strides = [32, 1, 2]
    offset = 1 * 16
    out = q.permute(h, torch.from_numpy(src).cuda(), dims, strides, offset=offset).cpu().numpy()
    assert np.array_equal(out, _ref_gather(src, dims, strides, offset))
    del shape, fstr
