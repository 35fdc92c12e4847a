"""Tall images whose height has a large prime factor: the column pass then runs Bluestein
convolutions long enough (about 2.2 x the height) that a one-column tile fills the shared
memory, and the pass reads its twiddles from global memory instead of a shared copy.

Checks: the amplitude sums A_o of such an image against the oracle's FP64 filter bank
(§II-A/B), and a smaller image bit-identical whether it shares a launch with the tall one
(which turns the shared twiddle copy off for the whole launch) or is extracted alone
(with the copy)."""
import numpy as np
import pytest

import oracle as O
import synth
from parity_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AMP_FLOOR = 2.5e-3   # as the other parity tests: 1e-4 relative down to 2.5e-3 of the maximum


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge
    ge.build()
    import paper_2303_00319_gb300 as p
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return p


def _amp_oracle(img):
    x = img.astype(np.float64)
    F = np.fft.fft2(x)
    r, th = O.frequency_grid(*x.shape)
    out = []
    for o in range(O.DEFAULT.n_orient):
        ang = O.angular(th, o)
        out.append(sum(np.abs(np.fft.ifft2(F * (O.radial(r, s) * ang))) for s in range(O.DEFAULT.n_scales)))
    return np.stack(out)


def test_tall_bluestein_height(pkg):
    dev = torch.device("cuda:0")
    tall = synth.make_pair(4001, 160, synth.pair_seed(13, 0), angle_deg=None).a    # 4001 is prime
    small = synth.make_pair(1031, 200, synth.pair_seed(13, 1), angle_deg=None).a  # 1031 is prime
    ctx = pkg.Context(pkg.default_params(max_keypoints=300), device=0)
    ft, fs = ctx.extract([torch.from_numpy(tall).to(dev), torch.from_numpy(small).to(dev)], debug=True)
    ctx.sync()
    got = ft.debug["amp"].cpu().numpy()
    exp = _amp_oracle(tall)
    for o in range(got.shape[0]):
        assert rel_err(got[o], exp[o], AMP_FLOOR) < 1e-4, o
    assert len(ft.host()["xy"]) > 0
    alone, = ctx.extract([torch.from_numpy(small).to(dev)], debug=True)
    ctx.sync()
    a, b = fs.host(), alone.host()
    for k in a:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    for name in ("amp", "er", "q", "an0", "moment", "mim", "noise_t"):
        assert np.array_equal(fs.debug[name].cpu().numpy(), alone.debug[name].cpu().numpy()), name
