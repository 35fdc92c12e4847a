"""Launch groups of mixed image sizes (one launch per stage over a per-image size table)
against groups of one size (RIFT2_FLAG_SIZE_GROUPS): every output of every image is
bit-identical, each result lands in its own caller buffer although the library orders the
images by size, and the mixed groups enqueue far fewer kernels.

The sizes mix every transform path: power-of-two sides (register-tiled kernels, run by run
inside the mixed group), 13-smooth sides (shared-memory transforms), sides with a prime
factor above 13 (Bluestein), a width whose rows take the split row pass, and images
smaller than the patch (no keypoints)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [(384, 640), (1024, 512), (257, 263), (640, 384), (512, 1024), (150, 2053),
         (384, 640), (80, 90), (1536, 256), (211, 331), (256, 256), (160, 900)]


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge
    ge.build()
    import paper_2303_00319_gb300 as p
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return p


@pytest.fixture(scope="module")
def images():
    dev = torch.device("cuda:0")
    return [torch.from_numpy(synth.make_pair(h, w, synth.pair_seed(7, i), angle_deg=None).a).to(dev)
            for i, (h, w) in enumerate(SIZES)]


def _run(pkg, images, flags, debug=False, budget=None, max_kp=300):
    kw = {} if budget is None else {"hbm_budget": budget}
    ctx = pkg.Context(pkg.default_params(max_keypoints=max_kp, flags=flags), device=0, **kw)
    ctx.extract(images, debug=debug)   # creates the plans and tables of every size
    ctx.sync()
    before = ctx.launch_count()
    feats = ctx.extract(images, debug=debug)
    ctx.sync()
    launches = ctx.launch_count() - before   # kernels of one call with the plans in place
    out = []
    for f in feats:
        h = f.host()
        if debug:
            for name, t in f.debug.items():
                h["map_" + name] = t.cpu().numpy()
        out.append(h)
    return out, launches, ctx


def _assert_same(a, b, what):
    assert len(a) == len(b)
    for i, (x, y) in enumerate(zip(a, b)):
        for k in x:
            assert np.array_equal(np.asarray(x[k]), np.asarray(y[k])), f"{what}: image {i} {SIZES[i]} field {k}"


@pytest.mark.parametrize("extra", [0, "corners", "spatial", "ring"])
def test_mixed_groups_equal_size_groups(pkg, images, extra):
    flags = {0: 0, "corners": pkg.FLAG_CORNERS, "spatial": pkg.FLAG_SPATIAL_NORM,
             "ring": pkg.FLAG_RIFT_RING}[extra]
    mixed, n_mixed, _ = _run(pkg, images, flags)
    same, n_same, _ = _run(pkg, images, flags | pkg.FLAG_SIZE_GROUPS)
    _assert_same(mixed, same, f"flags {flags:#x}")
    for (h, w), r in zip(SIZES, mixed):
        if min(h, w) < 102:
            assert len(r["xy"]) == 0 and len(r["desc"]) == 0
        else:
            assert len(r["xy"]) > 0
    # 11 distinct sizes: the size groups enqueue every stage once per size
    assert n_mixed * 3 < n_same, (n_mixed, n_same)


def test_mixed_groups_maps_and_order(pkg, images):
    """The optional maps too, and each image's outputs in its own buffer: image i of the
    mixed call equals image i extracted alone."""
    mixed, _, _ = _run(pkg, images, 0, debug=True)
    for i in (0, 2, 5, 7, 9):
        alone, _, _ = _run(pkg, [images[i]], 0, debug=True)
        _assert_same([mixed[i]], alone, f"image {i} alone")


def test_mixed_group_split_by_budget(pkg, images):
    """A budget that holds only part of the group splits it; the results stay the same."""
    full, _, ctx = _run(pkg, images, 0)
    sizes = [tuple(im.shape) for im in images]
    need = ctx.workspace_bytes(sizes)
    half, _, _ = _run(pkg, images, 0, budget=need // 3)
    _assert_same(full, half, "budget split")


def test_workspace_figure_covers_the_mixed_group(pkg, images):
    """rift2_workspace_bytes applies the grouping rift2_extract forms: a context whose
    budget is exactly that figure extracts the batch without RIFT2_E_NOMEM."""
    ctx = pkg.Context(pkg.default_params(max_keypoints=300), device=0)
    need = ctx.workspace_bytes([tuple(im.shape) for im in images])
    same = pkg.Context(pkg.default_params(max_keypoints=300, flags=pkg.FLAG_SIZE_GROUPS), device=0)
    need_same = same.workspace_bytes([tuple(im.shape) for im in images])
    assert need > need_same   # one group of all twelve against the largest single size
    tight = pkg.Context(pkg.default_params(max_keypoints=300), device=0, hbm_budget=need)
    tight.extract(images)
    tight.sync()
