"""Python binding of the RIFT2 GB300 library (librift2.so, C ABI in include/rift2.h).

Argument marshalling only: every step of the pipeline runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  If the library has not been built the import
of `lib()` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librift2.so")

OK, E_INVAL, E_NOMEM, E_CAPACITY, E_CUDA, E_TIMEOUT, E_UNIMPL = 0, -1, -2, -3, -4, -5, -6
FLAG_PLAIN_MATCH = 0x1
FLAG_NO_GROUPING = 0x2
FLAG_RIFT_TEMPLATE = 0x4   # RIFT baseline: one descriptor per keypoint, unshifted MIM
FLAG_RIFT_RING = 0x8       # RIFT baseline: the No descriptors of the convolution ring
FLAG_CORNERS = 0x10        # RIFT's corner keypoints on the minimum moment, after the edge ones
FLAG_AUTOTUNE = 0x20       # time the column tiles of a new image size once, keep the fastest
FLAG_SPATIAL_NORM = 0x40   # variant: patch grid rotated into the dominant index's frame
FLAG_SIZE_GROUPS = 0x80    # launch groups of one image size only (mixed sizes share launches without it)
FLAG_TWO_LANES = 0x100     # halves of a call on two internal streams (overlaps under-filled stages)
NS, NO, PATCH, CELLS = 4, 6, 96, 6
DESC_DIM = CELLS * CELLS * NO

# Every symbol include/rift2.h declares.
EXPORTS = ("rift2_default_params", "rift2_status_str", "rift2_create", "rift2_extract",
           "rift2_match", "rift2_sync", "rift2_destroy", "rift2_set_profiling",
           "rift2_profile_read", "rift2_launch_count", "rift2_fft2", "rift2_detect",
           "rift2_describe", "rift2_detect_static", "rift2_tuned_tile", "rift2_tuned_match_split",
           "rift2_fft_plan", "rift2_plan_groups",
           "rift2_required_capacity", "rift2_set_wait_limit", "rift2_evaluate",
           "rift2_workspace_bytes")
STATIC_MAX_CANDIDATES = 262144
STAGES = ("fft_fwd", "lg_cols", "lg_rows", "noise", "moment", "detect", "describe", "match")


class Params(C.Structure):
    _fields_ = [("n_scales", C.c_int), ("n_orient", C.c_int), ("min_wavelength", C.c_float),
                ("mult", C.c_float), ("sigma_onf", C.c_float), ("k", C.c_float),
                ("g", C.c_float), ("cutoff", C.c_float), ("eps", C.c_float),
                ("lp_cutoff", C.c_float), ("lp_order", C.c_int), ("fast_threshold", C.c_float),
                ("fast_arc", C.c_int), ("max_keypoints", C.c_int), ("patch", C.c_int),
                ("cells", C.c_int), ("second_ratio", C.c_float), ("flags", C.c_int)]


class Image(C.Structure):
    _fields_ = [("data", C.c_void_p), ("height", C.c_int), ("width", C.c_int),
                ("pitch", C.c_longlong)]


class DebugMaps(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("amp", "er", "q", "an0", "pc", "moment", "mim",
                                          "noise_t", "spectrum")]


class FeaturesC(C.Structure):
    _fields_ = [("cap_kp", C.c_int), ("cap_desc", C.c_int), ("kp_xy", C.c_void_p),
                ("kp_score", C.c_void_p), ("desc", C.c_void_p), ("desc_norm", C.c_void_p),
                ("desc_kp", C.c_void_p), ("desc_dom", C.c_void_p), ("counts", C.c_void_p),
                ("debug", C.POINTER(DebugMaps))]


class MatchesC(C.Structure):
    _fields_ = [("cap", C.c_int), ("q_desc", C.c_void_p), ("nn_desc", C.c_void_p),
                ("kp_a", C.c_void_p), ("kp_b", C.c_void_p), ("d1", C.c_void_p),
                ("d2", C.c_void_p), ("near_tie", C.c_void_p), ("count", C.c_void_p)]


class Evaluation(C.Structure):
    _fields_ = [("n_matches", C.c_int), ("n_correct", C.c_int), ("success", C.c_int),
                ("reserved", C.c_int), ("rmse", C.c_double)]


_LIB = None


def lib():
    """The loaded library; raises if it is missing (build it with __graft_entry__.build())."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"RIFT2 CUDA library not built: {LIB_PATH} is missing")
        L = C.CDLL(LIB_PATH)
        L.rift2_status_str.restype = C.c_char_p
        L.rift2_status_str.argtypes = [C.c_int]
        L.rift2_default_params.argtypes = [C.POINTER(Params)]
        L.rift2_create.argtypes = [C.POINTER(Params), C.c_int, C.c_size_t, C.POINTER(C.c_void_p)]
        L.rift2_extract.argtypes = [C.c_void_p, C.c_int, C.POINTER(Image), C.POINTER(FeaturesC),
                                    C.c_void_p]
        L.rift2_match.argtypes = [C.c_void_p, C.c_int, C.POINTER(FeaturesC),
                                  C.POINTER(FeaturesC), C.POINTER(MatchesC), C.c_void_p]
        L.rift2_sync.argtypes = [C.c_void_p, C.c_void_p]
        L.rift2_destroy.argtypes = [C.c_void_p]
        L.rift2_set_profiling.argtypes = [C.c_void_p, C.c_int]
        L.rift2_profile_read.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_double),
                                         C.POINTER(C.c_longlong)]
        L.rift2_launch_count.argtypes = [C.c_void_p]
        L.rift2_launch_count.restype = C.c_longlong
        L.rift2_tuned_tile.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.rift2_tuned_match_split.argtypes = [C.c_void_p, C.c_int]
        L.rift2_fft_plan.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int]
        L.rift2_plan_groups.argtypes = [C.c_void_p, C.c_size_t, C.c_int, C.POINTER(C.c_int),
                                        C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.rift2_required_capacity.argtypes = [C.c_void_p, C.POINTER(C.c_int),
                                              C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.rift2_set_wait_limit.argtypes = [C.c_void_p, C.c_longlong]
        L.rift2_workspace_bytes.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                            C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_size_t)]
        L.rift2_evaluate.argtypes = [C.c_void_p, C.c_int, C.POINTER(FeaturesC),
                                     C.POINTER(FeaturesC), C.POINTER(MatchesC),
                                     C.POINTER(C.c_double), C.c_double, C.c_double, C.c_int,
                                     C.c_void_p, C.c_void_p]
        L.rift2_fft2.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                 C.c_void_p]
        L.rift2_detect.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                   C.POINTER(FeaturesC), C.c_void_p]
        L.rift2_describe.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                     C.POINTER(FeaturesC), C.c_void_p]
        L.rift2_detect_static.argtypes = [C.POINTER(Params), C.c_void_p, C.c_int, C.c_int,
                                          C.POINTER(FeaturesC), C.c_void_p]
        _LIB = L
    return _LIB


class Rift2Error(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {lib().rift2_status_str(code).decode()} ({code})")
        self.code = code


def _check(code: int, what: str):
    if code != OK:
        raise Rift2Error(code, what)


def default_params(**overrides) -> Params:
    p = Params()
    lib().rift2_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def fft_plan(n: int, rows: bool = False) -> tuple[int, list[int]]:
    """The transform the shared-memory kernels run for a side of length n (host only,
    rift2_fft_plan): (pass length, radices in pass order)."""
    length = C.c_int()
    rad = (C.c_int * 16)()
    k = lib().rift2_fft_plan(int(n), int(bool(rows)), C.byref(length), rad, 16)
    if k < 0:
        raise Rift2Error(k, "rift2_fft_plan")
    return int(length.value), [int(rad[i]) for i in range(k)]


def plan_groups(sizes, params: Params | None = None, hbm_budget: int = 0):
    """The launch groups rift2_extract forms for images of `sizes` [(H, W), ...] (host
    only, rift2_plan_groups): (launch order of the images, sizes of the groups)."""
    n = len(sizes)
    hs = (C.c_int * max(n, 1))(*[int(h) for h, _ in sizes])
    ws = (C.c_int * max(n, 1))(*[int(w) for _, w in sizes])
    order, gs, ng = (C.c_int * max(n, 1))(), (C.c_int * max(n, 1))(), C.c_int()
    p = params if params is not None else default_params()
    _check(lib().rift2_plan_groups(C.byref(p), int(hbm_budget), n, hs, ws, order, gs,
                                   C.byref(ng)), "rift2_plan_groups")
    return [int(order[i]) for i in range(n)], [int(gs[i]) for i in range(ng.value)]


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _require(t, name: str, dtype, ndim: int):
    """A dense CUDA tensor of the given dtype and rank: the C ABI reads it as a plain
    row-major array, so a strided view would be read wrongly without an error."""
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or t.dim() != ndim:
        raise ValueError(f"{name} must be a {ndim}-D {dtype} tensor, got {t.dim()}-D {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


@dataclass
class Features:
    """Device buffers of one image's features (see rift2_features in include/rift2.h)."""
    kp_xy: torch.Tensor      # int32 [cap_kp][2]
    kp_score: torch.Tensor   # float32 [cap_kp]
    desc: torch.Tensor       # uint16 as int16 storage [cap_desc][216]
    desc_norm: torch.Tensor  # float32 [cap_desc]
    desc_kp: torch.Tensor    # int32 [cap_desc]
    desc_dom: torch.Tensor   # uint8 [cap_desc]
    counts: torch.Tensor     # int32 [2]: n_kp, n_desc
    debug: dict | None = None

    @staticmethod
    def alloc(max_kp: int, device, debug_shape=None, desc_per_kp: int = 2):
        dev = torch.device(device)
        nd = desc_per_kp * max_kp
        f = Features(
            kp_xy=torch.zeros((max_kp, 2), dtype=torch.int32, device=dev),
            kp_score=torch.zeros(max_kp, dtype=torch.float32, device=dev),
            desc=torch.zeros((nd, DESC_DIM), dtype=torch.int16, device=dev),
            desc_norm=torch.zeros(nd, dtype=torch.float32, device=dev),
            desc_kp=torch.zeros(nd, dtype=torch.int32, device=dev),
            desc_dom=torch.zeros(nd, dtype=torch.uint8, device=dev),
            counts=torch.zeros(2, dtype=torch.int32, device=dev))
        if debug_shape is not None:
            h, w = debug_shape
            f.debug = {n: torch.zeros((NO, h, w), dtype=torch.float32, device=dev)
                       for n in ("amp", "er", "q", "an0", "pc")}
            f.debug["moment"] = torch.zeros((h, w), dtype=torch.float32, device=dev)
            f.debug["mim"] = torch.zeros((h, w), dtype=torch.uint8, device=dev)
            f.debug["noise_t"] = torch.zeros(NO, dtype=torch.float32, device=dev)
        return f

    def keep_maps(self, shape, names=("mim", "spectrum")):
        """Attach device buffers that the next extraction fills with the named maps (a
        subset of the debug maps; "spectrum" is complex64 [H][W], "mim" uint8 [H][W])."""
        h, w = shape
        dev = self.kp_xy.device
        shapes = {"mim": ((h, w), torch.uint8), "spectrum": ((h, w), torch.complex64),
                  "moment": ((h, w), torch.float32), "noise_t": ((NO,), torch.float32)}
        self.debug = {n: torch.empty(shapes[n][0], dtype=shapes[n][1], device=dev) for n in names}
        return self

    def to_c(self):
        c = FeaturesC(self.kp_xy.shape[0], self.desc.shape[0], _ptr(self.kp_xy).value,
                      _ptr(self.kp_score).value, _ptr(self.desc).value,
                      _ptr(self.desc_norm).value, _ptr(self.desc_kp).value,
                      _ptr(self.desc_dom).value, _ptr(self.counts).value, None)
        keep = None
        if self.debug is not None:
            keep = DebugMaps(*[self.debug[n].data_ptr() if n in self.debug else None
                               for n, _ in DebugMaps._fields_])
            c.debug = C.pointer(keep)
        return c, keep

    def host(self):
        """Trimmed CPU copies (synchronising): dict of numpy arrays."""
        n_kp, n_desc = [int(v) for v in self.counts.cpu()]
        return dict(xy=self.kp_xy[:n_kp].cpu().numpy(), score=self.kp_score[:n_kp].cpu().numpy(),
                    desc=self.desc[:n_desc].cpu().numpy().view("uint16"),
                    desc_norm=self.desc_norm[:n_desc].cpu().numpy(),
                    desc_kp=self.desc_kp[:n_desc].cpu().numpy(),
                    desc_dom=self.desc_dom[:n_desc].cpu().numpy())


@dataclass
class Matches:
    q_desc: torch.Tensor
    nn_desc: torch.Tensor
    kp_a: torch.Tensor
    kp_b: torch.Tensor
    d1: torch.Tensor
    d2: torch.Tensor
    near_tie: torch.Tensor
    count: torch.Tensor

    @staticmethod
    def alloc(cap: int, device):
        dev = torch.device(device)
        z = lambda dt: torch.zeros(cap, dtype=dt, device=dev)  # noqa: E731
        return Matches(z(torch.int32), z(torch.int32), z(torch.int32), z(torch.int32),
                       z(torch.float32), z(torch.float32), z(torch.uint8),
                       torch.zeros(1, dtype=torch.int32, device=dev))

    def to_c(self):
        return MatchesC(self.q_desc.shape[0], *[t.data_ptr() for t in (
            self.q_desc, self.nn_desc, self.kp_a, self.kp_b, self.d1, self.d2, self.near_tie,
            self.count)])

    def host(self):
        n = int(self.count.cpu()[0])
        return {k: getattr(self, k)[:n].cpu().numpy() for k in
                ("q_desc", "nn_desc", "kp_a", "kp_b", "d1", "d2", "near_tie")}


class Context:
    """One rift2_ctx on one CUDA device."""

    def __init__(self, params: Params | None = None, device: int = 0, hbm_budget: int = 0):
        self.params = params if params is not None else default_params()
        self.device = device
        h = C.c_void_p()
        _check(lib().rift2_create(C.byref(self.params), device, hbm_budget, C.byref(h)),
               "rift2_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().rift2_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def max_kp(self) -> int:
        return int(self.params.max_keypoints)

    @property
    def kp_cap(self) -> int:
        """Keypoint list capacity per image: max_keypoints, twice that with corners."""
        return self.max_kp * (2 if self.params.flags & FLAG_CORNERS else 1)

    @property
    def desc_per_kp(self) -> int:
        return NO if self.params.flags & FLAG_RIFT_RING else 2

    def alloc_features(self, debug_shape=None) -> Features:
        return Features.alloc(self.kp_cap, f"cuda:{self.device}", debug_shape, self.desc_per_kp)

    def alloc_matches(self) -> Matches:
        return Matches.alloc(self.desc_per_kp * self.kp_cap, f"cuda:{self.device}")

    def extract(self, images, feats=None, stream=None, debug=False):
        """images: list of float32 CUDA tensors [H][W] (rows may be strided)."""
        n = len(images)
        if feats is None:
            feats = [self.alloc_features(tuple(im.shape) if debug else None) for im in images]
        arr = (Image * n)()
        for i, im in enumerate(images):
            if not isinstance(im, torch.Tensor) or im.device.type != "cuda":
                raise ValueError("images must be CUDA tensors")
            if im.dtype != torch.float32 or im.dim() != 2 or im.stride(1) != 1:
                raise ValueError("images must be 2-D float32 with unit column stride")
            arr[i] = Image(im.data_ptr(), im.shape[0], im.shape[1], im.stride(0))
        fc = (FeaturesC * n)()
        keep = []
        for i, f in enumerate(feats):
            fc[i], k = f.to_c()
            keep.append(k)
        _check(lib().rift2_extract(self._h, n, arr, fc, _stream(stream)), "rift2_extract")
        return feats

    def match(self, fa, fb, out=None, stream=None):
        n = len(fa)
        if out is None:
            out = [self.alloc_matches() for _ in range(n)]
        ca, cb, cm = (FeaturesC * n)(), (FeaturesC * n)(), (MatchesC * n)()
        for i in range(n):
            ca[i], _ = fa[i].to_c()
            cb[i], _ = fb[i].to_c()
            cm[i] = out[i].to_c()
        _check(lib().rift2_match(self._h, n, ca, cb, cm, _stream(stream)), "rift2_match")
        return out

    def evaluate(self, fa, fb, matches, affines, tol=3.0, rmse_cap=20.0, min_correct=10,
                 out=None, stream=None):
        """Ground truth of each pair's matches under its known transform (rift2_evaluate):
        affines is a list of 6-tuples (t0..t5) mapping A's pixel coordinates into B's.
        Returns a CUDA byte tensor holding the rift2_evaluation structs; evaluation_host()
        reads it."""
        n = len(fa)
        if out is None:
            out = torch.zeros(n * C.sizeof(Evaluation), dtype=torch.uint8,
                              device=f"cuda:{self.device}")
        ca, cb, cm = (FeaturesC * n)(), (FeaturesC * n)(), (MatchesC * n)()
        for i in range(n):
            ca[i], _ = fa[i].to_c()
            cb[i], _ = fb[i].to_c()
            cm[i] = matches[i].to_c()
        tf = (C.c_double * (6 * n))(*[float(v) for t in affines for v in t])
        _check(lib().rift2_evaluate(self._h, n, ca, cb, cm, tf, tol, rmse_cap, min_correct,
                                    _ptr(out), _stream(stream)), "rift2_evaluate")
        return out

    @staticmethod
    def evaluation_host(out) -> list:
        """The rift2_evaluation structs of a Context.evaluate result as dicts."""
        raw = bytes(out.cpu().numpy())
        n = len(raw) // C.sizeof(Evaluation)
        res = []
        for i in range(n):
            e = Evaluation.from_buffer_copy(raw, i * C.sizeof(Evaluation))
            res.append(dict(matches=e.n_matches, correct=e.n_correct, success=bool(e.success),
                            rmse=e.rmse))
        return res

    def sync(self, stream=None):
        _check(lib().rift2_sync(self._h, _stream(stream)), "rift2_sync")

    # ---- tracing
    def set_profiling(self, on: bool):
        _check(lib().rift2_set_profiling(self._h, int(bool(on))), "rift2_set_profiling")

    def profile_read(self) -> dict:
        """{stage: (ms, launches)} accumulated since the last read (waits for the events)."""
        n = len(STAGES)
        ms = (C.c_double * n)()
        cnt = (C.c_longlong * n)()
        _check(lib().rift2_profile_read(self._h, n, ms, cnt), "rift2_profile_read")
        return {STAGES[i]: (ms[i], cnt[i]) for i in range(n)}

    def launch_count(self) -> int:
        return int(lib().rift2_launch_count(self._h))

    def required_capacity(self) -> dict:
        """Buffer capacities this context's calls require (cap_kp, cap_desc, cap_match)."""
        v = [C.c_int(), C.c_int(), C.c_int()]
        _check(lib().rift2_required_capacity(self._h, *[C.byref(x) for x in v]),
               "rift2_required_capacity")
        return dict(cap_kp=v[0].value, cap_desc=v[1].value, cap_match=v[2].value)

    def workspace_bytes(self, sizes, n_pairs: int = 0) -> int:
        """Workspace bytes an extract of images of `sizes` [(H, W), ...] followed by a match
        of n_pairs pairs needs in this context (rift2_workspace_bytes)."""
        n = len(sizes)
        hs = (C.c_int * max(n, 1))(*[int(h) for h, _ in sizes])
        ws = (C.c_int * max(n, 1))(*[int(w) for _, w in sizes])
        out = C.c_size_t()
        _check(lib().rift2_workspace_bytes(self._h, n, hs, ws, int(n_pairs), C.byref(out)),
               "rift2_workspace_bytes")
        return int(out.value)

    def set_wait_limit(self, iters: int = 1 << 24):
        """First-wait limit of the descriptor kernel's staged copies (0: give up at once,
        which exercises the RIFT2_E_TIMEOUT path; the default restores normal waits)."""
        _check(lib().rift2_set_wait_limit(self._h, int(iters)), "rift2_set_wait_limit")

    def tuned_tile(self, height: int, width: int) -> int:
        """Column tile the autotuner kept for this size (0: none tuned)."""
        return int(lib().rift2_tuned_tile(self._h, height, width))

    def tuned_match_split(self, n_pairs: int) -> int:
        """Split of B's columns the autotuner kept for match calls of n_pairs pairs (0: none)."""
        return int(lib().rift2_tuned_match_split(self._h, int(n_pairs)))

    # ---- stage entry points
    def fft2(self, img, stream=None):
        """img: float32 CUDA [n][H][W] contiguous -> complex64 [n][H][W]."""
        _require(img, "img", torch.float32, 3)
        n, h, w = img.shape
        out = torch.empty((n, h, w), dtype=torch.complex64, device=img.device)
        _check(lib().rift2_fft2(self._h, n, _ptr(img), h, w, _ptr(out), _stream(stream)),
               "rift2_fft2")
        return out

    def detect(self, moment, feats=None, stream=None):
        """moment: float32 CUDA [n][H][W] contiguous maximum-moment maps."""
        _require(moment, "moment", torch.float32, 3)
        n, h, w = moment.shape
        if feats is None:
            feats = [self.alloc_features() for _ in range(n)]
        fc = (FeaturesC * n)()
        for i, f in enumerate(feats):
            fc[i], _ = f.to_c()
        _check(lib().rift2_detect(self._h, n, _ptr(moment), h, w, fc, _stream(stream)),
               "rift2_detect")
        return feats

    def describe(self, mim, feats, stream=None):
        """mim: uint8 CUDA [n][H][W] contiguous maximum index maps (values 0..No-1)."""
        _require(mim, "mim", torch.uint8, 3)
        n, h, w = mim.shape
        fc = (FeaturesC * n)()
        for i, f in enumerate(feats):
            fc[i], _ = f.to_c()
        _check(lib().rift2_describe(self._h, n, _ptr(mim), h, w, fc, _stream(stream)),
               "rift2_describe")
        return feats


def detect_static(moment, feats: Features, params: Params | None = None, stream=None):
    """Keypoints of one moment map [H][W] (float32, CUDA) without any device allocation by
    the library (rift2_detect_static): for callers that must not allocate device memory.
    `feats` supplies the output buffers.  The call runs on the map's device (made current
    for the call) and on `stream`, by default that device's current stream.  Calls that
    overlap on the GPU share one static scratch array and must be serialised."""
    _require(moment, "moment", torch.float32, 2)
    h, w = moment.shape
    fc, _ = feats.to_c()
    p = C.byref(params) if params is not None else None
    with torch.cuda.device(moment.device):
        st = stream if stream is not None else torch.cuda.current_stream(moment.device)
        _check(lib().rift2_detect_static(p, _ptr(moment), h, w, C.byref(fc), _stream(st)),
               "rift2_detect_static")
    return feats
