"""GB300 (sm_103a) co-sparse data term: thin Python binding of libcosparse.so.

Every step of the computation runs in the library's CUDA kernels behind the
C ABI declared in ``include/cosparse.h``. This module only marshals
arguments: it allocates outputs as torch CUDA tensors, passes raw device
pointers and the current CUDA stream, and turns status codes into
exceptions. There is no CPU fallback: if the library is missing, ``lib()``
raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_build", "libcosparse.so")

CS_OK = 0
CS_ERR_INVALID_ARG = 1
CS_ERR_CUDA = 2
CS_ERR_NOMEM = 3
CS_ERR_TIMEOUT = 4
CS_ERR_UNSUPPORTED = 5
CS_ERR_DEVICE = 6

MODE_PERSAMPLE = 0
MODE_FACTORISED = 1
MODE_SMOOTH = 2  # smooth co-support texture (Eq. map_tsm, approx_cosupp, post_text); data_term only
FP32 = 0
BF16 = 1
FP8 = 2
CODES_AUTO = 0
CODES_FP32 = 1
CODES_TC = 2

STALL_NONE = 0
STALL_SEGMENT = 1
STALL_SUM = 2

# every symbol include/cosparse.h declares
EXPORTS = (
    "cs_params_default",
    "cs_version",
    "cs_create",
    "cs_destroy",
    "cs_last_error",
    "cs_sync_status",
    "cs_test_wait",
    "cs_codes",
    "cs_codes_noalloc",
    "cs_cosupport",
    "cs_likelihood",
    "cs_data_term",
    "cs_refined_count",
    "cs_seg_params_default",
    "cs_segment",
    "cs_kmeans",
    "cs_kmedians",
    "cs_unsup_params_default",
    "cs_unsup_data_term",
    "cs_batch_create",
    "cs_batch_run",
    "cs_batch_config",
    "cs_batch_set_config",
    "cs_batch_destroy",
    "cs_batch_data_term",
    "cs_batch_likelihood",
    "cs_surrogate_fit",
    "cs_surrogate_eval",
    "cs_surrogate_params",
    "cs_surrogate_info",
    "cs_surrogate_save",
    "cs_surrogate_load",
    "cs_mlp_param_count",
    "cs_mlp_forward",
    "cs_mlp_grad",
    "cs_unit_rates",
    "cs_profile_enable",
    "cs_profile_read",
)

STAGE_CODES = 0
STAGE_DIST = 1
STAGE_GATHER = 2
STAGE_SUM = 3
STAGE_SURROGATE = 4
STAGE_TRAIN = 5
SURR_BASIC = 0
SURR_EXTENDED = 1
FALLBACK_GUARANTEED = 0
FALLBACK_MARGIN = 1
FALLBACK_NONE = 2


class CsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"[cs status {status}] {msg}")
        self.status = status


class Params(ctypes.Structure):
    """Mirror of cs_params (include/cosparse.h)."""

    _fields_ = [
        ("p", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("codes_form", ctypes.c_int32),
        ("tau", ctypes.c_double),
        ("sigma_c2", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("d_min", ctypes.c_double),
        ("kappa_beta", ctypes.c_double),
        ("l_tol", ctypes.c_double),
        ("iota_sigma", ctypes.c_double),
        ("rho_variance", ctypes.c_int32),
        ("patch_order", ctypes.c_int32),
    ]

    @classmethod
    def default(cls, **kw):
        p = cls()
        lib().cs_params_default(ctypes.byref(p))
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    @classmethod
    def from_synth(cls, sp, **kw):
        """From a ``synth.Params`` dataclass."""
        p = cls.default(p=sp.p, mode=sp.mode, tau=sp.tau, sigma_c2=sp.sigma_c2, alpha=sp.alpha,
                        d_min=sp.d_min, kappa_beta=sp.kappa_beta,
                        iota_sigma=getattr(sp, "iota_sigma", 0.01),
                        rho_variance=int(getattr(sp, "rho_variance", 0)))
        for k, v in kw.items():
            setattr(p, k, v)
        return p


class SegParams(ctypes.Structure):
    """Mirror of cs_seg_params (include/cosparse.h)."""

    _fields_ = [
        ("lam", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("iterations", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]

    @classmethod
    def default(cls, **kw):
        p = cls()
        lib().cs_seg_params_default(ctypes.byref(p))
        for k, v in kw.items():
            setattr(p, k, v)
        return p


class UnsupParams(ctypes.Structure):
    """Mirror of cs_unsup_params (include/cosparse.h)."""

    _fields_ = [
        ("n_colour", ctypes.c_int32),
        ("n_texture", ctypes.c_int32),
        ("kmeans_iterations", ctypes.c_int32),
        ("kmedians_iterations", ctypes.c_int32),
        ("beta", ctypes.c_double),
    ]

    @classmethod
    def default(cls, **kw):
        p = cls()
        lib().cs_unsup_params_default(ctypes.byref(p))
        for k, v in kw.items():
            setattr(p, k, v)
        return p


class Image(ctypes.Structure):
    """Mirror of cs_image (include/cosparse.h)."""

    _fields_ = [
        ("img", ctypes.c_void_p),
        ("H", ctypes.c_int32),
        ("W", ctypes.c_int32),
        ("n_labels", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("label_off", ctypes.c_void_p),
        ("sample_pix", ctypes.c_void_p),
        ("bitmask", ctypes.c_void_p),
        ("dist2", ctypes.c_void_p),
        ("neglog", ctypes.c_void_p),
        ("post", ctypes.c_void_p),
    ]


BATCH_GRAPH = 1
BATCH_AUTOTUNE = 2

_lib = None


def lib(path: str | None = None):
    """Load libcosparse.so (built in-tree by ``build.build()``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    so = path or SO_PATH
    if not os.path.exists(so):
        raise RuntimeError(
            f"libcosparse.so not found at {so}: build it with "
            "`python -m paper_1312_4746_gb300.build` (there is no CPU fallback)")
    L = ctypes.CDLL(so)
    V, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.cs_params_default.argtypes = [ctypes.POINTER(Params)]
    L.cs_params_default.restype = None
    L.cs_version.restype = ctypes.c_char_p
    L.cs_create.argtypes = [ctypes.POINTER(V), I]
    L.cs_destroy.argtypes = [V]
    L.cs_destroy.restype = None
    L.cs_last_error.argtypes = [V]
    L.cs_last_error.restype = ctypes.c_char_p
    L.cs_sync_status.argtypes = [V, V]
    L.cs_test_wait.argtypes = [V, ctypes.c_int64, I]
    L.cs_refined_count.argtypes = [V, ctypes.POINTER(ctypes.c_int32), V]
    L.cs_seg_params_default.argtypes = [ctypes.POINTER(SegParams)]
    L.cs_seg_params_default.restype = None
    L.cs_segment.argtypes = [V, V, V, I, I, I, ctypes.POINTER(SegParams), V, V, V]
    L.cs_kmeans.argtypes = [V, V, I, I, V, I, V, V, V]
    L.cs_kmedians.argtypes = [V, V, I, I, I, V, I, V, V, V]
    L.cs_unsup_params_default.argtypes = [ctypes.POINTER(UnsupParams)]
    L.cs_unsup_params_default.restype = None
    L.cs_unsup_data_term.argtypes = [V, V, I, I, V, I, V, ctypes.POINTER(Params),
                                     ctypes.POINTER(UnsupParams), V, V, V, V, V, V, V, V]
    L.cs_codes.argtypes = [V, V, I, I, V, I, V, ctypes.POINTER(Params), V, V, V, V]
    L.cs_cosupport.argtypes = [V, V, I, I, D, V, V]
    L.cs_codes_noalloc.argtypes = [V, I, I, V, I, V, ctypes.POINTER(Params), V, V, V, V, V]
    L.cs_codes_noalloc.restype = I
    L.cs_likelihood.argtypes = [V, V, I, I, V, I, I, V, V, ctypes.POINTER(Params), V, V, V, V]
    L.cs_data_term.argtypes = [V, V, I, I, V, I, V, I, V, V, ctypes.POINTER(Params), V, V, V, V, V]
    L.cs_batch_create.argtypes = [V, ctypes.POINTER(Image), I, V, I, V, ctypes.POINTER(Params), I,
                                  ctypes.POINTER(V)]
    L.cs_batch_run.argtypes = [V, V]
    L.cs_batch_config.argtypes = [V, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(D), ctypes.POINTER(D),
                                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    L.cs_batch_set_config.argtypes = [V, I, I, I]
    L.cs_batch_destroy.argtypes = [V]
    L.cs_batch_destroy.restype = None
    L.cs_batch_data_term.argtypes = [V, ctypes.POINTER(Image), I, V, I, V, ctypes.POINTER(Params),
                                     V]
    L.cs_batch_likelihood.argtypes = [V, ctypes.POINTER(Image), I, I, ctypes.POINTER(Params), V]
    U64 = ctypes.c_uint64
    L.cs_surrogate_fit.argtypes = [V, V, I, I, V, V, I, I, V, V, ctypes.POINTER(Params), D, I, I,
                                   U64, V]
    L.cs_surrogate_eval.argtypes = [V, V, I, I, V, V, I, I, V, V, ctypes.POINTER(Params), I, D, V, V,
                                    V, V]
    L.cs_surrogate_params.argtypes = [V, V, I, ctypes.POINTER(I)]
    L.cs_surrogate_info.argtypes = [V, V, I, V, V, ctypes.POINTER(I), ctypes.POINTER(I),
                                    ctypes.POINTER(I)]
    L.cs_surrogate_save.argtypes = [V, ctypes.c_char_p]
    L.cs_surrogate_load.argtypes = [V, ctypes.c_char_p]
    L.cs_mlp_param_count.argtypes = [I, I]
    L.cs_mlp_param_count.restype = I
    L.cs_mlp_forward.argtypes = [V, V, I, I, V, I, V, V]
    L.cs_mlp_grad.argtypes = [V, V, I, I, V, V, I, V, V, V]
    L.cs_unit_rates.argtypes = [V, V, V]
    L.cs_unit_rates.restype = I
    L.cs_profile_enable.argtypes = [V, I]
    L.cs_profile_read.argtypes = [V, I, ctypes.POINTER(D), ctypes.POINTER(I)]
    for f in ("cs_create", "cs_sync_status", "cs_test_wait", "cs_refined_count", "cs_segment", "cs_codes", "cs_cosupport", "cs_likelihood",
              "cs_data_term", "cs_profile_enable", "cs_profile_read", "cs_surrogate_fit",
              "cs_surrogate_eval", "cs_surrogate_params", "cs_surrogate_info", "cs_surrogate_save",
              "cs_surrogate_load", "cs_mlp_forward",
              "cs_mlp_grad", "cs_batch_create", "cs_batch_run", "cs_batch_config",
              "cs_batch_set_config", "cs_batch_data_term", "cs_batch_likelihood"):
        getattr(L, f).restype = I
    if path is None:
        _lib = L
    return L


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """Owns a cs_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self._lib = lib()
        self.device = device
        h = ctypes.c_void_p()
        st = self._lib.cs_create(ctypes.byref(h), device)
        if st != CS_OK:
            raise CsError(st, self._lib.cs_last_error(None).decode())
        self.handle = h

    def check(self, st):
        if st != CS_OK:
            raise CsError(st, self._lib.cs_last_error(self.handle).decode())

    def sync(self):
        """Wait for the current stream and raise on a device-side error."""
        self.check(self._lib.cs_sync_status(self.handle, _stream()))

    def unit_rates(self):
        """cs_unit_rates: measured results per SM per clock of ex2, popc, FFMA
        and FFMA2, and the implied SM clock (MHz)."""
        out = (ctypes.c_double * 4)()
        clk = ctypes.c_double()
        self.check(self._lib.cs_unit_rates(self.handle, out, ctypes.byref(clk)))
        return {"ex2": out[0], "popc": out[1], "ffma": out[2], "ffma2": out[3],
                "clock_mhz": clk.value}

    def test_wait(self, limit_ns: int = 0, stall: int = 0):
        """Timeout-path test hook (cs_test_wait): the limit of the bounded
        device waits (0: the default 1 s) and a one-shot stall (STALL_*)."""
        self.check(self._lib.cs_test_wait(self.handle, int(limit_ns), int(stall)))

    def close(self):
        if getattr(self, "handle", None):
            self._lib.cs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile(self, on: bool = True):
        self.check(self._lib.cs_profile_enable(self.handle, int(on)))

    def profile_read(self, stage: int):
        """(summed milliseconds, launches) of one stage since the last read."""
        ms = ctypes.c_double()
        n = ctypes.c_int()
        self.check(self._lib.cs_profile_read(self.handle, stage, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    # ------------------------------------------------------------------ calls

    def codes(self, img, omega, mask, params: Params, want_codes=False, want_lead16=False,
              want_bitmask=True):
        """cs_codes: returns dict with 'bitmask' (P, Wk) int32 view of uint32
        words, and optionally 'codes' (P, k) and 'lead16' (P, 16) float32."""
        import torch

        H, W = int(img.shape[0]), int(img.shape[1])
        k = int(omega.shape[0])
        P = H * W
        dev = img.device
        out = {}
        out["codes"] = torch.empty((P, k), dtype=torch.float32, device=dev) if want_codes else None
        out["lead16"] = torch.empty((P, 16), dtype=torch.float32, device=dev) if want_lead16 else None
        out["bitmask"] = (torch.empty((P, (k + 31) // 32), dtype=torch.int32, device=dev)
                          if want_bitmask else None)
        self.check(self._lib.cs_codes(self.handle, _ptr(img), H, W, _ptr(omega), k, _ptr(mask),
                                      ctypes.byref(params), _ptr(out["codes"]),
                                      _ptr(out["lead16"]), _ptr(out["bitmask"]), _stream()))
        return out

    def cosupport(self, codes, tau, bitmask=None):
        import torch

        P, k = int(codes.shape[0]), int(codes.shape[1])
        if bitmask is None:
            bitmask = torch.empty((P, (k + 31) // 32), dtype=torch.int32, device=codes.device)
        self.check(self._lib.cs_cosupport(self.handle, _ptr(codes), P, k, float(tau),
                                          _ptr(bitmask), _stream()))
        return bitmask

    def likelihood(self, img, bitmask, k, label_off, sample_pix, params: Params,
                   want_dist2=False, want_post=True, out=None):
        """cs_likelihood: returns dict with 'neglog' (n, H, W), optionally
        'post' and 'dist2'. ``label_off`` is a host array (numpy or list);
        ``sample_pix`` a device int32 tensor."""
        import numpy as np
        import torch

        H, W = int(img.shape[0]), int(img.shape[1])
        off = np.ascontiguousarray(np.asarray(label_off, dtype=np.int32))
        nl = len(off) - 1
        dev = img.device
        if out is None:
            out = {
                "neglog": torch.empty((nl, H, W), dtype=torch.float32, device=dev),
                "post": torch.empty((nl, H, W), dtype=torch.float32, device=dev) if want_post else None,
                "dist2": torch.empty((nl, H, W), dtype=torch.int32, device=dev) if want_dist2 else None,
            }
        self.check(self._lib.cs_likelihood(
            self.handle, _ptr(img), H, W, _ptr(bitmask), int(k), nl,
            ctypes.c_void_p(off.ctypes.data), _ptr(sample_pix), ctypes.byref(params),
            _ptr(out.get("dist2")), _ptr(out["neglog"]), _ptr(out.get("post")), _stream()))
        return out


    def data_term(self, img, omega, mask, label_off, sample_pix, params: Params,
                  want_bitmask=False, want_dist2=False, want_post=True, out=None):
        """cs_data_term: codes, co-supports and likelihoods in one call.
        Returns dict with 'neglog' (n, H, W) and optionally 'post', 'bitmask',
        'dist2'. ``label_off`` is a host array; the other inputs are device
        tensors."""
        import numpy as np
        import torch

        H, W = int(img.shape[0]), int(img.shape[1])
        k = int(omega.shape[0])
        off = np.ascontiguousarray(np.asarray(label_off, dtype=np.int32))
        nl = len(off) - 1
        dev = img.device
        if out is None:
            out = {
                "neglog": torch.empty((nl, H, W), dtype=torch.float32, device=dev),
                "post": torch.empty((nl, H, W), dtype=torch.float32, device=dev) if want_post else None,
                "dist2": torch.empty((nl, H, W), dtype=torch.int32, device=dev) if want_dist2 else None,
                "bitmask": (torch.empty((H * W, (k + 31) // 32), dtype=torch.int32, device=dev)
                            if want_bitmask else None),
            }
        self.check(self._lib.cs_data_term(
            self.handle, _ptr(img), H, W, _ptr(omega), k, _ptr(mask), nl,
            ctypes.c_void_p(off.ctypes.data), _ptr(sample_pix), ctypes.byref(params),
            _ptr(out.get("bitmask")), _ptr(out.get("dist2")), _ptr(out["neglog"]),
            _ptr(out.get("post")), _stream()))
        return out

    def segment(self, f, img, sp: "SegParams", want_labels=True, out=None):
        """cs_segment: convex multilabel segmentation (Sec. 4) on the data term
        f (device (n, H, W) float32, e.g. neglog); returns dict 'u' (n, H, W)
        and 'labels' (H, W) int32."""
        import torch

        n, H, W = int(f.shape[0]), int(f.shape[1]), int(f.shape[2])
        dev = f.device
        if out is None:
            out = {"u": torch.empty((n, H, W), dtype=torch.float32, device=dev),
                   "labels": torch.empty((H, W), dtype=torch.int32, device=dev)
                   if want_labels else None}
        self.check(self._lib.cs_segment(self.handle, _ptr(f), _ptr(img), H, W, n,
                                        ctypes.byref(sp), _ptr(out["u"]), _ptr(out.get("labels")),
                                        _stream()))
        return out

    # ------------------------------------------------------------ unsupervised

    @staticmethod
    def _host_idx(idx):
        import numpy as np

        a = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
        return a, a.ctypes.data_as(ctypes.c_void_p)

    def kmeans(self, X, init, iterations, want_assign=True):
        """cs_kmeans on device points X (N, 3) float32 from the start indices
        ``init`` (host); returns dict 'centres' (n, 3) and 'assign' (N,)."""
        import torch

        keep, ip = self._host_idx(init)
        N, n = int(X.shape[0]), len(keep)
        out = {"centres": torch.empty((n, 3), dtype=torch.float32, device=X.device),
               "assign": torch.empty(N, dtype=torch.int32, device=X.device) if want_assign
               else None}
        self.check(self._lib.cs_kmeans(self.handle, _ptr(X), N, n, ip, int(iterations),
                                       _ptr(out["centres"]), _ptr(out["assign"]), _stream()))
        return out

    def kmedians(self, V, init, iterations, want_assign=True):
        """cs_kmedians on the columns of device V (k, N) float32."""
        import torch

        keep, ip = self._host_idx(init)
        k, N, n = int(V.shape[0]), int(V.shape[1]), len(keep)
        out = {"centres": torch.empty((n, k), dtype=torch.float32, device=V.device),
               "assign": torch.empty(N, dtype=torch.int32, device=V.device) if want_assign
               else None}
        self.check(self._lib.cs_kmedians(self.handle, _ptr(V), N, k, n, ip, int(iterations),
                                         _ptr(out["centres"]), _ptr(out["assign"]), _stream()))
        return out

    def unsup_data_term(self, img, omega, mask, params: Params, up: "UnsupParams", colour_init,
                        texture_init, out=None):
        """cs_unsup_data_term (Sec. 3.2): returns dict 'neglog'
        (n_colour n_texture, H, W), 'colour_centres', 'texture_centres',
        'colour_assign', 'texture_assign'."""
        import torch

        H, W = int(img.shape[0]), int(img.shape[1])
        k = int(omega.shape[0])
        dev = img.device
        ck, cp = self._host_idx(colour_init)
        tk, tp = self._host_idx(texture_init)
        if len(ck) != up.n_colour or len(tk) != up.n_texture:
            raise ValueError("start index counts must equal n_colour and n_texture")
        if out is None:
            out = {"neglog": torch.empty((up.n_colour * up.n_texture, H, W), dtype=torch.float32,
                                         device=dev),
                   "colour_centres": torch.empty((up.n_colour, 3), dtype=torch.float32, device=dev),
                   "texture_centres": torch.empty((up.n_texture, k), dtype=torch.float32,
                                                  device=dev),
                   "colour_assign": torch.empty((H, W), dtype=torch.int32, device=dev),
                   "texture_assign": torch.empty((H, W), dtype=torch.int32, device=dev)}
        self.check(self._lib.cs_unsup_data_term(
            self.handle, _ptr(img), H, W, _ptr(omega), k, _ptr(mask), ctypes.byref(params),
            ctypes.byref(up), cp, tp, _ptr(out["neglog"]), _ptr(out.get("colour_centres")),
            _ptr(out.get("texture_centres")), _ptr(out.get("colour_assign")),
            _ptr(out.get("texture_assign")), _stream()))
        return out

    def refined_count(self):
        """Pixels the last tensor-core sum recomputed in FP64 (cs_refined_count)."""
        n = ctypes.c_int32()
        self.check(self._lib.cs_refined_count(self.handle, ctypes.byref(n), _stream()))
        return n.value

    # ------------------------------------------------------------------ batches

    def batch(self, images, omega, mask, params: Params, flags=0, want_post=True,
              want_bitmask=False, want_dist2=False):
        """cs_batch_create over ``images``: a list of dicts with device tensors
        'img' (H, W, 3) and 'sample_pix', and host 'label_off'. Outputs are
        allocated here (torch) and returned with the batch."""
        return Batch(self, images, omega, mask, params, flags, want_post, want_bitmask, want_dist2)

    def batch_likelihood(self, images, k, params: Params, want_post=True):
        """cs_batch_likelihood: every image dict also carries its device
        'bitmask' (from codes); one-shot, synchronises the current stream."""
        arr, outs, keep = _batch_descs(images, int(k), want_post, False, False, bitmask_in=True)
        self.check(self._lib.cs_batch_likelihood(self.handle, arr, len(images), int(k),
                                                 ctypes.byref(params), _stream()))
        return outs

    def batch_data_term(self, images, omega, mask, params: Params, want_post=True):
        """cs_batch_data_term (one-shot; synchronises the current stream)."""
        arr, outs, keep = _batch_descs(images, int(omega.shape[0]), want_post, False, False)
        self.check(self._lib.cs_batch_data_term(
            self.handle, arr, len(images), _ptr(omega), int(omega.shape[0]), _ptr(mask),
            ctypes.byref(params), _stream()))
        return outs


    # ------------------------------------------------------------------ surrogate

    def surrogate_fit(self, img, bitmask, lead16, k, label_off, sample_pix, params: Params,
                      frac=0.05, steps=1000, features=0, seed=1):
        """cs_surrogate_fit (network kept in the context); features: SURR_BASIC
        or SURR_EXTENDED."""
        import numpy as np

        H, W = int(img.shape[0]), int(img.shape[1])
        off = np.ascontiguousarray(np.asarray(label_off, dtype=np.int32))
        self.check(self._lib.cs_surrogate_fit(
            self.handle, _ptr(img), H, W, _ptr(bitmask), _ptr(lead16), int(k), len(off) - 1,
            ctypes.c_void_p(off.ctypes.data), _ptr(sample_pix), ctypes.byref(params),
            float(frac), int(steps), int(features), ctypes.c_uint64(seed), _stream()))

    def surrogate_eval(self, img, bitmask, lead16, k, label_off, sample_pix, params: Params,
                       margin=0.1, rule=0, out=None, want_post=True, count=True):
        """cs_surrogate_eval: returns (dict with 'neglog'/'post', n_fallback or None);
        rule: FALLBACK_GUARANTEED, FALLBACK_MARGIN or FALLBACK_NONE."""
        import numpy as np
        import torch

        H, W = int(img.shape[0]), int(img.shape[1])
        off = np.ascontiguousarray(np.asarray(label_off, dtype=np.int32))
        nl = len(off) - 1
        if out is None:
            out = {"neglog": torch.empty((nl, H, W), dtype=torch.float32, device=img.device),
                   "post": (torch.empty((nl, H, W), dtype=torch.float32, device=img.device)
                            if want_post else None)}
        nfb = ctypes.c_int32(-1)
        self.check(self._lib.cs_surrogate_eval(
            self.handle, _ptr(img), H, W, _ptr(bitmask), _ptr(lead16), int(k), nl,
            ctypes.c_void_p(off.ctypes.data), _ptr(sample_pix), ctypes.byref(params),
            int(rule), float(margin), _ptr(out["neglog"]), _ptr(out.get("post")),
            ctypes.byref(nfb) if count else None, _stream()))
        return out, (nfb.value if count else None)

    def surrogate_params(self):
        import numpy as np

        n = ctypes.c_int()
        self.check(self._lib.cs_surrogate_params(self.handle, None, 0, ctypes.byref(n)))
        buf = np.zeros(n.value, np.float32)
        self.check(self._lib.cs_surrogate_params(self.handle, ctypes.c_void_p(buf.ctypes.data),
                                                 n.value, ctypes.byref(n)))
        return buf

    def surrogate_info(self, n_labels):
        """(stats mu_x, sd_x, mu_t, sd_t; eta; last loss; n_train; n_val; n_in)."""
        import numpy as np

        eta = ctypes.c_float()
        loss = ctypes.c_float()
        ntr = ctypes.c_int()
        nva = ctypes.c_int()
        nin = ctypes.c_int()
        self.check(self._lib.cs_surrogate_info(self.handle, None, 0, None, None, None, None,
                                               ctypes.byref(nin)))
        m = nin.value
        st = np.zeros(2 * m + 2 * n_labels, np.float32)
        self.check(self._lib.cs_surrogate_info(self.handle, ctypes.c_void_p(st.ctypes.data), st.size,
                                               ctypes.byref(eta), ctypes.byref(loss),
                                               ctypes.byref(ntr), ctypes.byref(nva), None))
        n = n_labels
        return {"mu_x": st[:m], "sd_x": st[m:2 * m], "mu_t": st[2 * m:2 * m + n],
                "sd_t": st[2 * m + n:2 * m + 2 * n], "eta": eta.value, "loss": loss.value,
                "n_train": ntr.value, "n_val": nva.value, "n_in": m}

    def surrogate_save(self, path):
        """cs_surrogate_save (synchronises)."""
        self.check(self._lib.cs_surrogate_save(self.handle, os.fsencode(path)))

    def surrogate_load(self, path):
        """cs_surrogate_load (synchronises)."""
        self.check(self._lib.cs_surrogate_load(self.handle, os.fsencode(path)))

    def mlp_forward(self, params_dev, n_out, X):
        """cs_mlp_forward on standardised rows X (rows x n_in)."""
        import torch

        Z = torch.empty((X.shape[0], n_out), dtype=torch.float32, device=X.device)
        self.check(self._lib.cs_mlp_forward(self.handle, _ptr(params_dev), int(X.shape[1]), n_out,
                                            _ptr(X), int(X.shape[0]), _ptr(Z), _stream()))
        return Z

    def mlp_grad(self, params_dev, n_out, X, T):
        """cs_mlp_grad: (gradient, loss) on standardised rows X and targets T."""
        import torch

        n_in = int(X.shape[1])
        g = torch.empty(self._lib.cs_mlp_param_count(n_in, n_out), dtype=torch.float32,
                        device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        self.check(self._lib.cs_mlp_grad(self.handle, _ptr(params_dev), n_in, n_out, _ptr(X),
                                         _ptr(T), int(X.shape[0]), _ptr(g), _ptr(loss), _stream()))
        return g, loss


def _batch_descs(images, k, want_post, want_bitmask, want_dist2, bitmask_in=False):
    import numpy as np
    import torch

    n = len(images)
    arr = (Image * n)()
    outs, keep = [], []
    for i, d in enumerate(images):
        img = d["img"]
        H, W = int(img.shape[0]), int(img.shape[1])
        off = np.ascontiguousarray(np.asarray(d["label_off"], dtype=np.int32))
        nl = len(off) - 1
        dev = img.device
        o = {"neglog": torch.empty((nl, H, W), dtype=torch.float32, device=dev),
             "post": torch.empty((nl, H, W), dtype=torch.float32, device=dev) if want_post else None,
             "dist2": torch.empty((nl, H, W), dtype=torch.int32, device=dev) if want_dist2 else None,
             "bitmask": (d["bitmask"] if bitmask_in else
                         torch.empty((H * W, (k + 31) // 32), dtype=torch.int32, device=dev)
                         if want_bitmask else None)}
        arr[i] = Image(img.data_ptr(), H, W, nl, 0, off.ctypes.data, d["sample_pix"].data_ptr(),
                       _ptr(o["bitmask"]), _ptr(o["dist2"]), o["neglog"].data_ptr(), _ptr(o["post"]))
        outs.append(o)
        keep.append(off)
    return arr, outs, keep


class Batch:
    """A planned batch (cs_batch): ``run()`` recomputes every image's outputs
    from the current contents of the input tensors named at creation."""

    def __init__(self, ctx: Context, images, omega, mask, params, flags, want_post, want_bitmask,
                 want_dist2):
        self.ctx = ctx
        self._inputs = (images, omega, mask)  # keep the device buffers alive
        arr, self.outputs, keep = _batch_descs(images, int(omega.shape[0]), want_post,
                                               want_bitmask, want_dist2)
        h = ctypes.c_void_p()
        ctx.check(ctx._lib.cs_batch_create(
            ctx.handle, arr, len(images), _ptr(omega), int(omega.shape[0]), _ptr(mask),
            ctypes.byref(params), int(flags), ctypes.byref(h)))
        self.handle = h

    def run(self):
        self.ctx.check(self.ctx._lib.cs_batch_run(self.handle, _stream()))
        return self.outputs

    def config(self):
        ns, om, var = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        pairs, tms = ctypes.c_double(), ctypes.c_double()
        shape = (ctypes.c_int32 * 4)()
        self.ctx.check(self.ctx._lib.cs_batch_config(self.handle, ctypes.byref(ns), ctypes.byref(om),
                                                     ctypes.byref(pairs), ctypes.byref(tms),
                                                     ctypes.byref(var), shape))
        return {"n_streams": ns.value, "order": om.value, "pairs": pairs.value,
                "tuned_ms": tms.value, "sum_variant": var.value,
                "sum_shape": {"ctas_per_sm": shape[0], "ring_stages": shape[1],
                              "texture_buffers": shape[2], "epilogue_warps": shape[3]}}

    def set_config(self, n_streams, order, sum_variant):
        """cs_batch_set_config: an explicit configuration instead of tuning."""
        self.ctx.check(self.ctx._lib.cs_batch_set_config(self.handle, int(n_streams), int(order),
                                                         int(sum_variant)))

    def close(self):
        if self.handle:
            self.ctx._lib.cs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version() -> str:
    return lib().cs_version().decode()
