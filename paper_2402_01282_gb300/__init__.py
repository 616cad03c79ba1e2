"""Python binding of libs2w.so, the GB300 directional wavelet transform library.

Thin ctypes marshalling over the C ABI declared in ``include/s2w.h``: every step of
every transform runs in the library's CUDA kernels; PyTorch only provides device
memory and the CUDA stream.  There is no fallback: if the compiled library is
missing or fails to load, ``load()`` raises.

Arrays are torch tensors on the GPU, C-contiguous, float64 (real spin-0 plans) or
complex128, with the layouts of ``include/s2w.h``.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libs2w.so")
_lib = None

S2W_FP64, S2W_FP32_SPLIT, S2W_BF16, S2W_FP64_NATIVE, S2W_FP64_TC = 0, 1, 2, 3, 4
S2W_SAMPLING_MW, S2W_SAMPLING_DH = 0, 1
STATUS = {0: "S2W_OK", 1: "S2W_EINVAL", 2: "S2W_ENOMEM", 3: "S2W_ECUDA", 4: "S2W_ETIMEOUT",
          5: "S2W_EUNSUPPORTED", 6: "S2W_ENONFINITE"}

# every symbol include/s2w.h declares
EXPORTS = ["s2w_plan_create", "s2w_plan_destroy", "s2w_query_layout", "s2w_forward", "s2w_inverse",
           "s2w_sht_forward", "s2w_sht_inverse", "s2w_wigner_forward", "s2w_wigner_inverse",
           "s2w_check", "s2w_last_error", "s2w_version", "s2w_trace_enable", "s2w_trace_reset",
           "s2w_trace_read", "s2w_kernel_name", "s2w_sht_inverse_static", "s2w_ball_plan_create",
           "s2w_ball_plan_destroy", "s2w_ball_nodes", "s2w_laguerre_forward", "s2w_laguerre_inverse",
           "s2w_ball_sl_forward", "s2w_ball_sl_inverse", "s2w_forward_adjoint", "s2w_inverse_adjoint",
           "s2w_ball_wav_plan_create", "s2w_ball_wav_plan_destroy", "s2w_ball_wav_query_layout",
           "s2w_ball_forward", "s2w_ball_inverse", "s2w_ball_forward_adjoint", "s2w_ball_inverse_adjoint",
           "s2w_ball_wav_check", "s2w_plan_autotune", "s2w_plan_launch_shapes", "s2w_plan_dft_forms", "s2w_batch_create",
           "s2w_batch_launch", "s2w_batch_destroy", "s2w_plan_device_bytes",
           "s2w_plan_inject_timeout", "s2w_plan_set_dft_forms", "s2w_shard_layout", "s2w_sht_inverse_columns",
           "s2w_sht_inverse_rings", "s2w_sht_forward_rings", "s2w_sht_forward_columns",
           "s2w_ball_wav_plan_autotune"]
KERNEL_KINDS = 5


class S2WError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class BallParams(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("P", ctypes.c_int), ("spin", ctypes.c_int), ("reality", ctypes.c_int),
                ("batch", ctypes.c_int), ("precision", ctypes.c_int), ("tau", ctypes.c_double),
                ("sampling", ctypes.c_int)]


class BallWavParams(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("N", ctypes.c_int), ("P", ctypes.c_int), ("J0", ctypes.c_int),
                ("J0r", ctypes.c_int), ("spin", ctypes.c_int), ("reality", ctypes.c_int), ("batch", ctypes.c_int),
                ("precision", ctypes.c_int), ("precompute", ctypes.c_int), ("lam", ctypes.c_double),
                ("nu", ctypes.c_double), ("tau", ctypes.c_double), ("sampling", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("N", ctypes.c_int), ("J0", ctypes.c_int), ("spin", ctypes.c_int),
                ("reality", ctypes.c_int), ("batch", ctypes.c_int), ("precision", ctypes.c_int),
                ("precompute", ctypes.c_int), ("lam", ctypes.c_double), ("sampling", ctypes.c_int)]


def rings(L: int, sampling: int = 0) -> int:
    """Colatitude rings of the grid at band-limit L: L (S2W_SAMPLING_MW) or 2L (S2W_SAMPLING_DH)."""
    if sampling not in (S2W_SAMPLING_MW, S2W_SAMPLING_DH):
        raise ValueError(f"unknown sampling {sampling}")
    return 2 * L if sampling == S2W_SAMPLING_DH else L


def shard_layout(L: int, spin: int, reality: bool, sampling: int, nranks: int, rank: int):
    """(c_begin, c_end, ring_begin, ring_end) of rank `rank` of `nranks` for the m-sharded spin
    SHT (s2w_shard_layout: host logic of the library, no GPU needed)."""
    lib = load()
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib.s2w_shard_layout(L, spin, int(bool(reality)), sampling, nranks, rank, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def load(path: str = LIB_PATH):
    """Load libs2w.so (raises if it is missing: there is no CPU path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libs2w.so not found at {path}; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    vp, i64p, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)
    lib.s2w_plan_create.argtypes = [ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]
    lib.s2w_plan_destroy.argtypes = [vp]
    lib.s2w_query_layout.argtypes = [vp, i64p, i64p, i64p, ip, i64p, ip, ip, ip]
    lib.s2w_forward.argtypes = [vp, vp, vp, vp, vp]
    lib.s2w_inverse.argtypes = [vp, vp, vp, vp, vp]
    lib.s2w_forward_adjoint.argtypes = [vp, vp, vp, vp, vp]
    lib.s2w_inverse_adjoint.argtypes = [vp, vp, vp, vp, vp]
    lib.s2w_sht_forward.argtypes = [vp, vp, vp, vp]
    lib.s2w_sht_inverse.argtypes = [vp, vp, vp, vp]
    lib.s2w_sht_inverse_static.argtypes = [vp, vp, vp, vp]
    lib.s2w_shard_layout.argtypes = [ctypes.c_int] * 6 + [ip] * 4
    for name in ("s2w_sht_inverse_columns", "s2w_sht_inverse_rings", "s2w_sht_forward_rings",
                 "s2w_sht_forward_columns"):
        getattr(lib, name).argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    lib.s2w_wigner_forward.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.s2w_wigner_inverse.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.s2w_check.argtypes = [vp]
    lib.s2w_ball_wav_plan_create.argtypes = [ctypes.POINTER(BallWavParams), vp, ctypes.POINTER(vp)]
    lib.s2w_ball_wav_plan_destroy.argtypes = [vp]
    lib.s2w_ball_wav_query_layout.argtypes = [vp, i64p, i64p, ip, ip, ip, i64p, ip, ip, ip]
    for name in ("s2w_ball_forward", "s2w_ball_inverse", "s2w_ball_forward_adjoint", "s2w_ball_inverse_adjoint"):
        getattr(lib, name).argtypes = [vp, vp, vp, vp, vp]
    lib.s2w_ball_wav_check.argtypes = [vp]
    lib.s2w_ball_wav_plan_autotune.argtypes = [vp, vp]
    lib.s2w_plan_autotune.argtypes = [vp, vp]
    lib.s2w_plan_launch_shapes.argtypes = [vp, ctypes.c_int, ip, ip, ip]
    lib.s2w_plan_dft_forms.argtypes = [vp, ctypes.c_int, ip, ip]
    lib.s2w_plan_set_dft_forms.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.s2w_plan_device_bytes.argtypes = [vp, i64p, i64p]
    lib.s2w_plan_inject_timeout.argtypes = [vp, ctypes.c_int]
    vpp = ctypes.POINTER(vp)
    lib.s2w_batch_create.argtypes = [vpp, ctypes.c_int, vpp, vpp, vpp, vpp, ctypes.c_int, vp, vpp]
    lib.s2w_batch_launch.argtypes = [vp, vp]
    lib.s2w_batch_destroy.argtypes = [vp]
    lib.s2w_last_error.restype = ctypes.c_char_p
    lib.s2w_version.restype = ctypes.c_char_p
    lib.s2w_trace_enable.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.s2w_trace_reset.argtypes = [vp]
    lib.s2w_trace_read.argtypes = [vp, ctypes.c_int, i64p, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]
    lib.s2w_ball_plan_create.argtypes = [ctypes.POINTER(BallParams), vp, ctypes.POINTER(vp)]
    lib.s2w_ball_plan_destroy.argtypes = [vp]
    lib.s2w_ball_nodes.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    for nm in ("s2w_laguerre_forward", "s2w_laguerre_inverse", "s2w_ball_sl_forward", "s2w_ball_sl_inverse"):
        getattr(lib, nm).argtypes = [vp, vp, vp, vp]
    lib.s2w_kernel_name.argtypes = [ctypes.c_int]
    lib.s2w_kernel_name.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("s2w_last_error", "s2w_version", "s2w_kernel_name"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise S2WError(status, _lib.s2w_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t, real: bool, name: str, need: int | None = None):
    """Device address of tensor t after checking what the kernels rely on: a contiguous CUDA
    tensor of the plan's element type on the CURRENT device (the library launches on the current
    device and indexes the buffer from its start) holding at least `need` elements (the sizes the
    C ABI's layouts give; the kernels would read or write past a smaller buffer)."""
    import torch
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {t.device}, but the current device is cuda:{torch.cuda.current_device()}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    want = torch.float64 if real else torch.complex128
    if t.dtype != want:
        raise ValueError(f"{name} must be {want}, got {t.dtype}")
    if need is not None and t.numel() < need:
        raise ValueError(f"{name} holds {t.numel()} elements, the plan needs {need}")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A transform plan: the parameters of Algorithm 1 plus the batch size.

    Parameters follow the paper's statement of the problem: band-limits L and N,
    dilation ``lam`` (lambda), lowest scale J0, spin, reality of the signal and the
    number of maps per call; ``sampling`` picks the grid (S2W_SAMPLING_MW or
    S2W_SAMPLING_DH).
    """

    def __init__(self, L: int, N: int, lam: float = 2.0, J0: int = 0, spin: int = 0,
                 reality: bool = False, batch: int = 1, precision: int = S2W_FP64, stream=None,
                 precompute: int = 0, sampling: int = 0):
        lib = load()
        self.params = Params(L, N, J0, spin, int(reality), batch, precision, int(precompute), float(lam),
                             int(sampling))
        self.sampling = int(sampling)
        h = ctypes.c_void_p()
        _check(lib.s2w_plan_create(ctypes.byref(self.params), _stream(stream), ctypes.byref(h)))
        self._h = h
        self.L, self.N, self.lam, self.J0, self.spin = L, N, lam, J0, spin
        self.real = bool(reality) and spin == 0
        self.batch = batch
        me, we, se = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        ns, lphi = ctypes.c_int(), ctypes.c_int()
        _check(lib.s2w_query_layout(h, ctypes.byref(me), ctypes.byref(we), ctypes.byref(se),
                                    ctypes.byref(ns), None, None, None, ctypes.byref(lphi)))
        n = ns.value
        offs = (ctypes.c_int64 * (n + 1))()
        Lj = (ctypes.c_int * n)()
        Nj = (ctypes.c_int * n)()
        _check(lib.s2w_query_layout(h, None, None, None, None, offs, Lj, Nj, None))
        self.map_elems, self.wav_elems, self.scal_elems = me.value, we.value, se.value
        self.nscales, self.L_phi = n, lphi.value
        self.wav_offsets = list(offs)
        self.Lj, self.Nj = list(Lj), list(Nj)
        self.Mc = L if self.real else 2 * L - 1
        self.R, self.R_phi = rings(L, self.sampling), rings(self.L_phi, self.sampling)

    # ------------------------------------------------------------------ buffers
    @property
    def dtype(self):
        import torch
        return torch.float64 if self.real else torch.complex128

    def empty_map(self, device="cuda"):
        import torch
        return torch.empty((self.batch, self.R, 2 * self.L - 1), dtype=self.dtype, device=device)

    def empty_wav(self, device="cuda"):
        import torch
        return torch.empty((self.batch, self.wav_elems), dtype=self.dtype, device=device)

    def empty_scal(self, device="cuda"):
        import torch
        return torch.empty((self.batch, self.R_phi, 2 * self.L_phi - 1), dtype=self.dtype, device=device)

    def empty_flm(self, device="cuda"):
        import torch
        return torch.empty((self.batch, self.L, self.Mc), dtype=torch.complex128, device=device)

    def scale_shape(self, s: int):
        return (2 * self.Nj[s] - 1, rings(self.Lj[s], self.sampling), 2 * self.Lj[s] - 1)

    def empty_flmn(self, s: int, device="cuda"):
        import torch
        Lj, Nj = self.Lj[s], self.Nj[s]
        Mcj = Lj if self.real else 2 * Lj - 1
        return torch.empty((self.batch, 2 * Nj - 1, Lj, Mcj), dtype=torch.complex128, device=device)

    def scale_view(self, wav, s: int):
        """View of scale index s of a [batch, wav_elems] tensor as [batch, 2N_j-1, R(L_j), 2L_j-1]."""
        a, b = self.wav_offsets[s], self.wav_offsets[s + 1]
        return wav[:, a:b].view(self.batch, *self.scale_shape(s))

    # ------------------------------------------------------------------ transforms
    # elements of each buffer a call reads or writes (the layouts of include/s2w.h)
    def _n_map(self):
        return self.batch * self.map_elems

    def _n_wav(self):
        return self.batch * self.wav_elems

    def _n_scal(self):
        return self.batch * self.scal_elems

    def _n_flm(self):
        return self.batch * self.L * self.Mc

    def _n_scale(self, s: int):
        if not 0 <= s < self.nscales:
            raise ValueError(f"scale index {s} out of range [0, {self.nscales})")
        return self.batch * (self.wav_offsets[s + 1] - self.wav_offsets[s])

    def _n_flmn(self, s: int):
        Lj, Nj = self.Lj[s], self.Nj[s]
        return self.batch * (2 * Nj - 1) * Lj * (Lj if self.real else 2 * Lj - 1)

    def forward(self, f, wav, scal, stream=None):
        _check(_lib.s2w_forward(self._h, _ptr(f, self.real, "f", self._n_map()),
                                _ptr(wav, self.real, "wav", self._n_wav()),
                                _ptr(scal, self.real, "scal", self._n_scal()), _stream(stream)))

    def inverse(self, wav, scal, f, stream=None):
        _check(_lib.s2w_inverse(self._h, _ptr(wav, self.real, "wav", self._n_wav()),
                                _ptr(scal, self.real, "scal", self._n_scal()),
                                _ptr(f, self.real, "f", self._n_map()), _stream(stream)))

    def forward_adjoint(self, gwav, gscal, gf, stream=None):
        """gf = A^H (gwav, gscal), A the analysis operator of forward()."""
        _check(_lib.s2w_forward_adjoint(self._h, _ptr(gwav, self.real, "gwav", self._n_wav()),
                                        _ptr(gscal, self.real, "gscal", self._n_scal()),
                                        _ptr(gf, self.real, "gf", self._n_map()), _stream(stream)))

    def inverse_adjoint(self, gf, gwav, gscal, stream=None):
        """(gwav, gscal) = S^H gf, S the synthesis operator of inverse()."""
        _check(_lib.s2w_inverse_adjoint(self._h, _ptr(gf, self.real, "gf", self._n_map()),
                                        _ptr(gwav, self.real, "gwav", self._n_wav()),
                                        _ptr(gscal, self.real, "gscal", self._n_scal()), _stream(stream)))

    def sht_forward(self, f, flm, stream=None):
        _check(_lib.s2w_sht_forward(self._h, _ptr(f, self.real, "f", self._n_map()),
                                    _ptr(flm, False, "flm", self._n_flm()), _stream(stream)))

    def sht_inverse(self, flm, f, stream=None):
        _check(_lib.s2w_sht_inverse(self._h, _ptr(flm, False, "flm", self._n_flm()),
                                    _ptr(f, self.real, "f", self._n_map()), _stream(stream)))

    def sht_inverse_static(self, flm, f, stream=None):
        """s2w_sht_inverse with its scratch in the library's fixed device array (allocates nothing)."""
        _check(_lib.s2w_sht_inverse_static(self._h, _ptr(flm, False, "flm", self._n_flm()),
                                           _ptr(f, self.real, "f", self._n_map()), _stream(stream)))

    # ---------------------------------------------- m-sharded spin SHT stages (include/s2w.h)
    def _n_cols(self):
        return self.batch * self.R * self.Mc

    def empty_cols(self, device="cuda"):
        """Column buffer [batch, R(L), Mc] of the sharded SHT stages."""
        import torch
        return torch.empty((self.batch, self.R, self.Mc), dtype=torch.complex128, device=device)

    def sht_inverse_columns(self, flm, cols, c_begin: int, c_end: int, stream=None):
        """flm -> columns [c_begin, c_end) of cols (column c holds m = c + m_min)."""
        _check(_lib.s2w_sht_inverse_columns(self._h, _ptr(flm, False, "flm", self._n_flm()),
                                            _ptr(cols, False, "cols", self._n_cols()), c_begin, c_end,
                                            _stream(stream)))

    def sht_inverse_rings(self, cols, f, ring_begin: int, ring_end: int, stream=None):
        """Rows [ring_begin, ring_end) of cols -> those rings of f."""
        _check(_lib.s2w_sht_inverse_rings(self._h, _ptr(cols, False, "cols", self._n_cols()),
                                          _ptr(f, self.real, "f", self._n_map()), ring_begin, ring_end,
                                          _stream(stream)))

    def sht_forward_rings(self, f, cols, ring_begin: int, ring_end: int, stream=None):
        """Rings [ring_begin, ring_end) of f -> those rows of cols."""
        _check(_lib.s2w_sht_forward_rings(self._h, _ptr(f, self.real, "f", self._n_map()),
                                          _ptr(cols, False, "cols", self._n_cols()), ring_begin, ring_end,
                                          _stream(stream)))

    def sht_forward_columns(self, cols, flm, c_begin: int, c_end: int, stream=None):
        """Columns [c_begin, c_end) of cols -> the coefficients of those m in flm."""
        _check(_lib.s2w_sht_forward_columns(self._h, _ptr(cols, False, "cols", self._n_cols()),
                                            _ptr(flm, False, "flm", self._n_flm()), c_begin, c_end,
                                            _stream(stream)))

    def wigner_forward(self, s: int, f, flmn, stream=None):
        _check(_lib.s2w_wigner_forward(self._h, s, _ptr(f, self.real, "f", self._n_scale(s)),
                                       _ptr(flmn, False, "flmn", self._n_flmn(s)), _stream(stream)))

    def wigner_inverse(self, s: int, flmn, f, stream=None):
        _check(_lib.s2w_wigner_inverse(self._h, s, _ptr(flmn, False, "flmn", self._n_flmn(s)),
                                       _ptr(f, self.real, "f", self._n_scale(s)), _stream(stream)))

    def check(self):
        _check(_lib.s2w_check(self._h))

    def inject_timeout(self, on: bool = True):
        """Failure-path test hook: the plan's tensor-core contraction waits run out (S2W_ETIMEOUT)."""
        _check(_lib.s2w_plan_inject_timeout(self._h, int(on)))

    # ------------------------------------------------------------------ runtime
    def autotune(self, stream=None):
        """Times the candidate launch shapes on this plan's shapes and keeps the fastest."""
        _check(_lib.s2w_plan_autotune(self._h, _stream(stream)))

    def launch_shapes(self, transform: int):
        """(DFT threads forward, DFT threads inverse, maps per block of the inverse contraction)
        of transform 0 (spin SHT), 1 (scaling function) or 2 + s (wavelet scale s)."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.s2w_plan_launch_shapes(self._h, transform, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def dft_forms(self, transform: int):
        """(forward, inverse) form of the azimuthal DFTs of a transform: 2 = tensor cores,
        prime-factor form; 1 = tensor cores, direct form; 0 = the precision mode's SIMT kernels
        (numbering as in launch_shapes)."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(_lib.s2w_plan_dft_forms(self._h, transform, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_dft_forms(self, transform: int, fwd: int, inv: int):
        """Forces the DFT forms of a transform (codes of dft_forms, -1 = default)."""
        _check(_lib.s2w_plan_set_dft_forms(self._h, transform, fwd, inv))

    def device_bytes(self):
        """(table bytes, workspace bytes) of device memory the plan holds."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.s2w_plan_device_bytes(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    # ------------------------------------------------------------------ tracing
    def trace(self, on: bool = True, capacity: int = 4096):
        _check(_lib.s2w_trace_enable(self._h, int(on), capacity))

    def trace_reset(self):
        _check(_lib.s2w_trace_reset(self._h))

    def trace_read(self):
        """{kernel name: (launches, device ms, algorithmic float64 ops)} since the last reset."""
        out = {}
        for k in range(KERNEL_KINDS):
            n, ms, fl = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
            _check(_lib.s2w_trace_read(self._h, k, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl)))
            out[_lib.s2w_kernel_name(k).decode()] = (n.value, ms.value, fl.value)
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.s2w_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BallPlan:
    """Fourier-Laguerre (Eqs. 6-8) and spherical-Laguerre (Eqs. 9-11) transforms of a batch of
    ball signals with angular band-limit L and radial band-limit P."""

    def __init__(self, L: int, P: int, tau: float = 1.0, spin: int = 0, reality: bool = False,
                 batch: int = 1, precision: int = S2W_FP64, stream=None, sampling: int = 0):
        lib = load()
        self.params = BallParams(L, P, spin, int(reality), batch, precision, float(tau), int(sampling))
        self.sampling, self.R = int(sampling), rings(L, int(sampling))
        h = ctypes.c_void_p()
        _check(lib.s2w_ball_plan_create(ctypes.byref(self.params), _stream(stream), ctypes.byref(h)))
        self._h = h
        self.L, self.P, self.tau, self.batch = L, P, tau, batch
        self.real = bool(reality) and spin == 0
        self.Mc = L if self.real else 2 * L - 1

    def nodes(self):
        import numpy as np
        r = (ctypes.c_double * self.P)()
        om = (ctypes.c_double * self.P)()
        _check(_lib.s2w_ball_nodes(self._h, r, om))
        return np.array(r[:]), np.array(om[:])

    def empty_coeffs(self, device="cuda"):
        import torch
        return torch.empty((self.batch, self.P, self.L, self.Mc), dtype=torch.complex128, device=device)

    def empty_pixels(self, device="cuda"):
        import torch
        dt = torch.float64 if self.real else torch.complex128
        return torch.empty((self.batch, self.P, self.R, 2 * self.L - 1), dtype=dt, device=device)

    def _n_coef(self):
        return self.batch * self.P * self.L * self.Mc

    def _n_pix(self):
        return self.batch * self.P * self.R * (2 * self.L - 1)

    def laguerre_forward(self, f_r, f_p, stream=None):
        _check(_lib.s2w_laguerre_forward(self._h, _ptr(f_r, False, "f_r", self._n_coef()),
                                         _ptr(f_p, False, "f_p", self._n_coef()), _stream(stream)))

    def laguerre_inverse(self, f_p, f_r, stream=None):
        _check(_lib.s2w_laguerre_inverse(self._h, _ptr(f_p, False, "f_p", self._n_coef()),
                                         _ptr(f_r, False, "f_r", self._n_coef()), _stream(stream)))

    def sl_forward(self, f, flmp, stream=None):
        _check(_lib.s2w_ball_sl_forward(self._h, _ptr(f, self.real, "f", self._n_pix()),
                                        _ptr(flmp, False, "flmp", self._n_coef()), _stream(stream)))

    def sl_inverse(self, flmp, f, stream=None):
        _check(_lib.s2w_ball_sl_inverse(self._h, _ptr(flmp, False, "flmp", self._n_coef()),
                                        _ptr(f, self.real, "f", self._n_pix()), _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            _lib.s2w_ball_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Transforms of several plans replayed as one CUDA graph (s2w_batch_*).  `what`: 0 analysis,
    1 synthesis, 2 both.  The tensors are bound at creation and must stay alive."""

    def __init__(self, plans, f=None, wav=None, scal=None, out=None, what: int = 2, stream=None):
        lib = load()
        n = len(plans)
        vp = ctypes.c_void_p

        sizes = {"f": lambda p: p._n_map(), "out": lambda p: p._n_map(), "wav": lambda p: p._n_wav(),
                 "scal": lambda p: p._n_scal()}

        def arr(ts, name):
            if ts is None:
                return None
            a = (vp * n)()
            for i, (t, p) in enumerate(zip(ts, plans)):
                a[i] = _ptr(t, p.real, name, sizes[name](p))
            return a
        self._keep = (list(plans), f, wav, scal, out)
        hp = (vp * n)(*[p._h for p in plans])
        h = vp()
        _check(lib.s2w_batch_create(hp, n, arr(f, "f"), arr(wav, "wav"), arr(scal, "scal"), arr(out, "out"), what,
                                    _stream(stream), ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(_lib.s2w_batch_launch(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            _lib.s2w_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BallWavPlan:
    """Directional wavelet transform on the ball (Sec. 3.2, Algorithm 2) of a batch of spin-0
    fields with angular band-limit L, radial band-limit P and N directions."""

    def __init__(self, L: int, N: int, P: int, lam: float = 2.0, nu: float = 2.0, J0: int = 0, J0r: int = 0,
                 tau: float = 1.0, reality: bool = True, batch: int = 1, precision: int = S2W_FP64,
                 precompute: int = 0, stream=None, sampling: int = 0):
        lib = load()
        self.params = BallWavParams(L, N, P, J0, J0r, 0, int(reality), batch, precision, int(precompute),
                                    float(lam), float(nu), float(tau), int(sampling))
        self.sampling, self.R = int(sampling), rings(L, int(sampling))
        h = ctypes.c_void_p()
        _check(lib.s2w_ball_wav_plan_create(ctypes.byref(self.params), _stream(stream), ctypes.byref(h)))
        self._h = h
        self.L, self.N, self.P, self.batch = L, N, P, batch
        self.real = bool(reality)
        fe, we, ns = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(lib.s2w_ball_wav_query_layout(h, ctypes.byref(fe), ctypes.byref(we), ctypes.byref(ns),
                                             None, None, None, None, None, None))
        n = ns.value
        arr = lambda t, k: (t * k)()   # noqa: E731
        j, jr, Lj, Nj, Pj = arr(ctypes.c_int, n), arr(ctypes.c_int, n), arr(ctypes.c_int, n), arr(ctypes.c_int, n), \
            arr(ctypes.c_int, n)
        offs = arr(ctypes.c_int64, n + 1)
        _check(lib.s2w_ball_wav_query_layout(h, None, None, None, j, jr, offs, Lj, Nj, Pj))
        self.field_elems, self.wav_elems, self.nscales = fe.value, we.value, n
        self.scales = [(j[k], jr[k]) for k in range(n)]
        self.Lj, self.Nj, self.Pj = list(Lj), list(Nj), list(Pj)
        self.wav_offsets = list(offs)

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.real else torch.complex128

    def empty_field(self, device="cuda"):
        import torch
        return torch.empty((self.batch, self.P, self.R, 2 * self.L - 1), dtype=self.dtype, device=device)

    def empty_wav(self, device="cuda"):
        import torch
        return torch.empty((self.wav_elems,), dtype=self.dtype, device=device)

    def scale_view(self, wav, k: int):
        """Block k of the wavelet coefficients as [batch, P_j', 2N_j-1, R(L_j), 2L_j-1]."""
        a, b = self.wav_offsets[k], self.wav_offsets[k + 1]
        return wav[a:b].view(self.batch, self.Pj[k], 2 * self.Nj[k] - 1, rings(self.Lj[k], self.sampling),
                             2 * self.Lj[k] - 1)

    def _n_field(self):
        return self.batch * self.field_elems

    def forward(self, f, wav, scal, stream=None):
        nf = self._n_field()
        _check(_lib.s2w_ball_forward(self._h, _ptr(f, self.real, "f", nf), _ptr(wav, self.real, "wav", self.wav_elems),
                                     _ptr(scal, self.real, "scal", nf), _stream(stream)))

    def inverse(self, wav, scal, f, stream=None):
        nf = self._n_field()
        _check(_lib.s2w_ball_inverse(self._h, _ptr(wav, self.real, "wav", self.wav_elems),
                                     _ptr(scal, self.real, "scal", nf), _ptr(f, self.real, "f", nf), _stream(stream)))

    def forward_adjoint(self, gwav, gscal, gf, stream=None):
        nf = self._n_field()
        _check(_lib.s2w_ball_forward_adjoint(self._h, _ptr(gwav, self.real, "gwav", self.wav_elems),
                                             _ptr(gscal, self.real, "gscal", nf), _ptr(gf, self.real, "gf", nf),
                                             _stream(stream)))

    def inverse_adjoint(self, gf, gwav, gscal, stream=None):
        nf = self._n_field()
        _check(_lib.s2w_ball_inverse_adjoint(self._h, _ptr(gf, self.real, "gf", nf),
                                             _ptr(gwav, self.real, "gwav", self.wav_elems),
                                             _ptr(gscal, self.real, "gscal", nf), _stream(stream)))

    def check(self):
        _check(_lib.s2w_ball_wav_check(self._h))

    def autotune(self, stream=None):
        """s2w_ball_wav_plan_autotune: launch shapes and DFT forms of the sphere transforms."""
        _check(_lib.s2w_ball_wav_plan_autotune(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            _lib.s2w_ball_wav_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version() -> str:
    return load().s2w_version().decode()
