"""ctypes binding of liblo_afqmc.so (argument marshalling only).

Every function here forwards to the C ABI declared in include/lo_afqmc.h.
Arrays may be numpy arrays (host memory) or CUDA torch tensors (device
memory on the context's device); their data pointers are passed as they are.
No arithmetic of the method happens in Python.  The shared library must have
been built (``python -m paper_2202_00832_b300.build``); loading fails loudly
otherwise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblo_afqmc.so")

MODE_FULL, MODE_LO, MODE_LO_JK = 0, 1, 2
PREC_FP64, PREC_FP16X3, PREC_BF16X3, PREC_FP16X3_F64INV, PREC_TF32 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": PREC_FP64, "fp16x3": PREC_FP16X3, "bf16x3": PREC_BF16X3,
              "fp16x3_f64inv": PREC_FP16X3_F64INV, "tf32": PREC_TF32}
MODES = {"full": MODE_FULL, "lo": MODE_LO, "lo_jk": MODE_LO_JK}

STATUS = {0: "LOAF_OK", 1: "LOAF_ERR_ARG", 2: "LOAF_ERR_SHAPE", 3: "LOAF_ERR_CUDA",
          4: "LOAF_ERR_OOM", 5: "LOAF_ERR_SINGULAR", 6: "LOAF_ERR_NOT_READY",
          7: "LOAF_ERR_TIMEOUT", 8: "LOAF_ERR_NAN", 9: "LOAF_ERR_UNSUPPORTED"}

# (name, restype, argtypes) of every exported entry point
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = [
    ("loaf_create", _I, [ctypes.POINTER(_P), _I, _P]),
    ("loaf_destroy", _I, [_P]),
    ("loaf_status_str", ctypes.c_char_p, [_I]),
    ("loaf_last_error", ctypes.c_char_p, [_P]),
    ("ao_load_cholesky", _I, [_P, _I, _I, _P, _P, _I, _I, _P, _P, _D, _I]),
    ("lo_localize_compress", _I, [_P, _D, _P, _I, _I, _P, _P]),
    ("walkers_energy", _I, [_P, _I, _P, _I, _I, _P, _P, _P]),
    ("walkers_energy_submit", _I, [_P, _I, _P, _I, _I, _P, _P, _P]),
    ("walkers_energy_wait", _I, [_P]),
    ("walkers_energy_multi", _I, [_P, _I, _P, _P, _I, _I, _P, _P, _P, _I, _P]),
    ("walkers_theta", _I, [_P, _I, _P, _P, _P, _P]),
    ("walkers_force_bias", _I, [_P, _I, _P, _I, _P, _P, _P]),
    ("walkers_propagator", _I, [_P, _I, _P, _I, _P]),
    ("walkers_energy_cas", _I, [_P, _I, _I, _P, _I, _P, _P, _P, _P, _P]),
    ("walkers_pair_exchange", _I, [_P, _I, _P, _I, _P]),
    ("loaf_num_pairs", _I, [_P]),
    ("lo_get_localized_trial", _I, [_P, _I, _P]),
    ("walkers_theta_noalloc", _I, [_P, _I, _P, _P, _P, _P]),
    ("loaf_screen_num_params", _I, []),
    ("pair_screen_train", _I, [_P, _I, _P, _I, ctypes.c_float, _P, _P]),
    ("pair_screen_set", _I, [_P, _D, _P]),
    ("pair_screen_query", _I, [_P, _P, _P, _P, _P, _P]),
    ("mlp_loss_grad", _I, [_I, _I, _P, _P, _P, _P, _P]),
    ("loaf_test_withhold_stage", _I, [_P, _I]),
    ("loaf_set_tiles", _I, [_P, _I, _I]),
    ("loaf_get_tiles", _I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    ("loaf_profile", _I, [_P, _I]),
    ("loaf_profile_count", _I, [_P]),
    ("loaf_profile_get", _I, [_P, _I, ctypes.POINTER(ctypes.c_char_p),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_long),
                              ctypes.POINTER(ctypes.c_long)]),
]

_lib = None


class LoafError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


def load_library(path: str = LIB_PATH):
    """Load (once) and return the shared library; raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with "
                           "`python -m paper_2202_00832_b300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a) -> Optional[int]:
    """Data pointer of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)!r}")


def _check_dtype(a, kind: str):
    if a is None:
        return
    if isinstance(a, np.ndarray):
        want = {"f8": np.float64, "c16": np.complex128, "i4": np.int32}[kind]
        if a.dtype != want:
            raise TypeError(f"expected {np.dtype(want)}, got {a.dtype}")
    else:
        import torch
        want = {"f8": torch.float64, "c16": torch.complex128, "i4": torch.int32}[kind]
        if a.dtype != want:
            raise TypeError(f"expected {want}, got {a.dtype}")


class Context:
    """One loaf_ctx: a loaded system on one device and its workspace."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        lib = load_library()
        self._lib = lib
        h = _P()
        self._check(lib.loaf_create(ctypes.byref(h), device, stream), "loaf_create", None)
        self._h = h
        self.M = self.X = self.n_alpha = self.n_beta = 0
        self.closed = True

    def _check(self, code: int, where: str, h=...):
        if code != 0:
            handle = self._h if h is ... else h
            msg = self._lib.loaf_last_error(handle).decode() if handle else ""
            raise LoafError(code, where, msg)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.loaf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- setup ------------------------------------------------------------
    def ao_load_cholesky(self, h, L, trial_a, trial_b=None, e0: float = 0.0,
                         on_device: bool = False):
        for a in (h, L, trial_a, trial_b):
            _check_dtype(a, "f8")
        M = int(h.shape[0])
        X = int(L.shape[0])
        na = int(trial_a.shape[1])
        nb = int(trial_b.shape[1]) if trial_b is not None else na
        self._check(self._lib.ao_load_cholesky(self._h, M, X, _ptr(h), _ptr(L), na, nb,
                                               _ptr(trial_a), _ptr(trial_b), float(e0),
                                               int(on_device)), "ao_load_cholesky")
        self.M, self.X, self.n_alpha, self.n_beta = M, X, na, nb
        self.closed = trial_b is None
        return self

    def load_molecule(self, mol, e0: float = 0.0):
        """Load a synthetic molecule (closed shells use one restricted trial)."""
        return self.ao_load_cholesky(mol.h, mol.L, mol.trial_a,
                                     None if mol.closed_shell else mol.trial_b, e0)

    def lo_localize_compress(self, t_svd: float, r_ops: Optional[np.ndarray] = None,
                             localize: bool = True):
        """Returns (compression_pct, m_svd_per_pair)."""
        n_ops = 0
        if r_ops is not None:
            _check_dtype(r_ops, "f8")
            n_ops = int(r_ops.shape[0])
        npairs = self.n_alpha * (self.n_alpha + 1) // 2
        if not self.closed:
            npairs += self.n_beta * (self.n_beta + 1) // 2
        pct = ctypes.c_double(0.0)
        msvd = np.zeros(npairs, dtype=np.int32)
        self._check(self._lib.lo_localize_compress(self._h, float(t_svd), _ptr(r_ops), n_ops,
                                                   int(localize), ctypes.byref(pct), _ptr(msvd)),
                    "lo_localize_compress")
        return pct.value, msvd

    def localized_trial(self, spin: int = 0) -> np.ndarray:
        n = self.n_alpha if spin == 0 else self.n_beta
        out = np.zeros((self.M, n))
        self._check(self._lib.lo_get_localized_trial(self._h, spin, _ptr(out)),
                    "lo_get_localized_trial")
        return out

    @property
    def num_pairs(self) -> int:
        return int(self._lib.loaf_num_pairs(self._h))

    @property
    def ntot(self) -> int:
        return self.n_alpha if self.closed else self.n_alpha + self.n_beta

    def test_withhold_stage(self, n: int = 1):
        """Failure-path test hook: the next n LO tensor-core launches leave one
        pipeline stage unfilled, so their bounded waits run out (LOAF_ERR_TIMEOUT)."""
        self._check(self._lib.loaf_test_withhold_stage(self._h, int(n)), "loaf_test_withhold_stage")

    # -- tile shapes ----------------------------------------------------------
    def set_tiles(self, lo_chunk_cap: int = 256, coulomb_split: int = 0):
        """Largest LO chunk (the MMA's N, a multiple of 32 in [64, 256]) and the
        Coulomb k-split (0: the library's rule) of this context's kernels."""
        self._check(self._lib.loaf_set_tiles(self._h, int(lo_chunk_cap), int(coulomb_split)),
                    "loaf_set_tiles")

    def tiles(self) -> tuple:
        """(lo_chunk_cap, coulomb_split) in use (split 0: the library's rule)."""
        cap, split = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.loaf_get_tiles(self._h, ctypes.byref(cap), ctypes.byref(split)),
                    "loaf_get_tiles")
        return cap.value, split.value

    # -- stage timers ---------------------------------------------------------
    def profile(self, enable: bool = True):
        """Enable (and reset) or disable the per-stage CUDA-event timers."""
        self._check(self._lib.loaf_profile(self._h, int(enable)), "loaf_profile")

    def profile_read(self) -> dict:
        """{stage: (total_ms, calls, kernel_launches)} since profile(True)."""
        out = {}
        for k in range(self._lib.loaf_profile_count(self._h)):
            name = ctypes.c_char_p()
            ms = ctypes.c_double()
            calls = ctypes.c_long()
            launches = ctypes.c_long()
            self._check(self._lib.loaf_profile_get(self._h, k, ctypes.byref(name),
                                                   ctypes.byref(ms), ctypes.byref(calls),
                                                   ctypes.byref(launches)), "loaf_profile_get")
            out[name.value.decode()] = (ms.value, calls.value, launches.value)
        return out

    # -- hot path -----------------------------------------------------------
    def walkers_energy(self, phi, mode="lo", precision="fp64", e_out=None, logdet_out=None,
                       walker_status=None, raise_on_singular: bool = True):
        """Energies of W walkers.  Host arrays in -> host arrays out by default."""
        _check_dtype(phi, "c16")
        W = int(phi.shape[0])
        if e_out is None:
            e_out = np.zeros(W, dtype=np.complex128)
        if logdet_out is None and isinstance(phi, np.ndarray):
            logdet_out = np.zeros(W, dtype=np.complex128)
        if walker_status is None and isinstance(phi, np.ndarray):
            walker_status = np.zeros(W, dtype=np.int32)
        code = self._lib.walkers_energy(self._h, W, _ptr(phi), MODES.get(mode, mode),
                                        PRECISIONS.get(precision, precision), _ptr(e_out),
                                        _ptr(logdet_out), _ptr(walker_status))
        if code == 5 and not raise_on_singular:
            return e_out, logdet_out, walker_status
        self._check(code, "walkers_energy")
        return e_out, logdet_out, walker_status

    def walkers_energy_submit(self, phi, e_out, logdet_out=None, walker_status=None, mode="lo",
                              precision="fp16x3"):
        """Queue walkers_energy on phi (pinned host or device) into the given
        output buffers and return; the buffers are held until walkers_energy_wait."""
        _check_dtype(phi, "c16")
        _check_dtype(e_out, "c16")
        _check_dtype(logdet_out, "c16")
        _check_dtype(walker_status, "i4")
        W = int(phi.shape[0])
        code = self._lib.walkers_energy_submit(self._h, W, _ptr(phi), MODES.get(mode, mode),
                                               PRECISIONS.get(precision, precision), _ptr(e_out),
                                               _ptr(logdet_out), _ptr(walker_status))
        self._check(code, "walkers_energy_submit")
        if not hasattr(self, "_inflight"):
            self._inflight = []
        self._inflight.append((phi, e_out, logdet_out, walker_status))

    def walkers_energy_wait(self, raise_on_singular: bool = True):
        """Wait for every submitted call; returns the status code (0 or a
        walker failure when raise_on_singular is False)."""
        code = self._lib.walkers_energy_wait(self._h)
        self._inflight = []
        if code in (5, 8) and not raise_on_singular:
            return code
        self._check(code, "walkers_energy_wait")
        return code

    def walkers_propagator(self, x, precision="fp64", out=None):
        """V_w = sum_g x_wg L_g for fields x (W x X complex128): W x M x M complex128."""
        _check_dtype(x, "c16")
        W = int(x.shape[0])
        if out is None:
            out = np.zeros((W, self.M, self.M), dtype=np.complex128)
        self._check(self._lib.walkers_propagator(self._h, W, _ptr(x), PRECISIONS.get(precision, precision),
                                                 _ptr(out)), "walkers_propagator")
        return out

    def walkers_energy_cas(self, phi, dets, coeffs, e_out=None, logov_out=None, walker_status=None):
        """Mixed-estimate energy with a CAS trial (the context's trial = the CAS
        orbitals): phi W x M x N complex128, dets n_det x N int32 (dets[0] the
        reference), coeffs n_det float64.  Returns (E, log overlap, status)."""
        _check_dtype(phi, "c16")
        W, N = int(phi.shape[0]), int(phi.shape[2])
        dets = np.ascontiguousarray(dets, dtype=np.int32)
        coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
        if e_out is None:
            e_out = np.zeros(W, dtype=np.complex128)
        if logov_out is None and isinstance(phi, np.ndarray):
            logov_out = np.zeros(W, dtype=np.complex128)
        if walker_status is None and isinstance(phi, np.ndarray):
            walker_status = np.zeros(W, dtype=np.int32)
        self._check(self._lib.walkers_energy_cas(self._h, W, N, _ptr(phi), int(dets.shape[0]), _ptr(dets),
                                                 _ptr(coeffs), _ptr(e_out), _ptr(logov_out),
                                                 _ptr(walker_status)), "walkers_energy_cas")
        return e_out, logov_out, walker_status

    def walkers_force_bias(self, phi, precision="fp64", out=None, logdet_out=None,
                           walker_status=None):
        """<L_g>_w = sum_sigma tr(Lbar^sigma_g Theta^sigma), W x X complex128."""
        _check_dtype(phi, "c16")
        W = int(phi.shape[0])
        if out is None:
            out = np.zeros((W, self.X), dtype=np.complex128)
        if logdet_out is None and isinstance(phi, np.ndarray):
            logdet_out = np.zeros(W, dtype=np.complex128)
        if walker_status is None and isinstance(phi, np.ndarray):
            walker_status = np.zeros(W, dtype=np.int32)
        self._check(self._lib.walkers_force_bias(self._h, W, _ptr(phi), PRECISIONS.get(precision, precision),
                                                 _ptr(out), _ptr(logdet_out), _ptr(walker_status)),
                    "walkers_force_bias")
        return out, logdet_out, walker_status

    def walkers_theta(self, phi, theta_out=None, logdet_out=None, walker_status=None,
                      raise_on_singular: bool = True):
        _check_dtype(phi, "c16")
        W = int(phi.shape[0])
        if theta_out is None:
            theta_out = np.zeros((W, self.ntot, self.M), dtype=np.complex128)
        if logdet_out is None:
            logdet_out = np.zeros(W, dtype=np.complex128)
        if walker_status is None:
            walker_status = np.zeros(W, dtype=np.int32)
        code = self._lib.walkers_theta(self._h, W, _ptr(phi), _ptr(theta_out), _ptr(logdet_out),
                                       _ptr(walker_status))
        if code == 5 and not raise_on_singular:
            return theta_out, logdet_out, walker_status
        self._check(code, "walkers_theta")
        return theta_out, logdet_out, walker_status

    def walkers_theta_noalloc(self, phi, theta_out, logdet_out=None, walker_status=None):
        """walkers_theta with device buffers only and no device allocation.

        For callers that cannot allocate during the call; scratch comes from a
        fixed 32 MiB array in the library (W * Ntot * M <= 2,086,912, W <= 4096).
        Asynchronous on the context stream; singular walkers show up only in
        walker_status.
        """
        _check_dtype(phi, "c16")
        W = int(phi.shape[0])
        self._check(self._lib.walkers_theta_noalloc(self._h, W, _ptr(phi), _ptr(theta_out),
                                                    _ptr(logdet_out), _ptr(walker_status)),
                    "walkers_theta_noalloc")
        return theta_out, logdet_out, walker_status

    # -- learned pair screen ------------------------------------------------
    def pair_screen_train(self, phi, init_params, epochs=500, lr=3e-3):
        """Train the screen on walkers phi; returns the loss history."""
        _check_dtype(phi, "c16")
        init = np.ascontiguousarray(init_params, dtype=np.float32)
        hist = np.zeros(epochs, dtype=np.float32)
        self._check(self._lib.pair_screen_train(self._h, int(phi.shape[0]), _ptr(phi), int(epochs),
                                                float(lr), _ptr(init), _ptr(hist)),
                    "pair_screen_train")
        return hist

    def pair_screen_set(self, cutoff_ha: float) -> int:
        kept = ctypes.c_int(0)
        self._check(self._lib.pair_screen_set(self._h, float(cutoff_ha), ctypes.byref(kept)),
                    "pair_screen_set")
        return kept.value

    def pair_screen_query(self, trained: bool = True) -> dict:
        n = self.num_pairs
        out = {"features": np.zeros((n, 8)), "keep": np.zeros(n, dtype=np.uint8)}
        if trained:
            out.update(params=np.zeros(self._lib.loaf_screen_num_params(), dtype=np.float32),
                       pred=np.zeros(n), target=np.zeros(n))
        self._check(self._lib.pair_screen_query(
            self._h, _ptr(out.get("params")), _ptr(out["features"]), _ptr(out.get("pred")),
            _ptr(out.get("target")), _ptr(out["keep"])), "pair_screen_query")
        return out

    def walkers_pair_exchange(self, phi, precision="fp64", out=None):
        _check_dtype(phi, "c16")
        W = int(phi.shape[0])
        if out is None:
            out = np.zeros((self.num_pairs, W), dtype=np.complex128)
        self._check(self._lib.walkers_pair_exchange(self._h, W, _ptr(phi),
                                                    PRECISIONS.get(precision, precision),
                                                    _ptr(out)), "walkers_pair_exchange")
        return out


def mlp_loss_grad(x, t, params, device: int = 0):
    """(loss, gradient) of the screening network on the GPU (float32 in/out)."""
    lib = load_library()
    x = np.ascontiguousarray(x, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    params = np.ascontiguousarray(params, dtype=np.float32)
    g = np.zeros(lib.loaf_screen_num_params(), dtype=np.float32)
    loss = ctypes.c_float(0.0)
    code = lib.mlp_loss_grad(device, int(len(t)), _ptr(x), _ptr(t), _ptr(params),
                             ctypes.byref(loss), _ptr(g))
    if code != 0:
        raise LoafError(code, "mlp_loss_grad", "")
    return float(loss.value), g


def walkers_energy_multi(ctxs, phis, e_outs, logdet_outs=None, statuses=None, mode="lo",
                         precision="fp16x3", autotune: bool = True):
    """Energies of several systems in one graph launch (device tensors only).
    Returns the SM budget chosen for each system (0 = the whole GPU); with
    autotune the tile shapes chosen per system are read by Context.tiles()."""
    lib = load_library()
    n = len(ctxs)
    for a in phis:
        _check_dtype(a, "c16")
    arr = lambda vals, typ=_P: (typ * n)(*vals)
    caps = (ctypes.c_int * n)()
    W = arr([int(a.shape[0]) for a in phis], ctypes.c_int)
    ld = arr([_ptr(a) for a in logdet_outs]) if logdet_outs is not None else None
    st = arr([_ptr(a) for a in statuses]) if statuses is not None else None
    code = lib.walkers_energy_multi(arr([c._h for c in ctxs]), n, W, arr([_ptr(a) for a in phis]),
                                    MODES.get(mode, mode), PRECISIONS.get(precision, precision),
                                    arr([_ptr(a) for a in e_outs]), ld, st, int(bool(autotune)), caps)
    if code != 0:
        msg = lib.loaf_last_error(ctxs[0]._h).decode()
        raise LoafError(code, "walkers_energy_multi", msg)
    return list(caps)


def init_screen_params(seed: int = 0) -> np.ndarray:
    """Seeded Glorot-uniform initial weights (zero biases) for the screen."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in [(64, 8), (64, 64), (1, 64)]:
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-lim, lim, fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def position_operators(mol) -> np.ndarray:
    """diag(x), diag(y), diag(z) of the orbital centres (orthonormal synthetic basis)."""
    pos = mol.orbital_pos
    return np.ascontiguousarray(np.stack([np.diag(pos[:, d]) for d in range(3)]))
