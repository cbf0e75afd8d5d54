"""Python binding of libemc (include/emc.h): argument marshalling only.

Every step of the EMC hot path runs in the CUDA library; this module turns
torch tensors into device pointers and streams, allocates the caller-owned
buffers the ABI asks for, and raises on a non-zero status. There is no CPU
fallback: if libemc.so is missing or no GPU is present, calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libemc.so")

PREC_FP32, PREC_BF16, PREC_BF16_SPLIT, PREC_FP16_SPLIT = 0, 1, 2, 3
PRECISIONS = {"fp32": PREC_FP32, "bf16": PREC_BF16, "bf16_split": PREC_BF16_SPLIT,
              "fp16_split": PREC_FP16_SPLIT}
COMPRESS_DEFERRED, COMPRESS_IDW = 0, 1
FLAG_STORE_SCORES = 1
FLAG_SPARSE_K = 2
FLAG_WIDE_COUNTS = 4
FLAG_DENSE_ESTEP = 8
MODEL_POISSON, MODEL_GAUSSIAN, MODEL_POISSON_FLUENCE = 0, 1, 2
MODELS = {"poisson": MODEL_POISSON, "gaussian": MODEL_GAUSSIAN,
          "poisson_fluence": MODEL_POISSON_FLUENCE}

_lock = threading.Lock()
_lib = None


class EmcError(RuntimeError):
    pass


class Config(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("n_pix", ctypes.c_int64), ("n_rot", ctypes.c_int64),
                ("n_data", ctypes.c_int64), ("w_floor", ctypes.c_double),
                ("compress_mode", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("rot_chunk", ctypes.c_int64), ("n_cand", ctypes.c_int32),
                ("model", ctypes.c_int32), ("sigma", ctypes.c_double)]


class BufferSizes(ctypes.Structure):
    _fields_ = [("ld_pix", ctypes.c_int64), ("ld_data", ctypes.c_int64), ("rows", ctypes.c_int64),
                ("logw_bytes", ctypes.c_size_t), ("bias_bytes", ctypes.c_size_t),
                ("prob_bytes", ctypes.c_size_t), ("num_bytes", ctypes.c_size_t),
                ("den_bytes", ctypes.c_size_t), ("lse_bytes", ctypes.c_size_t),
                ("score_bytes", ctypes.c_size_t), ("grid_bytes", ctypes.c_size_t)]


class IterStats(ctypes.Structure):
    _fields_ = [("loglik", ctypes.c_double), ("ms_expand", ctypes.c_double),
                ("ms_loglik", ctypes.c_double), ("ms_normalize", ctypes.c_double),
                ("ms_update", ctypes.c_double), ("ms_compress", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("device_status", ctypes.c_int32),
                ("kernels", ctypes.c_int32), ("pass1_tiles", ctypes.c_int64),
                ("pass1_exact", ctypes.c_int64), ("pass1_pruned", ctypes.c_int32),
                ("pass1_delta", ctypes.c_int32), ("pass1_bound_pairs", ctypes.c_int64)]


_vp, _i64, _i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); every entry point declared in include/emc.h
_SIGS = {
    "emc_status_string": (ctypes.c_char_p, [_i32]),
    "emc_quat_count": (_i64, [_i32]),
    "emc_quat_generate": (_i64, [_i32, _i32, _dp, _dp, _i64]),
    "emc_buffer_sizes_for": (_i32, [ctypes.POINTER(Config), _i64, ctypes.POINTER(BufferSizes)]),
    "emc_workspace_size": (_i32, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_size_t)]),
    "emc_ctx_create": (_i32, [ctypes.POINTER(Config), _dp, _dp, _dp, _vp, ctypes.c_size_t, _vp,
                              ctypes.POINTER(_vp)]),
    "emc_ctx_destroy": (_i32, [_vp]),
    "emc_ctx_status": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "emc_ctx_set_wait_limit": (_i32, [_vp, ctypes.c_uint64, _i32]),
    "emc_set_frames": (_i32, [_vp, _vp, _i64, _vp]),
    "emc_expand": (_i32, [_vp, _vp, _i64, _i64, _vp, _vp, _vp]),
    "emc_loglik": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp, _i32, _vp, _vp]),
    "emc_normalize": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp]),
    "emc_update": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "emc_compress": (_i32, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i32, _vp]),
    "emc_finalize": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "emc_iteration": (_i32, [_vp, _vp, _vp, ctypes.POINTER(IterStats), _vp]),
    "emc_loglik_static": (_i32, [ctypes.POINTER(Config), _vp, _vp, _vp, _i64, _vp, _vp, _i32,
                                 _vp, _vp]),
    "emc_features": (_i32, [_vp, _vp, _vp]),
    "emc_mlp_param_count": (_i64, [_i64]),
    "emc_mlp_work_size": (_i32, [_i64, _i64, ctypes.POINTER(ctypes.c_size_t)]),
    "emc_mlp_forward": (_i32, [_i64, _vp, _vp, _i64, _vp, _vp, _vp]),
    "emc_mlp_train_step": (_i32, [_i64, _vp, _vp, _vp, _vp, _i32, ctypes.c_float, _vp, _vp, _vp,
                                  _i64, _i32, _vp, _vp, _vp]),
    "emc_loglik_sparse_k": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp, _i32, _vp]),
    "emc_merge_candidates": (_i32, [_vp, _i32, _vp, _i32, _i64, _i32, _vp, _vp]),
    "emc_topm": (_i32, [_vp, _i64, _i64, _i64, _i32, _vp, _vp]),
    "emc_targets_from_scores": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp]),
    "emc_set_candidates": (_i32, [_vp, _vp, _vp]),
    "emc_sparse_estep": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "emc_sparse_update": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "emc_sparse_iteration": (_i32, [_vp, _vp, _vp, ctypes.POINTER(IterStats), _vp]),
    "emc_missed_mass": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "emc_iteration_lse": (_i32, [_vp, _vp, _vp]),
    "emc_responsibilities": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "emc_collect_bytes": (ctypes.c_size_t, [_vp, _i64]),
    "emc_set_collect": (_i32, [_vp, _vp, _i64]),
    "emc_collected_targets": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp]),
}


def lib():
    """Load libemc.so (built in-tree by ``paper_1409_4256_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise EmcError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1409_4256_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().emc_status_string(code).decode()


def _check(code: int, what: str):
    if code != 0:
        raise EmcError(f"{what}: {status_string(code)} ({code})")


def quat_count(n: int) -> int:
    return int(lib().emc_quat_count(n))


def quat_generate(n: int, uniform: bool = False):
    """Eq. 2.7 sampling from the library: (quat[M_rot, 4], weight[M_rot])."""
    m = quat_count(n)
    quat = np.empty((m, 4), dtype=np.float64)
    w = np.empty(m, dtype=np.float64)
    r = lib().emc_quat_generate(n, int(uniform), quat.ctypes.data_as(_dp), w.ctypes.data_as(_dp), m)
    if r != m:
        raise EmcError(f"emc_quat_generate returned {r}, expected {m}")
    return quat, w


def loglik_static(cfg: Config, L, bias, frames, nrot: int, lse_m, lse_s,
                  accumulate: bool = False, device_status=None, stream=None) -> None:
    """emc_loglik_static: E-step pass 1 with no context, no workspace and no
    device allocation (its scratch is a static array inside the library)."""
    _check(lib().emc_loglik_static(ctypes.byref(cfg), _ptr(L), _ptr(bias), _ptr(frames), nrot,
                                   _ptr(lse_m), _ptr(lse_s), int(accumulate),
                                   _ptr(device_status), _stream(stream)), "emc_loglik_static")


def mlp_param_count(n_out: int) -> int:
    r = int(lib().emc_mlp_param_count(n_out))
    if r < 0:
        raise EmcError(f"emc_mlp_param_count: {status_string(r)}")
    return r


def mlp_work_size(n_out: int, batch: int) -> int:
    nb = ctypes.c_size_t()
    _check(lib().emc_mlp_work_size(n_out, batch, ctypes.byref(nb)), "emc_mlp_work_size")
    return int(nb.value)


def mlp_forward(n_out: int, params, X, batch: int, work, logits, stream=None) -> None:
    _check(lib().emc_mlp_forward(n_out, _ptr(params), _ptr(X), batch, _ptr(work), _ptr(logits),
                                 _stream(stream)), "emc_mlp_forward")


def mlp_train_step(n_out: int, params, grads, m, v, step: int, lr: float, X, tidx, tprob,
                   batch: int, R: int, work, loss, stream=None) -> None:
    _check(lib().emc_mlp_train_step(n_out, _ptr(params), _ptr(grads), _ptr(m), _ptr(v), step, lr,
                                    _ptr(X), _ptr(tidx), _ptr(tprob), batch, R, _ptr(work),
                                    _ptr(loss), _stream(stream)), "emc_mlp_train_step")


def topm(logits, batch: int, n: int, ld: int, M: int, cand, stream=None) -> None:
    _check(lib().emc_topm(_ptr(logits), batch, n, ld, M, _ptr(cand), _stream(stream)), "emc_topm")


def merge_candidates(first, rest, M: int, out=None, stream=None):
    """first int32 [n, R] (or None), rest int32 [n, M_rest >= M] -> int32 [n, M]."""
    import torch
    n = rest.shape[0]
    if out is None:
        out = torch.empty((n, M), dtype=torch.int32, device=rest.device)
    R = 0 if first is None else first.shape[1]
    _check(lib().emc_merge_candidates(_ptr(first), R, _ptr(rest), rest.shape[1], n, M, _ptr(out),
                                      _stream(stream)), "emc_merge_candidates")
    return out


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Context:
    """An emc_ctx plus its caller-owned workspace (a torch uint8 tensor).

    model: "poisson", "poisson_fluence" or "gaussian"; dense_estep=True sets
    EMC_FLAG_DENSE_ESTEP (emc_iteration then contracts every pass-1 tile)."""

    def __init__(self, N: int, q: np.ndarray, quat: np.ndarray, weight: np.ndarray, n_data: int,
                 precision=None, w_floor: float = 1e-10, compress_mode: int = 0,
                 rot_chunk: int = 0, store_scores: bool = False, n_cand: int = 0,
                 device: str = "cuda", stream=None, model: str = "poisson", sigma: float = 1.0,
                 sparse_k: bool = False, wide_counts: bool = False, dense_estep: bool = False):
        import torch
        self.torch = torch
        gauss = MODELS[model] == MODEL_GAUSSIAN
        if precision is None:
            precision = "fp16_split" if gauss else "bf16_split"
        store_scores = store_scores or gauss  # the Gaussian pass 2 reads the stored scores
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        q = np.ascontiguousarray(q, dtype=np.float64)
        quat = np.ascontiguousarray(quat, dtype=np.float64)
        weight = np.ascontiguousarray(weight, dtype=np.float64)
        self.cfg = Config(N=N, precision=precision, n_pix=q.shape[0], n_rot=quat.shape[0],
                          n_data=n_data, w_floor=w_floor, compress_mode=compress_mode,
                          flags=(FLAG_STORE_SCORES if store_scores else 0) |
                          (FLAG_SPARSE_K if sparse_k else 0) |
                          (FLAG_WIDE_COUNTS if wide_counts else 0) |
                          (FLAG_DENSE_ESTEP if dense_estep else 0), rot_chunk=rot_chunk,
                          n_cand=n_cand, model=MODELS[model], sigma=float(sigma))
        L = lib()
        nb = ctypes.c_size_t()
        _check(L.emc_workspace_size(ctypes.byref(self.cfg), ctypes.byref(nb)), "emc_workspace_size")
        self.device = torch.device(device)
        self.workspace = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        h = _vp()
        _check(L.emc_ctx_create(ctypes.byref(self.cfg), q.ctypes.data_as(_dp),
                                quat.ctypes.data_as(_dp), weight.ctypes.data_as(_dp),
                                self.workspace.data_ptr(), nb.value, _stream(stream),
                                ctypes.byref(h)), "emc_ctx_create")
        self.h = h
        self.sizes_all = self.buffer_sizes(self.cfg.n_rot)

    # -- housekeeping -------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            lib().emc_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def N(self) -> int:
        return self.cfg.N

    @property
    def ld_pix(self) -> int:
        return self.sizes_all.ld_pix

    @property
    def ld_data(self) -> int:
        return self.sizes_all.ld_data

    def buffer_sizes(self, nrot: int) -> BufferSizes:
        b = BufferSizes()
        _check(lib().emc_buffer_sizes_for(ctypes.byref(self.cfg), nrot, ctypes.byref(b)),
               "emc_buffer_sizes_for")
        return b

    def status(self) -> int:
        v = _i32()
        _check(lib().emc_ctx_status(self.h, ctypes.byref(v)), "emc_ctx_status")
        return v.value

    def set_wait_limit(self, wait_limit_ns: int = 0, stall: bool = False):
        """Limit of the tensor-core kernels' bounded waits (0: default) and the
        stall test hook of emc_ctx_set_wait_limit."""
        _check(lib().emc_ctx_set_wait_limit(self.h, int(wait_limit_ns), int(bool(stall))),
               "emc_ctx_set_wait_limit")

    def _bytes(self, n: int):
        return self.torch.empty(int(n), dtype=self.torch.uint8, device=self.device)

    # -- the ABI calls --------------------------------------------------------
    def set_frames(self, K, stream=None):
        """K: device int32 [n_data, ld_k] photon counts."""
        assert K.dtype == self.torch.int32 and K.is_cuda and K.is_contiguous()
        _check(lib().emc_set_frames(self.h, K.data_ptr(), K.shape[1], _stream(stream)),
               "emc_set_frames")

    def expand(self, grid, rot0: int, nrot: int, stream=None):
        b = self.buffer_sizes(nrot)
        L = self._bytes(b.logw_bytes)
        bias = self.torch.empty(b.bias_bytes // 8, dtype=self.torch.float64, device=self.device)
        _check(lib().emc_expand(self.h, _ptr(grid), rot0, nrot, _ptr(L), _ptr(bias),
                                _stream(stream)), "emc_expand")
        return L, bias

    def scores_buffer(self, nrot: int):
        """A buffer for the stored scores of emc_loglik / emc_normalize."""
        return self._bytes(self.buffer_sizes(nrot).score_bytes)

    def loglik(self, L, bias, nrot: int, lse_m=None, lse_s=None, accumulate: bool = False,
               scores=None, stream=None):
        if lse_m is None:
            lse_m = self.torch.empty(self.ld_data, dtype=self.torch.float64, device=self.device)
            lse_s = self.torch.empty(self.ld_data, dtype=self.torch.float64, device=self.device)
        _check(lib().emc_loglik(self.h, _ptr(L), _ptr(bias), nrot, _ptr(lse_m), _ptr(lse_s),
                                int(accumulate), _ptr(scores), _stream(stream)), "emc_loglik")
        return lse_m, lse_s

    def loglik_sparse_k(self, L, bias, nrot: int, lse_m=None, lse_s=None,
                        accumulate: bool = False, stream=None):
        if lse_m is None:
            lse_m = self.torch.empty(self.ld_data, dtype=self.torch.float64, device=self.device)
            lse_s = self.torch.empty(self.ld_data, dtype=self.torch.float64, device=self.device)
        _check(lib().emc_loglik_sparse_k(self.h, _ptr(L), _ptr(bias), nrot, _ptr(lse_m),
                                         _ptr(lse_s), int(accumulate), _stream(stream)),
               "emc_loglik_sparse_k")
        return lse_m, lse_s

    def normalize(self, L, bias, nrot: int, lse_m, lse_s, scores=None, stream=None):
        b = self.buffer_sizes(nrot)
        P = self._bytes(b.prob_bytes)
        _check(lib().emc_normalize(self.h, _ptr(L), _ptr(bias), nrot, _ptr(lse_m), _ptr(lse_s),
                                   _ptr(scores), _ptr(P), _stream(stream)), "emc_normalize")
        return P

    def update(self, P, nrot: int, stream=None):
        b = self.buffer_sizes(nrot)
        Num = self.torch.empty((b.rows, b.ld_pix), dtype=self.torch.float32, device=self.device)
        den = self.torch.empty(b.rows, dtype=self.torch.float32, device=self.device)
        _check(lib().emc_update(self.h, _ptr(P), nrot, _ptr(Num), _ptr(den), _stream(stream)),
               "emc_update")
        return Num, den

    def compress(self, rot0: int, nrot: int, Num, den, g_num=None, g_den=None,
                 accumulate: bool = False, stream=None):
        N = self.N
        if g_num is None:
            g_num = self.torch.empty((N, N, N), dtype=self.torch.float64, device=self.device)
            g_den = self.torch.empty((N, N, N), dtype=self.torch.float64, device=self.device)
        _check(lib().emc_compress(self.h, rot0, nrot, _ptr(Num), _ptr(den), _ptr(g_num),
                                  _ptr(g_den), int(accumulate), _stream(stream)), "emc_compress")
        return g_num, g_den

    def finalize(self, g_num, g_den, grid_prev, grid_out=None, stream=None):
        if grid_out is None:
            grid_out = self.torch.empty_like(grid_prev)
        _check(lib().emc_finalize(self.h, _ptr(g_num), _ptr(g_den), _ptr(grid_prev),
                                  _ptr(grid_out), _stream(stream)), "emc_finalize")
        return grid_out

    def iteration(self, grid_in, grid_out=None, stats: bool = True, stream=None):
        if grid_out is None:
            grid_out = self.torch.empty_like(grid_in)
        st = IterStats()
        _check(lib().emc_iteration(self.h, _ptr(grid_in), _ptr(grid_out),
                                   ctypes.byref(st) if stats else None, _stream(stream)),
               "emc_iteration")
        if not stats:
            return grid_out, None
        return grid_out, {f: getattr(st, f) for f, _ in IterStats._fields_}

    def iteration_lse(self, stream=None):
        """lse_k of every frame after the last iteration (device float64 [n_data])."""
        lse = self.torch.empty(self.cfg.n_data, dtype=self.torch.float64, device=self.device)
        _check(lib().emc_iteration_lse(self.h, _ptr(lse), _stream(stream)), "emc_iteration_lse")
        return lse

    def responsibilities(self, frames, stream=None):
        """P_jk of the given frames after the last iteration (device float32
        [len(frames), n_rot]); frames: device int32."""
        assert frames.dtype == self.torch.int32 and frames.is_contiguous()
        n = int(frames.numel())
        P = self.torch.empty((n, self.cfg.n_rot), dtype=self.torch.float32, device=self.device)
        _check(lib().emc_responsibilities(self.h, _ptr(frames), n, _ptr(P), _stream(stream)),
               "emc_responsibilities")
        return P

    # -- learned proposal and sparse Maximize ------------------------------------
    def features(self, stream=None):
        feat = self.torch.empty((self.ld_data, 512), dtype=self.torch.float32, device=self.device)
        _check(lib().emc_features(self.h, _ptr(feat), _stream(stream)), "emc_features")
        return feat

    def targets_from_scores(self, R: int, scores=None, stream=None):
        nd = self.cfg.n_data
        tidx = self.torch.empty((nd, R), dtype=self.torch.int32, device=self.device)
        tprob = self.torch.empty((nd, R), dtype=self.torch.float32, device=self.device)
        _check(lib().emc_targets_from_scores(self.h, _ptr(scores), R, _ptr(tidx), _ptr(tprob),
                                             _stream(stream)), "emc_targets_from_scores")
        return tidx, tprob

    def set_candidates(self, cand, stream=None):
        assert cand.dtype == self.torch.int32 and cand.is_contiguous()
        _check(lib().emc_set_candidates(self.h, _ptr(cand), _stream(stream)),
               "emc_set_candidates")

    def sparse_estep(self, L, bias, stream=None):
        P = self.torch.empty((self.ld_data, self.cfg.n_cand), dtype=self.torch.float32,
                             device=self.device)
        lse = self.torch.empty(self.ld_data, dtype=self.torch.float64, device=self.device)
        _check(lib().emc_sparse_estep(self.h, _ptr(L), _ptr(bias), _ptr(P), _ptr(lse),
                                      _stream(stream)), "emc_sparse_estep")
        return P, lse

    def sparse_update(self, P, stream=None):
        b = self.sizes_all
        Num = self.torch.empty((b.rows, b.ld_pix), dtype=self.torch.float32, device=self.device)
        den = self.torch.empty(b.rows, dtype=self.torch.float32, device=self.device)
        _check(lib().emc_sparse_update(self.h, _ptr(P), _ptr(Num), _ptr(den), _stream(stream)),
               "emc_sparse_update")
        return Num, den

    def sparse_iteration(self, grid_in, grid_out=None, stats: bool = True, stream=None):
        if grid_out is None:
            grid_out = self.torch.empty_like(grid_in)
        st = IterStats()
        _check(lib().emc_sparse_iteration(self.h, _ptr(grid_in), _ptr(grid_out),
                                          ctypes.byref(st) if stats else None, _stream(stream)),
               "emc_sparse_iteration")
        if not stats:
            return grid_out, None
        return grid_out, {f: getattr(st, f) for f, _ in IterStats._fields_}

    def collect(self, per_frame: int = 32):
        """Record the non-zero responsibilities of every later iteration into a
        list of per_frame * n_data entries that this object owns (0 stops)."""
        if per_frame <= 0:
            _check(lib().emc_set_collect(self.h, None, 0), "emc_set_collect")
            self._collect_buf = None
            return
        cap = per_frame * self.cfg.n_data
        nbytes = lib().emc_collect_bytes(self.h, cap)
        buf = self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.device)
        _check(lib().emc_set_collect(self.h, _ptr(buf), cap), "emc_set_collect")
        self._collect_buf = buf

    def collected_targets(self, R: int, missed: bool = False, stream=None):
        """(tidx, tprob[, missed]) from the responsibilities the last iteration
        recorded (see collect)."""
        nd = self.cfg.n_data
        tidx = self.torch.empty((nd, R), dtype=self.torch.int32, device=self.device)
        tprob = self.torch.empty((nd, R), dtype=self.torch.float32, device=self.device)
        mm = (self.torch.empty(nd, dtype=self.torch.float32, device=self.device)
              if missed else None)
        _check(lib().emc_collected_targets(self.h, R, _ptr(tidx), _ptr(tprob), _ptr(mm),
                                           _stream(stream)), "emc_collected_targets")
        return (tidx, tprob, mm) if missed else (tidx, tprob)

    def missed_mass(self, scores=None, lse_m=None, lse_s=None, stream=None):
        out = self.torch.empty(self.cfg.n_data, dtype=self.torch.float32, device=self.device)
        _check(lib().emc_missed_mass(self.h, _ptr(scores), _ptr(lse_m), _ptr(lse_s), _ptr(out),
                                     _stream(stream)), "emc_missed_mass")
        return out
