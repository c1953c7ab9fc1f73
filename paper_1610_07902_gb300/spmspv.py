"""Thin ctypes binding of the C ABI in include/spmspv.h.

Every function here has the name of the C entry point it calls and only
marshals arguments: torch tensors are passed as raw device pointers, the
torch stream as a cudaStream_t.  All computation happens in the CUDA
kernels of libspmspv.so.  If the library cannot be loaded the import fails
loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import builder as _build

# ---- constants mirrored from include/spmspv.h ----
SPMSPV_OK = 0
SPMSPV_ERR_ARG = 1
SPMSPV_ERR_STATE = 2
SPMSPV_ERR_OOM = 3
SPMSPV_ERR_CUDA = 4
SPMSPV_ERR_CAPACITY = 5
SPMSPV_ERR_TIMEOUT = 6
SPMSPV_ERR_INDEX = 7
SPMSPV_ERR_UNSUPPORTED = 8

SPMSPV_VAL_NONE = 0
SPMSPV_VAL_F32 = 1

SPMSPV_CSC_PATTERN_SYMMETRIC = 1
SPMSPV_CSC_SYMMETRIC = 3

SPMSPV_PLUS_TIMES_F32 = 0
SPMSPV_MIN_SELECT2ND_I32 = 1
SPMSPV_OR_AND_BOOL = 2

SPMSPV_MASK_COMPLEMENT = 1
SPMSPV_SORTED_OUT = 2
SPMSPV_SCHED_AUTO = 4
SPMSPV_SCHED_FORCE = 8
SPMSPV_SCHED_SHIFT = 8
SPMSPV_NUM_SCHEDULES = 12

SPMSPV_STAGE_SCAN = 0
SPMSPV_STAGE_SELECT = 1
SPMSPV_STAGE_SCATTER = 2
SPMSPV_STAGE_MERGE = 3
SPMSPV_STAGE_PULL = 4
SPMSPV_NUM_STAGES = 5

SPMSPV_WITH_FEATURES = 16
SPMSPV_SELECTOR_NPARAM = 1688

SPMSPV_DEV_CAPACITY = 1
SPMSPV_DEV_TIMEOUT = 2
SPMSPV_DEV_INDEX = 4
SPMSPV_DEV_BOUND = 8
SPMSPV_SORT_X = 32
SPMSPV_SCHED_RULE = 64
SPMSPV_BUCKETS_ONLY = 128  # spmspv_run, (+,*): never the direct form
SPMSPV_X_IDS = 65536  # (min, select2nd): x values equal their indices (the pull may stop early)
SPMSPV_LANES_PERSISTENT = -1  # spmspv_run_batched: the persistent one-launch form


def SPMSPV_SCHED_OPT(s: int) -> int:
    return SPMSPV_SCHED_FORCE | (int(s) << SPMSPV_SCHED_SHIFT)


class SpmspvError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed with status %d: %s" % (where, code, spmspv_last_error()))


_lib = None
_P = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libspmspv.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError("libspmspv.so not found at %s; run build()" % _build.LIB)
        lib = ctypes.CDLL(_build.LIB)
        lib.spmspv_last_error.restype = ctypes.c_char_p
        lib.spmspv_last_error.argtypes = []
        lib.spmspv_create_csc.argtypes = [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int64, _P, _P, _P, ctypes.c_int, ctypes.c_uint32]
        lib.spmspv_destroy.argtypes = [_P]
        lib.spmspv_run.argtypes = [_P, ctypes.c_int, _P, _P, ctypes.c_int32, _P, ctypes.c_uint32,
                                   _P, _P, ctypes.c_int32, _P, _P]
        lib.spmspv_run_host.argtypes = [_P, ctypes.c_int, _P, _P, ctypes.c_int32, _P, ctypes.c_uint32,
                                        _P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _P]
        lib.spmspv_device_status.argtypes = [_P, ctypes.POINTER(ctypes.c_uint32)]
        lib.spmspv_last_work.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
        lib.spmspv_run_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P, _P,
                                           _P, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int32,
                                           _P, ctypes.c_uint32, _P, _P, ctypes.c_int32, _P, _P]
        lib.spmspv_bfs.argtypes = [_P, ctypes.c_int32, _P, _P, _P, ctypes.c_uint32, _P]
        lib.spmspv_selector_set.argtypes = [_P, _P, ctypes.c_int32]
        lib.spmspv_selector_get.argtypes = [_P, _P, ctypes.c_int32]
        lib.spmspv_selector_load.argtypes = [_P, ctypes.c_char_p]
        lib.spmspv_last_features.argtypes = [_P, _P]
        lib.spmspv_last_schedule.argtypes = [_P, ctypes.POINTER(ctypes.c_int32)]
        lib.spmspv_default_schedule.argtypes = [_P, ctypes.POINTER(ctypes.c_int32)]
        lib.spmspv_selector_train.argtypes = [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, _P]
        lib.spmspv_selector_grad.argtypes = [_P, _P, _P, _P, ctypes.c_int32, _P, _P]
        lib.spmspv_run_batched.argtypes = [_P, ctypes.c_int, ctypes.c_int32, _P, _P, _P, _P, _P,
                                           ctypes.c_int64, ctypes.c_uint32, _P, _P, _P, _P, _P,
                                           ctypes.c_int32, _P]
        lib.spmspv_batched_phase_times.argtypes = [_P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        lib.spmspv_msbfs.argtypes = [_P, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_uint32,
                                     ctypes.c_int32, _P]
        lib.spmspv_acl.argtypes = [_P, ctypes.c_int32, _P, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_int32, _P, _P, _P, ctypes.c_int32, _P]
        lib.spmspv_tune_key.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int32,
                                        ctypes.c_int64]
        lib.spmspv_tune_key.restype = ctypes.c_uint64
        lib.spmspv_last_tuned.argtypes = [_P, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        lib.spmspv_tune_entries.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_int32)]
        lib.spmspv_tune_set.argtypes = [_P, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32]
        lib.spmspv_tune_clear.argtypes = [_P]
        lib.spmspv_selftest_wait_timeout.argtypes = [_P, ctypes.c_uint32, _P]
        lib.spmspv_cc.argtypes = [_P, _P, _P, ctypes.c_uint32, _P]
        lib.spmspv_mis.argtypes = [_P, _P, _P, _P, ctypes.c_uint32, _P]
        lib.spmspv_create_dcsc.argtypes = [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                           ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int, ctypes.c_uint32]
        lib.spmspv_dcsc_index.argtypes = [ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]
        lib.spmspv_mcm.argtypes = [_P, _P, _P, _P, _P, ctypes.c_uint32, _P]
        lib.spmspv_profile_begin.argtypes = [_P]
        lib.spmspv_profile_end.argtypes = [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_int32)]
        _lib = lib
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc, where):
    if rc != SPMSPV_OK:
        raise SpmspvError(rc, where)


def spmspv_last_error() -> str:
    return load().spmspv_last_error().decode(errors="replace")


def spmspv_create_csc(m, n, nnz, colptr, rowidx, val, val_type, flags=0):
    """Returns an opaque handle (int).  colptr/rowidx/val are CUDA tensors."""
    h = _P()
    rc = load().spmspv_create_csc(ctypes.byref(h), int(m), int(n), int(nnz), _ptr(colptr),
                                  _ptr(rowidx), _ptr(val), int(val_type), int(flags))
    _check(rc, "spmspv_create_csc")
    return h.value


def spmspv_destroy(h):
    _check(load().spmspv_destroy(h), "spmspv_destroy")


def spmspv_run(h, semiring, x_idx, x_val, nnz_x, mask, opts, y_idx, y_val, y_capacity, d_nnz_y,
               stream=None):
    rc = load().spmspv_run(h, int(semiring), _ptr(x_idx), _ptr(x_val), int(nnz_x), _ptr(mask),
                           int(opts), _ptr(y_idx), _ptr(y_val), int(y_capacity), _ptr(d_nnz_y),
                           _stream(stream))
    _check(rc, "spmspv_run")


def spmspv_run_noalloc(m, n, nnz, colptr, rowidx, val, val_type, semiring, x_idx, x_val, nnz_x,
                       mask, opts, y_idx, y_val, y_capacity, d_nnz_y, stream=None):
    """The handle-free entry point that allocates no device memory."""
    rc = load().spmspv_run_noalloc(int(m), int(n), int(nnz), _ptr(colptr), _ptr(rowidx), _ptr(val),
                                   int(val_type), int(semiring), _ptr(x_idx), _ptr(x_val),
                                   int(nnz_x), _ptr(mask), int(opts), _ptr(y_idx), _ptr(y_val),
                                   int(y_capacity), _ptr(d_nnz_y), _stream(stream))
    _check(rc, "spmspv_run_noalloc")


def spmspv_bfs(h, src, level, parent, d_nlevels, opts=0, stream=None):
    _check(load().spmspv_bfs(h, int(src), _ptr(level), _ptr(parent), _ptr(d_nlevels), int(opts),
                             _stream(stream)), "spmspv_bfs")


def spmspv_selector_set(h, params):
    import numpy as np
    arr = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().spmspv_selector_set(h, arr.ctypes.data, int(arr.size)), "spmspv_selector_set")


def spmspv_selector_load(h, path):
    _check(load().spmspv_selector_load(h, os.fsencode(str(path))), "spmspv_selector_load")


def spmspv_selector_get(h):
    import numpy as np
    arr = np.empty(SPMSPV_SELECTOR_NPARAM, dtype=np.float32)
    _check(load().spmspv_selector_get(h, arr.ctypes.data, int(arr.size)), "spmspv_selector_get")
    return arr


def spmspv_last_features(h):
    import numpy as np
    arr = np.empty(6, dtype=np.float32)
    _check(load().spmspv_last_features(h, arr.ctypes.data), "spmspv_last_features")
    return arr


def spmspv_last_schedule(h) -> int:
    v = ctypes.c_int32(0)
    _check(load().spmspv_last_schedule(h, ctypes.byref(v)), "spmspv_last_schedule")
    return int(v.value)


TUNE_BATCHED, TUNE_MSBFS, TUNE_ACL = 0, 1, 2


def spmspv_tune_key(kind, semiring, masked, B, total_nnz_x) -> int:
    return int(load().spmspv_tune_key(int(kind), int(semiring), 1 if masked else 0, int(B),
                                      int(total_nnz_x)))


def spmspv_last_tuned(h):
    """(lanes, schedule, from_cache) of the handle's last autotuned call."""
    a, b, c = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load().spmspv_last_tuned(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "spmspv_last_tuned")
    return int(a.value), int(b.value), bool(c.value)


def spmspv_tune_entries(h):
    """List of (key, lanes, schedule, ms) in the handle's tuning cache."""
    import numpy as np
    cnt = ctypes.c_int32(0)
    _check(load().spmspv_tune_entries(h, None, None, None, None, 0, ctypes.byref(cnt)),
           "spmspv_tune_entries")
    n = int(cnt.value)
    keys = np.zeros(n, np.uint64)
    lanes = np.zeros(n, np.int32)
    sched = np.zeros(n, np.int32)
    ms = np.zeros(n, np.float32)
    _check(load().spmspv_tune_entries(h, keys.ctypes.data, lanes.ctypes.data, sched.ctypes.data,
                                      ms.ctypes.data, n, ctypes.byref(cnt)), "spmspv_tune_entries")
    return [(int(keys[i]), int(lanes[i]), int(sched[i]), float(ms[i])) for i in range(n)]


def spmspv_tune_set(h, key, lanes, sched):
    _check(load().spmspv_tune_set(h, int(key), int(lanes), int(sched)), "spmspv_tune_set")


def spmspv_tune_clear(h):
    _check(load().spmspv_tune_clear(h), "spmspv_tune_clear")


def spmspv_default_schedule(h) -> int:
    v = ctypes.c_int32(0)
    _check(load().spmspv_default_schedule(h, ctypes.byref(v)), "spmspv_default_schedule")
    return int(v.value)


def spmspv_selector_train(h, feats, target, valid, n, epochs, batch, lr, seed):
    """feats/target/valid: CUDA tensors.  Returns the per-epoch mean loss."""
    import numpy as np
    loss = np.zeros(max(int(epochs), 1), dtype=np.float32)
    _check(load().spmspv_selector_train(h, _ptr(feats), _ptr(target), _ptr(valid), int(n),
                                        int(epochs), int(batch), float(lr), int(seed),
                                        loss.ctypes.data), "spmspv_selector_train")
    return loss[:int(epochs)]


def spmspv_selector_grad(h, feats, target, valid, n):
    import numpy as np
    g = np.zeros(1676, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _check(load().spmspv_selector_grad(h, _ptr(feats), _ptr(target), _ptr(valid), int(n),
                                       g.ctypes.data, loss.ctypes.data), "spmspv_selector_grad")
    return g, float(loss[0])


def spmspv_run_host(h, semiring, x_idx, x_val, nnz_x, mask, opts, y_idx, y_val, y_capacity, stream=None):
    """spmspv_run with x and y in host memory (CPU tensors, ideally pinned);
    returns nnz(y).  mask stays a device bitmap."""
    n = ctypes.c_int32(0)
    _check(load().spmspv_run_host(h, int(semiring), _ptr(x_idx), _ptr(x_val), int(nnz_x), _ptr(mask), int(opts),
                                  _ptr(y_idx), _ptr(y_val), int(y_capacity), ctypes.byref(n), _stream(stream)),
           "spmspv_run_host")
    return int(n.value)


def spmspv_run_batched(h, semiring, B, x_off, x_cnt, x_idx, x_val, masks, mask_stride, opts,
                       y_off, y_cap, y_idx, y_val, d_nnz_y, lanes=4, stream=None):
    _check(load().spmspv_run_batched(h, int(semiring), int(B), _ptr(x_off), _ptr(x_cnt), _ptr(x_idx),
                                     _ptr(x_val), _ptr(masks), int(mask_stride), int(opts),
                                     _ptr(y_off), _ptr(y_cap), _ptr(y_idx), _ptr(y_val),
                                     _ptr(d_nnz_y), int(lanes), _stream(stream)),
           "spmspv_run_batched")


def spmspv_batched_phase_times(h):
    """(ms[8], waves) of the last persistent batched launch: scan, plan, tile
    starts, expand, merge, whole launch, direct expand, direct compaction
    (device clock)."""
    import numpy as np
    ms = np.zeros(8, dtype=np.float64)
    w = ctypes.c_int32(0)
    _check(load().spmspv_batched_phase_times(h, ms.ctypes.data, 8, ctypes.byref(w)),
           "spmspv_batched_phase_times")
    return ms, int(w.value)


def spmspv_msbfs(h, B, sources, level, parent, nlevels, opts=0, lanes=8, stream=None):
    _check(load().spmspv_msbfs(h, int(B), _ptr(sources), _ptr(level), _ptr(parent), _ptr(nlevels),
                               int(opts), int(lanes), _stream(stream)), "spmspv_msbfs")


def spmspv_acl(h, B, seeds, alpha, eps, max_steps, p_out, r_out, steps_out, lanes=8, stream=None):
    _check(load().spmspv_acl(h, int(B), _ptr(seeds), float(alpha), float(eps), int(max_steps),
                             _ptr(p_out), _ptr(r_out), _ptr(steps_out), int(lanes), _stream(stream)),
           "spmspv_acl")


def spmspv_cc(h, labels, d_nrounds=None, opts=0, stream=None):
    _check(load().spmspv_cc(h, _ptr(labels), _ptr(d_nrounds), int(opts), _stream(stream)), "spmspv_cc")


def spmspv_mis(h, prio, in_set, d_nrounds=None, opts=0, stream=None):
    _check(load().spmspv_mis(h, _ptr(prio), _ptr(in_set), _ptr(d_nrounds), int(opts), _stream(stream)),
           "spmspv_mis")


def spmspv_create_dcsc(m, n, nnz, nzc, jc, cp, rowidx, val=None, val_type=SPMSPV_VAL_F32, flags=0):
    """Returns an opaque handle (int) of a DCSC matrix.  jc/cp/rowidx/val are CUDA tensors."""
    h = _P()
    _check(load().spmspv_create_dcsc(ctypes.byref(h), int(m), int(n), int(nnz), int(nzc), _ptr(jc), _ptr(cp),
                                     _ptr(rowidx), _ptr(val), int(val_type), int(flags)),
           "spmspv_create_dcsc")
    return h.value


def spmspv_dcsc_index(n, jc):
    """Host computation of a DCSC matrix's auxiliary column index: (aux
    int32 numpy array, shift).  jc: host numpy int32 array of stored column ids."""
    import numpy as np
    jc = np.ascontiguousarray(jc, dtype=np.int32)
    length = ctypes.c_int64(0)
    shift = ctypes.c_int32(0)
    _check(load().spmspv_dcsc_index(int(n), int(jc.size), jc.ctypes.data if jc.size else None, None, 0,
                                    ctypes.byref(length), ctypes.byref(shift)), "spmspv_dcsc_index")
    aux = np.zeros(length.value, dtype=np.int32)
    _check(load().spmspv_dcsc_index(int(n), int(jc.size), jc.ctypes.data if jc.size else None,
                                    aux.ctypes.data, int(aux.size), ctypes.byref(length), ctypes.byref(shift)),
           "spmspv_dcsc_index")
    return aux, int(shift.value)


def spmspv_mcm(h, mate_r, mate_c, d_card=None, d_nphases=None, opts=0, stream=None):
    _check(load().spmspv_mcm(h, _ptr(mate_r), _ptr(mate_c), _ptr(d_card), _ptr(d_nphases), int(opts),
                             _stream(stream)), "spmspv_mcm")


def spmspv_selftest_wait_timeout(h, spins=1000, stream=None):
    _check(load().spmspv_selftest_wait_timeout(h, int(spins), _stream(stream)),
           "spmspv_selftest_wait_timeout")


def spmspv_device_status(h) -> int:
    v = ctypes.c_uint32(0)
    _check(load().spmspv_device_status(h, ctypes.byref(v)), "spmspv_device_status")
    return int(v.value)


def spmspv_last_work(h) -> int:
    v = ctypes.c_int64(0)
    _check(load().spmspv_last_work(h, ctypes.byref(v)), "spmspv_last_work")
    return int(v.value)


def spmspv_profile_begin(h):
    _check(load().spmspv_profile_begin(h), "spmspv_profile_begin")


def spmspv_profile_end(h):
    """Returns (per-stage summed milliseconds list, number of calls)."""
    arr = (ctypes.c_double * SPMSPV_NUM_STAGES)()
    n = ctypes.c_int32(0)
    _check(load().spmspv_profile_end(h, arr, SPMSPV_NUM_STAGES, ctypes.byref(n)),
           "spmspv_profile_end")
    return [float(v) for v in arr], int(n.value)


class CscMatrix:
    """A CSC matrix resident on the GPU plus its library handle.

    Keeps references to the device tensors the handle borrows, so they
    outlive the handle.
    """

    def __init__(self, m, n, colptr, rowidx, val=None, flags=0, device="cuda"):
        dev = torch.device(device)
        self.m, self.n = int(m), int(n)
        self.flags = int(flags)
        self.colptr = torch.as_tensor(colptr, dtype=torch.int32).to(dev).contiguous()
        self.rowidx = torch.as_tensor(rowidx, dtype=torch.int32).to(dev).contiguous()
        self.val = None if val is None else torch.as_tensor(val, dtype=torch.float32).to(dev).contiguous()
        self.nnz = int(self.rowidx.numel())
        self.handle = spmspv_create_csc(self.m, self.n, self.nnz, self.colptr, self.rowidx, self.val,
                                        SPMSPV_VAL_NONE if self.val is None else SPMSPV_VAL_F32, flags)

    def close(self):
        if self.handle:
            spmspv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bfs(self, src, opts=0, stream=None):
        """(level, parent, nlevels) of a BFS from src; level/parent are CUDA tensors."""
        dev = self.colptr.device
        level = torch.empty(self.n, dtype=torch.int32, device=dev)
        parent = torch.empty(self.n, dtype=torch.int32, device=dev)
        nl = torch.zeros(1, dtype=torch.int32, device=dev)
        spmspv_bfs(self.handle, src, level, parent, nl, opts, stream)
        return level, parent, int(nl.item())

    def multiply(self, semiring, x_idx, x_val=None, mask=None, opts=0, y_capacity=None,
                 stream=None, out=None):
        """y = A (+).(x) x; returns (y_idx, y_val or None) as CUDA tensors (synchronises)."""
        dev = self.colptr.device
        cap = min(self.m, self.nnz) if y_capacity is None else int(y_capacity)
        if out is None:
            y_idx = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
            if semiring == SPMSPV_PLUS_TIMES_F32:
                y_val = torch.empty(max(cap, 1), dtype=torch.float32, device=dev)
            elif semiring == SPMSPV_MIN_SELECT2ND_I32:
                y_val = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
            else:
                y_val = None
            nnz_y = torch.zeros(1, dtype=torch.int32, device=dev)
        else:
            y_idx, y_val, nnz_y = out
        spmspv_run(self.handle, semiring, x_idx, x_val, int(x_idx.numel()), mask, opts, y_idx,
                   y_val, cap, nnz_y, stream)
        k = int(nnz_y.item())
        kk = min(k, cap)
        return y_idx[:kk], (None if y_val is None else y_val[:kk]), k


class DcscMatrix(CscMatrix):
    """A DCSC matrix (only the columns holding entries are stored, with their
    ids in jc) resident on the GPU plus its library handle."""

    def __init__(self, m, n, jc, cp, rowidx, val=None, flags=0, device="cuda"):
        dev = torch.device(device)
        self.m, self.n = int(m), int(n)
        self.flags = int(flags)
        self.jc = torch.as_tensor(jc, dtype=torch.int32).to(dev).contiguous()
        self.cp = torch.as_tensor(cp, dtype=torch.int32).to(dev).contiguous()
        self.colptr = self.cp  # the device the arrays live on, for the shared helpers
        self.rowidx = torch.as_tensor(rowidx, dtype=torch.int32).to(dev).contiguous()
        self.val = None if val is None else torch.as_tensor(val, dtype=torch.float32).to(dev).contiguous()
        self.nnz = int(self.rowidx.numel())
        self.nzc = int(self.jc.numel())
        self.handle = spmspv_create_dcsc(self.m, self.n, self.nnz, self.nzc, self.jc, self.cp, self.rowidx,
                                         self.val, SPMSPV_VAL_NONE if self.val is None else SPMSPV_VAL_F32,
                                         flags)
