"""ctypes front end of the oracle's C join (bgp_join.c) -- test infrastructure."""

from __future__ import annotations

import ctypes

import numpy as np

from .build import build

ORACLE_OK = 0
ORACLE_ERR_INVALID = 1
ORACLE_ERR_UNSUPPORTED = 2
ORACLE_ERR_ROW_LIMIT = 3
ORACLE_ERR_OOM = 4


class OracleError(RuntimeError):
    def __init__(self, code: int):
        names = {1: "invalid", 2: "unsupported", 3: "row limit", 4: "out of memory"}
        super().__init__(f"oracle error {code}: {names.get(code, '?')}")
        self.code = code


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        lib.oracle_index_build.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(vp)]
        lib.oracle_index_build.restype = ctypes.c_int
        lib.oracle_index_free.argtypes = [vp]
        lib.oracle_index_size.argtypes = [vp]
        lib.oracle_index_size.restype = ctypes.c_int64
        lib.oracle_bgp.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                   ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64), vp]
        lib.oracle_bgp.restype = ctypes.c_int
        lib.oracle_free.argtypes = [vp]
        _lib = lib
    return _lib


def _pattern_array(patterns) -> np.ndarray:
    """Accept a BGP object, an (n, 6) array (s, p, o, s_var, p_var, o_var) or
    a list of (s, p, o, s_var, o_var) tuples."""
    if hasattr(patterns, "as_array"):
        arr = patterns.as_array()
    else:
        arr = np.asarray(patterns, dtype=np.int64)
        if arr.ndim == 2 and arr.shape[1] == 5:
            arr = np.stack([arr[:, 0], arr[:, 1], arr[:, 2], arr[:, 3],
                            np.zeros(arr.shape[0], np.int64), arr[:, 4]], axis=1)
    return np.ascontiguousarray(arr, dtype=np.int64).reshape(-1, 6)


class OracleIndex:
    """The triple set sorted by (p,s,o) and (p,o,s), duplicates removed."""

    def __init__(self, triples: np.ndarray):
        lib = _load()
        t = np.ascontiguousarray(np.asarray(triples, dtype=np.int32).reshape(-1, 3))
        h = ctypes.c_void_p()
        rc = lib.oracle_index_build(t.ctypes.data, t.shape[0], ctypes.byref(h))
        if rc:
            raise OracleError(rc)
        self._h = h
        self._lib = lib

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.oracle_index_free(h)
            self._h = None

    @property
    def n_unique(self) -> int:
        return int(self._lib.oracle_index_size(self._h))

    def query(self, patterns, n_vars: int | None = None, row_limit: int = 1 << 62,
              return_steps: bool = False):
        """Sorted result rows, an (n_rows, n_vars) int32 array."""
        arr = _pattern_array(patterns)
        if n_vars is None:
            n_vars = patterns.n_vars
        out = ctypes.c_void_p()
        nrows = ctypes.c_int64()
        steps = np.zeros(arr.shape[0], dtype=np.int64)
        rc = self._lib.oracle_bgp(self._h, arr.ctypes.data, arr.shape[0], int(n_vars), int(row_limit),
                                  ctypes.byref(out), ctypes.byref(nrows), steps.ctypes.data)
        if rc:
            raise OracleError(rc)
        n = int(nrows.value)
        if n_vars > 0 and n > 0:
            buf = (ctypes.c_int32 * (n * n_vars)).from_address(out.value)
            rows = np.frombuffer(buf, dtype=np.int32).reshape(n, n_vars).copy()
            self._lib.oracle_free(out)
        else:
            rows = np.zeros((n, n_vars), dtype=np.int32)
        return (rows, steps) if return_steps else rows


def oracle_query(triples, patterns, n_vars=None, row_limit: int = 1 << 62):
    return OracleIndex(triples).query(patterns, n_vars, row_limit)
