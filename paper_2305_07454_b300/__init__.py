"""Python binding of libcvetl.so, the CUDA (sm_103a) connected-vehicle ETL library.

Argument marshalling only: every step of extract / transform / load runs in the library's
own CUDA kernels behind the C ABI declared in ``include/cvetl.h`` (arXiv 2305.07454,
Accelerated ETL section and Algorithm 2). PyTorch supplies device memory and streams.
There is no CPU fallback: importing this package without the built library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcvetl.so")

OK, EINVAL, ENOMEM, EFULL, ESTATE, ECUDA, ETIMEOUT, EPARSE = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "EFULL", "ESTATE", "ECUDA", "ETIMEOUT", "EPARSE"]
FP64, FP32 = 0, 1
IN_COLUMNS, IN_CSV = 0, 1
BATCH, STREAM = 0, 1
KEY_INVALID = 0xFFFFFFFF
F_START, F_DUP, F_OFFGRID, F_STOP = 0x01, 0x02, 0x04, 0x08

_P = ctypes.c_void_p


class Config(ctypes.Structure):
    _fields_ = [
        ("lat_min", ctypes.c_double), ("lon_min", ctypes.c_double), ("cell_deg", ctypes.c_double),
        ("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32), ("n_bins", ctypes.c_int32),
        ("t0_ms", ctypes.c_int64), ("bin_ms", ctypes.c_int64),
        ("v_stop_kmh", ctypes.c_float), ("earth_radius_m", ctypes.c_double),
        ("precision", ctypes.c_int32), ("materialize_points", ctypes.c_int32),
        ("profile", ctypes.c_int32), ("device", ctypes.c_int32),
        ("mem_budget_bytes", ctypes.c_size_t), ("stream", _P),
        ("mode", ctypes.c_int32), ("lateness_ms", ctypes.c_int64), ("graph", ctypes.c_int32),
    ]


class Input(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("on_device", ctypes.c_int32), ("n", ctypes.c_int64),
        ("jid", _P), ("ts", _P), ("lat", _P), ("lon", _P), ("speed", _P), ("heading", _P),
        ("csv", _P), ("csv_len", ctypes.c_size_t), ("window_end_ms", ctypes.c_int64),
    ]


_CELL = [("key", "<u4"), ("row", "<i4"), ("col", "<i4"), ("bin", "<i4"), ("count", "<u4"),
         ("sum", "<f8"), ("mean", "<f8"), ("min", "<f4"), ("max", "<f4"), ("volume", "<u4")]
_JOURNEY = [("id", "<i8"), ("n", "<i8"), ("offset", "<i8"), ("start_ts", "<i8"), ("end_ts", "<i8"),
            ("duration_ms", "<i8"), ("distance_m", "<f8"), ("dwell_ms", "<i8"),
            ("start_lat", "<f8"), ("start_lon", "<f8"), ("end_lat", "<f8"), ("end_lon", "<f8")]
_POINT = [("perm", "<u4"), ("d", "<f8"), ("vhat", "<f4"), ("accel", "<f4"), ("dwell", "<i8"),
          ("key", "<u4"), ("flags", "|u1"), ("stop_ms", "<i8"), ("accel_v", "<f4")]
_EXTRACTED = [("jid", "<i8"), ("ts", "<i8"), ("lat", "<f8"), ("lon", "<f8"), ("speed", "<f4"),
              ("heading", "<f4")]
_COUNTERS = ["n_in", "n_malformed", "n_valid", "n_out_of_grid", "n_dup", "n_too_late", "n_runs"]


class Tables(ctypes.Structure):
    _fields_ = (
        [("n_cells", ctypes.c_int64)] + [("cell_" + k, _P) for k, _ in _CELL]
        + [("n_journeys", ctypes.c_int64)] + [("j_" + k, _P) for k, _ in _JOURNEY]
        + [("n_points", ctypes.c_int64)] + [("p_" + k, _P) for k, _ in _POINT]
        + [("n_extracted", ctypes.c_int64)] + [("x_" + k, _P) for k, _ in _EXTRACTED]
        + [(k, ctypes.c_int64) for k in _COUNTERS]
    )


MAX_STAGES = 32


class Stats(ctypes.Structure):
    _fields_ = [("n_stages", ctypes.c_int32), ("name", ctypes.c_char_p * MAX_STAGES),
                ("ms", ctypes.c_double * MAX_STAGES), ("launches", ctypes.c_int64 * MAX_STAGES),
                ("total_launches", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("graph_replays", ctypes.c_int64)]


class Instance(ctypes.Structure):
    _fields_ = [("lat_min", ctypes.c_double), ("lon_min", ctypes.c_double),
                ("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32), ("t0_ms", ctypes.c_int64),
                ("n", ctypes.c_int64), ("jid", _P), ("ts", _P), ("lat", _P), ("lon", _P), ("speed", _P)]


MAX_INSTANCES = 32
GRID_KEYS = ("lat_min", "lon_min", "n_rows", "n_cols", "t0_ms")


class Tuning(ctypes.Structure):
    _fields_ = [("journey_ctas", ctypes.c_int32), ("row_unroll", ctypes.c_int32),
                ("small_sort_max", ctypes.c_int32), ("row_block", ctypes.c_int32),
                ("small_journey_max", ctypes.c_int32), ("scatter_block", ctypes.c_int32)]


DXN_CARDINAL, DXN_QUADRANT = 0, 1


class LatticeConfig(ctypes.Structure):
    _fields_ = [("bin_ms", ctypes.c_int64), ("n_bins", ctypes.c_int32), ("direction", ctypes.c_int32),
                ("dense", ctypes.c_int32), ("normalize", ctypes.c_int32)]


_LATTICE = [("key", "<u4"), ("bin", "<i4"), ("dxn", "<i4"), ("row", "<i4"), ("col", "<i4"), ("count", "<u4"),
            ("sum", "<f8"), ("mean", "<f4"), ("volume", "<u4"), ("mean_norm", "<f4"), ("volume_norm", "<f4")]


class Lattice(ctypes.Structure):
    _fields_ = ([("n_cells", ctypes.c_int64)] + [(k, _P) for k, _ in _LATTICE]
                + [("n_dropped", ctypes.c_int64), ("dense", _P), ("n_bins", ctypes.c_int32),
                   ("ch_min", ctypes.c_float * 8), ("ch_max", ctypes.c_float * 8)])


class ServerConfig(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int32), ("device", ctypes.c_int32),
                ("mem_budget_bytes", ctypes.c_size_t)]


class TicketInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("feed", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("slot", ctypes.c_int32), ("n", ctypes.c_int64), ("submit_ns", ctypes.c_int64),
                ("start_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
                ("peak_in_flight", ctypes.c_int32), ("message", ctypes.c_char * 164)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libcvetl.so is not built ({LIB_PATH}); run "
                          "`python paper_2305_07454_b300/build.py` (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    lib.cvetl_config_default.argtypes = [ctypes.POINTER(Config)]
    lib.cvetl_config_default.restype = None
    lib.cvetl_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(_P)]
    lib.cvetl_extract.argtypes = [_P, ctypes.POINTER(Input)]
    lib.cvetl_transform.argtypes = [_P]
    lib.cvetl_load.argtypes = [_P]
    lib.cvetl_results.argtypes = [_P, ctypes.POINTER(Tables)]
    lib.cvetl_flush.argtypes = [_P]
    lib.cvetl_stats_get.argtypes = [_P, ctypes.POINTER(Stats)]
    lib.cvetl_stats_reset.argtypes = [_P]
    lib.cvetl_destroy.argtypes = [_P]
    lib.cvetl_last_error.argtypes = [_P]
    lib.cvetl_last_error.restype = ctypes.c_char_p
    lib.cvetl_version.restype = ctypes.c_int32
    lib.cvetl_sort_u64_noalloc.argtypes = [_P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P]
    lib.cvetl_sort_u64_noalloc.restype = ctypes.c_int
    lib.cvetl_probe_fp64.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P,
                                     ctypes.POINTER(ctypes.c_int64), _P]
    lib.cvetl_probe_fp64.restype = ctypes.c_int
    lib.cvetl_extract_batch.argtypes = [_P, ctypes.POINTER(Instance), ctypes.c_int32, ctypes.c_int32]
    _I64P = ctypes.POINTER(ctypes.c_int64)
    lib.cvetl_batch_ranges.argtypes = [_P, _I64P, _I64P, _I64P, _I64P, ctypes.c_int32]
    lib.cvetl_lattice_config_default.argtypes = [ctypes.POINTER(LatticeConfig)]
    lib.cvetl_lattice_config_default.restype = None
    lib.cvetl_lattice_build.argtypes = [_P, ctypes.POINTER(LatticeConfig), ctypes.POINTER(Lattice)]
    lib.cvetl_tuning_get.argtypes = [_P, ctypes.POINTER(Tuning)]
    lib.cvetl_tuning_set.argtypes = [_P, ctypes.POINTER(Tuning)]
    lib.cvetl_autotune.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(Tuning), ctypes.POINTER(ctypes.c_double)]
    lib.cvetl_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)]
    lib.cvetl_server_add_feed.argtypes = [_P, ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_int32)]
    lib.cvetl_server_submit.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(Input), ctypes.POINTER(ctypes.c_uint64)]
    lib.cvetl_server_submit_flush.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]
    lib.cvetl_server_wait.argtypes = [_P, ctypes.c_uint64, ctypes.POINTER(TicketInfo)]
    lib.cvetl_server_drain.argtypes = [_P]
    lib.cvetl_server_feed.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(_P)]
    lib.cvetl_server_destroy.argtypes = [_P]
    lib.cvetl_server_last_error.argtypes = [_P]
    lib.cvetl_server_last_error.restype = ctypes.c_char_p
    for f in ("cvetl_create", "cvetl_extract", "cvetl_transform", "cvetl_load", "cvetl_results",
              "cvetl_flush", "cvetl_stats_get", "cvetl_stats_reset", "cvetl_destroy",
              "cvetl_extract_batch", "cvetl_batch_ranges", "cvetl_tuning_get", "cvetl_tuning_set",
              "cvetl_autotune", "cvetl_lattice_build", "cvetl_server_create", "cvetl_server_add_feed", "cvetl_server_submit",
              "cvetl_server_submit_flush", "cvetl_server_wait", "cvetl_server_drain",
              "cvetl_server_feed", "cvetl_server_destroy"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


lib = _load()

# The C-ABI entry points declared in include/cvetl.h (checked by the tests).
EXPORTS = ("cvetl_config_default", "cvetl_create", "cvetl_extract", "cvetl_transform", "cvetl_load",
           "cvetl_results", "cvetl_flush", "cvetl_stats_get", "cvetl_stats_reset", "cvetl_destroy",
           "cvetl_last_error", "cvetl_version", "cvetl_sort_u64_noalloc", "cvetl_extract_batch",
           "cvetl_batch_ranges", "cvetl_tuning_get", "cvetl_tuning_set", "cvetl_autotune",
           "cvetl_lattice_config_default", "cvetl_lattice_build", "cvetl_server_create",
           "cvetl_server_add_feed", "cvetl_server_submit", "cvetl_server_submit_flush",
           "cvetl_server_wait", "cvetl_server_drain", "cvetl_server_feed", "cvetl_server_destroy",
           "cvetl_server_last_error", "cvetl_probe_fp64")
NOALLOC_MAX_PAIRS = 262144
SERVE_BYTES_PER_ROW = 320
SERVE_MAX_SLOTS = 64


PROBE_FMA, PROBE_ADD, PROBE_MUL, PROBE_MIX = range(4)


def probe_fp64(kind: int, blocks: int, threads: int, iters: int, sink, stream=None) -> int:
    """Enqueues the binary64 issue-rate probe (cvetl_probe_fp64) on `stream` (default: the
    current torch stream); sink: a float64 device tensor of blocks * threads elements. Returns
    the binary64 operations the launch performs; the caller times it with CUDA events."""
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    assert sink.dtype == torch.float64 and sink.is_cuda and sink.numel() >= blocks * threads
    ops = ctypes.c_int64(0)
    st = lib.cvetl_probe_fp64(kind, blocks, threads, iters, sink.data_ptr(), ctypes.byref(ops),
                              ctypes.c_void_p(stream.cuda_stream))
    if st != OK:
        raise CvetlError(st, lib.cvetl_last_error(None).decode())
    return int(ops.value)


class CvetlError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class _DeviceArray:
    """A device pointer exposed through the CUDA array interface (zero-copy for torch)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None, "stream": None}


def default_config(**kw) -> Config:
    cfg = Config()
    lib.cvetl_config_default(ctypes.byref(cfg))
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def _columns_input(cols: dict, window_end_ms: int = 0):
    """An Input over the five columns (torch tensors or numpy arrays) and the tensors to keep
    alive while the library may read them."""
    import torch

    names = ("jid", "ts", "lat", "lon", "speed")
    dtypes = (torch.int64, torch.int64, torch.float64, torch.float64, torch.float32)
    ts = []
    for k, dt in zip(names, dtypes):
        v = cols[k]
        if isinstance(v, np.ndarray):
            v = torch.from_numpy(np.ascontiguousarray(v))
        if v.dtype != dt or not v.is_contiguous() or v.dim() != 1:
            raise ValueError(f"column {k} must be a contiguous 1-D {dt} tensor")
        ts.append(v)
    hd = cols.get("heading")
    if hd is not None:
        if isinstance(hd, np.ndarray):
            hd = torch.from_numpy(np.ascontiguousarray(hd))
        if hd.dtype != torch.float32 or not hd.is_contiguous() or hd.dim() != 1:
            raise ValueError("column heading must be a contiguous 1-D torch.float32 tensor")
        ts.append(hd)
    n = ts[0].shape[0]
    if any(t.shape[0] != n for t in ts):
        raise ValueError("columns differ in length")
    dev = {t.is_cuda for t in ts}
    if len(dev) != 1:
        raise ValueError("columns must be all on the device or all on the host")
    on_device = dev.pop()
    inp = Input(kind=IN_COLUMNS, on_device=int(on_device), n=n,
                jid=ts[0].data_ptr(), ts=ts[1].data_ptr(), lat=ts[2].data_ptr(),
                lon=ts[3].data_ptr(), speed=ts[4].data_ptr(),
                heading=ts[5].data_ptr() if hd is not None else None,
                window_end_ms=int(window_end_ms))
    return inp, ts


class Pipeline:
    """One cvetl context: extract -> transform -> load -> results on one CUDA stream."""

    def __init__(self, stream=None, **cfg):
        import torch

        self._torch = torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.config = default_config(**cfg)
        self.config.stream = stream.cuda_stream
        self.config.device = stream.device.index if stream.device.index is not None else 0
        h = _P()
        st = lib.cvetl_create(ctypes.byref(self.config), ctypes.byref(h))
        if st != OK:
            raise CvetlError(st, lib.cvetl_last_error(None).decode())
        self._h = h
        self._keep = None
        self._owned = True

    @classmethod
    def _view(cls, handle):
        """A Pipeline over a context the library owns (a server feed): results and stats only."""
        import torch

        p = cls.__new__(cls)
        p._torch = torch
        p._h = handle
        p._keep = None
        p._owned = False
        return p

    def _check(self, st: int):
        if st != OK:
            raise CvetlError(st, lib.cvetl_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            if self._owned:
                lib.cvetl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def extract(self, cols: dict, window_end_ms: int = 0):
        """cols: jid, ts, lat, lon, speed (+ heading) as torch tensors, all on the device or
        all on the host, or numpy arrays (host). window_end_ms: stream mode only."""
        inp, self._keep = _columns_input(cols, window_end_ms)
        self._check(lib.cvetl_extract(self._h, ctypes.byref(inp)))

    def extract_batch(self, instances: list):
        """A batch of instances: each a dict with its grid (lat_min, lon_min, n_rows, n_cols,
        t0_ms) and its columns jid, ts, lat, lon, speed (all instances' columns on the device,
        or all on the host)."""
        arr = (Instance * len(instances))()
        keep, dev = [], set()
        for q, inst in zip(arr, instances):
            inp, ts = _columns_input(inst)
            keep.append(ts)
            dev.add(bool(inp.on_device))
            for k in GRID_KEYS:
                setattr(q, k, inst[k])
            q.n = inp.n
            q.jid, q.ts, q.lat, q.lon, q.speed = inp.jid, inp.ts, inp.lat, inp.lon, inp.speed
        if len(dev) > 1:
            raise ValueError("instances must be all on the device or all on the host")
        self._keep = keep
        self._check(lib.cvetl_extract_batch(self._h, arr, len(instances), int(dev.pop()) if dev else 0))

    def batch_ranges(self) -> dict:
        """First row, key, cell row and journey row of each instance (+ the totals)."""
        m = len(self._keep) + 1
        out = {k: (ctypes.c_int64 * m)() for k in ("row_begin", "key_begin", "cell_begin", "journey_begin")}
        self._check(lib.cvetl_batch_ranges(self._h, out["row_begin"], out["key_begin"], out["cell_begin"],
                                           out["journey_begin"], m))
        return {k: np.array(v[:], dtype=np.int64) for k, v in out.items()}

    def run_batch(self, instances: list, to_host: bool = True) -> list:
        """extract_batch -> transform -> load; each instance's cells and journeys (and points,
        when materialised) as its own result dict, plus the batch's total counters."""
        self.extract_batch(instances)
        self.transform()
        self.load()
        r = self.results(to_host=to_host)
        rg = self.batch_ranges()
        out = []
        for i in range(len(instances)):
            c0, c1 = rg["cell_begin"][i], rg["cell_begin"][i + 1]
            j0, j1 = rg["journey_begin"][i], rg["journey_begin"][i + 1]
            one = {"cells": {k: v[c0:c1] for k, v in r["cells"].items()},
                   "journeys": {k: v[j0:j1] for k, v in r["journeys"].items()},
                   "batch_counters": r["counters"], "ranges": {k: v[i] for k, v in rg.items()}}
            if "points" in r:
                p0 = int(r["journeys"]["offset"][j0]) if j1 > j0 else 0
                p1 = int(r["journeys"]["offset"][j1 - 1] + r["journeys"]["n"][j1 - 1]) if j1 > j0 else 0
                one["points"] = {k: v[p0:p1] for k, v in r["points"].items()}
            out.append(one)
        return out

    @property
    def tuning(self) -> dict:
        t = Tuning()
        self._check(lib.cvetl_tuning_get(self._h, ctypes.byref(t)))
        return {k: int(getattr(t, k)) for k, _ in Tuning._fields_}

    @tuning.setter
    def tuning(self, value: dict):
        t = Tuning(**{**self.tuning, **value})
        self._check(lib.cvetl_tuning_set(self._h, ctypes.byref(t)))

    def autotune(self, reps: int = 2) -> dict:
        """Tunes the launch shapes on the extracted rows (leaves the context extracted)."""
        t, ms = Tuning(), ctypes.c_double()
        self._check(lib.cvetl_autotune(self._h, int(reps), ctypes.byref(t), ctypes.byref(ms)))
        return {**{k: int(getattr(t, k)) for k, _ in Tuning._fields_}, "ms": float(ms.value)}

    def lattice(self, to_host: bool = True, **cfg) -> dict:
        """The 8-channel lattice of the last batch (after load): the occupied cells, the dense
        [n_bins, 8, n_rows, n_cols] tensor (a zero-copy device tensor, or None), the channel
        extremes and the count of dropped rows. cfg: bin_ms, n_bins, direction, dense, normalize."""
        torch = self._torch
        lc = LatticeConfig()
        lib.cvetl_lattice_config_default(ctypes.byref(lc))
        for k, v in cfg.items():
            setattr(lc, k, v)
        L = Lattice()
        self._check(lib.cvetl_lattice_build(self._h, ctypes.byref(lc), ctypes.byref(L)))

        def view(ptr, n, ty):
            if n == 0 or not ptr:
                return np.empty(0, np.dtype(ty)) if to_host else None
            a = torch.as_tensor(_DeviceArray(ptr, n, ty), device="cuda")
            return a.cpu().numpy() if to_host else a

        out = {"cells": {k: view(getattr(L, k), L.n_cells, ty) for k, ty in _LATTICE},
               "n_dropped": int(L.n_dropped), "ch_min": np.array(L.ch_min[:], np.float32),
               "ch_max": np.array(L.ch_max[:], np.float32), "dense": None}
        if L.dense:
            shape = (int(L.n_bins), 8, int(self.config.n_rows), int(self.config.n_cols))
            n = int(np.prod(shape))
            out["dense"] = torch.as_tensor(_DeviceArray(L.dense, n, "<f4"), device="cuda").view(shape)
        return out

    def extract_csv(self, text):
        """CSV text as bytes / numpy uint8 (host) or a uint8 torch tensor (host or device)."""
        torch = self._torch
        if isinstance(text, (bytes, bytearray)):
            text = np.frombuffer(bytes(text), dtype=np.uint8).copy()
        if isinstance(text, np.ndarray):
            text = torch.from_numpy(np.ascontiguousarray(text, dtype=np.uint8))
        if text.dtype != torch.uint8 or not text.is_contiguous() or text.dim() != 1:
            raise ValueError("CSV text must be a contiguous 1-D uint8 tensor")
        n = int(text.shape[0])
        inp = Input(kind=IN_CSV, on_device=int(text.is_cuda), n=0,
                    csv=text.data_ptr() if n else None, csv_len=n)
        self._keep = [text]
        self._check(lib.cvetl_extract(self._h, ctypes.byref(inp)))

    def extracted(self, to_host: bool = True) -> dict:
        """The extracted columns (the parsed rows of CSV input), valid until the next extract."""
        torch = self._torch
        t = self.tables()
        out = {}
        for k, ty in _EXTRACTED:
            ptr = getattr(t, "x_" + k)
            if not ptr or t.n_extracted == 0:
                out[k] = np.empty(0, np.dtype(ty)) if to_host else None
                continue
            a = torch.as_tensor(_DeviceArray(ptr, t.n_extracted, ty), device="cuda")
            out[k] = a.cpu().numpy() if to_host else a
        return out

    def flush(self):
        """Stream mode: finalise every pending point and close every open run."""
        self._check(lib.cvetl_flush(self._h))

    def push_window(self, cols: dict, window_end_ms: int):
        """Stream mode: one window (extract + transform + load)."""
        self.extract(cols, window_end_ms)
        self.transform()
        self.load()

    def transform(self):
        self._check(lib.cvetl_transform(self._h))

    def load(self):
        self._check(lib.cvetl_load(self._h))

    def tables(self) -> Tables:
        t = Tables()
        self._check(lib.cvetl_results(self._h, ctypes.byref(t)))
        return t

    def results(self, to_host: bool = True, out: "HostTables | None" = None) -> dict:
        """Cells, journeys, per-point columns (if materialised) and counters. to_host=False
        returns zero-copy device tensors valid until the next extract. With out (pinned host
        buffers from host_tables()), the columns are copied into them on the pipeline's stream
        with one synchronisation, and the returned arrays are views of out, valid until out is
        reused."""
        torch = self._torch
        t = self.tables()

        def dev(ptr, n, typestr):
            if n == 0 or not ptr:
                np_dt = np.dtype(typestr)
                return torch.empty(0, dtype=torch.from_numpy(np.empty(0, np_dt)).dtype, device="cuda")
            return torch.as_tensor(_DeviceArray(ptr, n, typestr), device="cuda")

        parts = {"cells": ("cell_", _CELL, t.n_cells), "journeys": ("j_", _JOURNEY, t.n_journeys)}
        if t.n_points and t.p_perm:
            parts["points"] = ("p_", _POINT, t.n_points)
        res = {}
        if to_host and out is not None:
            with torch.cuda.stream(self.stream):
                for part, (pre, cols, n) in parts.items():
                    res[part] = {}
                    for k, ty in cols:
                        buf = out.get(part, k, n)
                        if n:
                            buf.copy_(dev(getattr(t, pre + k), n, ty), non_blocking=True)
                        res[part][k] = buf.numpy()
            self.stream.synchronize()
        else:
            for part, (pre, cols, n) in parts.items():
                res[part] = {}
                for k, ty in cols:
                    arr = dev(getattr(t, pre + k), n, ty)
                    res[part][k] = arr.cpu().numpy() if to_host else arr
        res["counters"] = {k: int(getattr(t, k)) for k in _COUNTERS}
        res["counters"]["n_journeys"] = int(t.n_journeys)
        res["counters"]["n_cells"] = int(t.n_cells)
        return res

    def host_tables(self, cells: int, journeys: int, points: int = 0) -> "HostTables":
        """Pinned host buffers for results(out=...) with room for the given table sizes."""
        return HostTables(cells, journeys, points)

    def stats(self) -> dict:
        s = Stats()
        self._check(lib.cvetl_stats_get(self._h, ctypes.byref(s)))
        return {"stages": {s.name[i].decode(): {"ms": s.ms[i], "launches": int(s.launches[i])}
                           for i in range(s.n_stages)},
                "total_launches": int(s.total_launches), "device_bytes": int(s.device_bytes),
                "graph_replays": int(s.graph_replays)}

    def stats_reset(self):
        self._check(lib.cvetl_stats_reset(self._h))

    def run(self, cols: dict, to_host: bool = True) -> dict:
        self.extract(cols)
        self.transform()
        self.load()
        return self.results(to_host=to_host)


class HostTables:
    """Pinned host buffers for Pipeline.results(out=...): one per result column, grown on
    demand (a larger table reallocates that column)."""

    def __init__(self, cells: int, journeys: int, points: int = 0):
        import torch

        self._torch = torch
        self._cap = {"cells": cells, "journeys": journeys, "points": points}
        self._bufs = {}

    def get(self, part: str, name: str, n: int):
        torch = self._torch
        cols = {"cells": _CELL, "journeys": _JOURNEY, "points": _POINT}[part]
        ty = dict(cols)[name]
        b = self._bufs.get((part, name))
        if b is None or b.shape[0] < n:
            cap = max(n, self._cap[part])
            dt = torch.from_numpy(np.empty(0, np.dtype(ty))).dtype
            b = torch.empty(cap, dtype=dt, pin_memory=True)
            self._bufs[(part, name)] = b
        return b[:n]


class Server:
    """The serving runtime (cvetl_server_*): stream-mode feeds, one FIFO request queue,
    n_slots windows on the GPU at once (different feeds on their own CUDA streams), admission
    by a device-memory budget. submit() returns a ticket at once; wait() returns its record
    as a dict (status, feed, kind, slot, n, submit_ns, start_ns, done_ns, peak_in_flight,
    message) and raises CvetlError when the request failed and check is true."""

    def __init__(self, n_slots: int = 4, mem_budget_bytes: int = 0, device: int = 0):
        cfg = ServerConfig(n_slots=n_slots, device=device, mem_budget_bytes=mem_budget_bytes)
        h = _P()
        st = lib.cvetl_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise CvetlError(st, lib.cvetl_server_last_error(None).decode())
        self._h = h
        self._keep = {}

    def _check(self, st: int):
        if st != OK:
            raise CvetlError(st, lib.cvetl_server_last_error(self._h).decode())

    def add_feed(self, **cfg) -> int:
        c = default_config(**cfg)
        f = ctypes.c_int32()
        self._check(lib.cvetl_server_add_feed(self._h, ctypes.byref(c), ctypes.byref(f)))
        return int(f.value)

    def submit(self, feed: int, cols: dict, window_end_ms: int) -> int:
        """Queues a window (host columns should be in pinned memory); the columns are kept
        alive until wait() on the ticket."""
        inp, keep = _columns_input(cols, window_end_ms)
        t = ctypes.c_uint64()
        self._check(lib.cvetl_server_submit(self._h, int(feed), ctypes.byref(inp), ctypes.byref(t)))
        self._keep[int(t.value)] = keep
        return int(t.value)

    def submit_flush(self, feed: int) -> int:
        t = ctypes.c_uint64()
        self._check(lib.cvetl_server_submit_flush(self._h, int(feed), ctypes.byref(t)))
        return int(t.value)

    def wait(self, ticket: int, check: bool = True) -> dict:
        info = TicketInfo()
        st = lib.cvetl_server_wait(self._h, ctypes.c_uint64(ticket), ctypes.byref(info))
        if st == EINVAL and info.submit_ns == 0:
            self._check(st)
        self._keep.pop(int(ticket), None)
        out = {k: getattr(info, k) for k, _ in TicketInfo._fields_ if k != "message"}
        out["message"] = info.message.decode(errors="replace")
        if check and st != OK:
            raise CvetlError(st, out["message"])
        return out

    def drain(self):
        self._check(lib.cvetl_server_drain(self._h))

    def feed(self, feed: int) -> Pipeline:
        """A view of the feed's context (results, stats) while it has no request queued."""
        h = _P()
        self._check(lib.cvetl_server_feed(self._h, int(feed), ctypes.byref(h)))
        return Pipeline._view(h)

    def close(self):
        if getattr(self, "_h", None):
            lib.cvetl_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
