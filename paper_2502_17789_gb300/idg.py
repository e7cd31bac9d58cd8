"""ctypes binding of libidg (the C ABI declared in include/idg.h).

Argument marshalling only: every step of gridding and degridding runs in the
CUDA library.  The functions carry the C names; `Plan` wraps a plan handle
for torch tensors (device memory and the current CUDA stream come from
torch).  There is no CPU fallback: if libidg.so is missing or fails to load,
`load()` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libidg.so")

IDG_OK = 0
STATUS_NAMES = {0: "IDG_OK", 1: "IDG_ERR_INVALID_ARG", 2: "IDG_ERR_UNSORTED_FREQ", 3: "IDG_ERR_UV_OUT_OF_GRID",
                4: "IDG_ERR_W_TOO_LARGE", 5: "IDG_ERR_OOM", 6: "IDG_ERR_CUDA", 7: "IDG_ERR_TIMEOUT",
                8: "IDG_ERR_UNSUPPORTED"}
IDG_TAPER_KB, IDG_TAPER_USER = 0, 1
IDG_DROP_OUT_OF_GRID, IDG_SPLIT_AT_ATERM_INTERVALS, IDG_HOST_ONLY, IDG_PERSISTENT, IDG_W_LAYERS = 1, 2, 4, 8, 16
IDG_NORMALIZE_ATERM, IDG_STOKES_I = 32, 64
IDG_MAC_DEFAULT, IDG_MAC_FP32, IDG_MAC_TENSOR, IDG_MAC_TENSOR_DEGRID = 0, 1, 2, 3

# every function declared in include/idg.h
EXPORTS = ["idg_plan_create", "idg_grid", "idg_degrid", "idg_grid_graph", "idg_degrid_graph", "idg_set_stream", "idg_plan_stats", "idg_plan_subgrids",
           "idg_plan_segments", "idg_plan_layers", "idg_subgrid_images", "idg_synchronize", "idg_profile_enable", "idg_profile_read",
           "idg_grid_noalloc", "idg_invert", "idg_predict", "idg_wait_selftest", "idg_aterm_weights", "idg_last_error",
           "idg_plan_destroy", "idg_abi_version", "idg_peak_rates", "idg_grid_many", "idg_degrid_many"]
KERNEL_CLASSES = ["gridder", "fft_adder", "splitter_ifft", "degridder", "stage", "aterm_flags"]


class IdgError(RuntimeError):
    def __init__(self, status: int, where: str, message: str = ""):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Geometry(ctypes.Structure):
    _fields_ = [("grid_size", ctypes.c_int32), ("subgrid_size", ctypes.c_int32), ("kernel_padding", ctypes.c_int32),
                ("image_size", ctypes.c_double), ("taper_kind", ctypes.c_int32), ("taper_beta", ctypes.c_double),
                ("taper_user", ctypes.POINTER(ctypes.c_double)), ("aterm_nodes", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("degrid_channels", ctypes.c_int32), ("grid_chunk", ctypes.c_int32),
                ("mac_unit", ctypes.c_int32)]


class PlanStats(ctypes.Structure):
    _fields_ = [("n_subgrids", ctypes.c_int64), ("n_segments", ctypes.c_int64), ("n_vis", ctypes.c_int64),
                ("n_vis_dropped", ctypes.c_int64), ("n_subgrids_dropped", ctypes.c_int64),
                ("n_grid_items", ctypes.c_int64), ("n_degrid_items", ctypes.c_int64), ("n_batches", ctypes.c_int64),
                ("occupancy_hist", ctypes.c_int64 * 16), ("device_bytes", ctypes.c_int64),
                ("vis_pixels", ctypes.c_int64), ("subgrid_size", ctypes.c_int32), ("batch_capacity", ctypes.c_int32),
                ("n_w_layers", ctypes.c_int32), ("w_layer_min", ctypes.c_int32), ("w_layer_step", ctypes.c_double),
                ("n_pol", ctypes.c_int32), ("degrid_channels", ctypes.c_int32), ("grid_chunk", ctypes.c_int32),
                ("mac_unit", ctypes.c_int32)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["occupancy_hist"] = list(self.occupancy_hist)
        return d


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libidg.so (build it with paper_2502_17789_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libidg.so not found at {path}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.idg_plan_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Geometry), i32, i32, i32, i32, P, P, P, P, i32, P]
    lib.idg_grid.argtypes = [P, P, P, P]
    lib.idg_degrid.argtypes = [P, P, P, P]
    lib.idg_grid_graph.argtypes = [P, P, P, P]
    lib.idg_degrid_graph.argtypes = [P, P, P, P]
    lib.idg_set_stream.argtypes = [P, P]
    lib.idg_plan_stats.argtypes = [P, ctypes.POINTER(PlanStats)]
    lib.idg_plan_subgrids.argtypes = [P, P, i64, ctypes.POINTER(i64)]
    lib.idg_plan_segments.argtypes = [P, P, i64, ctypes.POINTER(i64)]
    lib.idg_plan_layers.argtypes = [P, P, i64, ctypes.POINTER(i64)]
    lib.idg_subgrid_images.argtypes = [P, P, P, i32, P]
    lib.idg_synchronize.argtypes = [P]
    lib.idg_grid_noalloc.argtypes = [P, P, P, P]
    lib.idg_wait_selftest.argtypes = [P, ctypes.c_int32]
    lib.idg_aterm_weights.argtypes = [P, P, i32]
    lib.idg_invert.argtypes = [P, P, P, P, P]
    lib.idg_predict.argtypes = [P, P, P, P, P]
    lib.idg_profile_enable.argtypes = [P, i32]
    lib.idg_peak_rates.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.idg_grid_many.argtypes = [i32, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), P]
    lib.idg_degrid_many.argtypes = [i32, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), P]
    lib.idg_profile_read.argtypes = [P, P, P]
    lib.idg_last_error.argtypes = [P]
    lib.idg_last_error.restype = ctypes.c_char_p
    lib.idg_plan_destroy.argtypes = [P]
    lib.idg_abi_version.argtypes = []
    for name in EXPORTS:
        if name not in ("idg_last_error",):
            getattr(lib, name).restype = i32
    _lib = lib
    return lib


def _check(status: int, where: str, plan=None):
    if status != IDG_OK:
        msg = load().idg_last_error(plan).decode(errors="replace")
        raise IdgError(status, where, msg)


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


# ----------------------------------------------------------------- C names

def idg_plan_create(geom: Geometry, n_stations: int, baselines, uvw_m, freqs_hz, aterm_offsets, stream=None):
    lib = load()
    bl = np.ascontiguousarray(baselines, dtype=np.int32)
    uvw = np.ascontiguousarray(uvw_m, dtype=np.float64)
    fr = np.ascontiguousarray(freqs_hz, dtype=np.float64)
    off = np.ascontiguousarray(aterm_offsets, dtype=np.int32)
    handle = ctypes.c_void_p()
    n_bl = int(bl.shape[0])
    n_t = int(uvw.shape[1]) if uvw.ndim == 3 else 0
    st = lib.idg_plan_create(ctypes.byref(handle), ctypes.byref(geom), int(n_stations), n_bl, n_t, int(fr.shape[0]),
                             _np_ptr(bl), _np_ptr(uvw), _np_ptr(fr), _np_ptr(off), int(off.shape[0] - 1),
                             ctypes.c_void_p(stream or 0))
    _check(st, "idg_plan_create")
    return handle


def idg_grid(plan, vis_ptr, aterms_ptr, grid_ptr):
    _check(load().idg_grid(plan, vis_ptr, aterms_ptr, grid_ptr), "idg_grid", plan)


def idg_grid_noalloc(plan, vis_ptr, aterms_ptr, grid_ptr):
    _check(load().idg_grid_noalloc(plan, vis_ptr, aterms_ptr, grid_ptr), "idg_grid_noalloc", plan)


def idg_invert(plan, vis_ptr, aterms_ptr, grid_ptr, image_ptr):
    _check(load().idg_invert(plan, vis_ptr, aterms_ptr, grid_ptr, image_ptr), "idg_invert", plan)


def idg_predict(plan, image_ptr, aterms_ptr, grid_ptr, vis_ptr):
    _check(load().idg_predict(plan, image_ptr, aterms_ptr, grid_ptr, vis_ptr), "idg_predict", plan)


def idg_wait_selftest(plan, limit_us: int):
    _check(load().idg_wait_selftest(plan, int(limit_us)), "idg_wait_selftest", plan)


def idg_degrid(plan, grid_ptr, aterms_ptr, vis_ptr):
    _check(load().idg_degrid(plan, grid_ptr, aterms_ptr, vis_ptr), "idg_degrid", plan)


def idg_grid_graph(plan, vis_ptr, aterms_ptr, grid_ptr):
    _check(load().idg_grid_graph(plan, vis_ptr, aterms_ptr, grid_ptr), "idg_grid_graph", plan)


def idg_degrid_graph(plan, grid_ptr, aterms_ptr, vis_ptr):
    _check(load().idg_degrid_graph(plan, grid_ptr, aterms_ptr, vis_ptr), "idg_degrid_graph", plan)


def idg_set_stream(plan, stream):
    _check(load().idg_set_stream(plan, ctypes.c_void_p(stream or 0)), "idg_set_stream", plan)


def idg_plan_stats(plan) -> PlanStats:
    s = PlanStats()
    _check(load().idg_plan_stats(plan, ctypes.byref(s)), "idg_plan_stats", plan)
    return s


def idg_plan_subgrids(plan) -> np.ndarray:
    lib = load()
    n = ctypes.c_int64(0)
    _check(lib.idg_plan_subgrids(plan, None, 0, ctypes.byref(n)), "idg_plan_subgrids", plan)
    out = np.zeros((max(n.value, 1), 8), np.int32)
    _check(lib.idg_plan_subgrids(plan, _np_ptr(out), n.value, ctypes.byref(n)), "idg_plan_subgrids", plan)
    return out[: n.value]


def idg_plan_layers(plan) -> np.ndarray:
    """int32 [n_subgrids, 2]: per subgrid its w layer k (w0 = (k + 1/2) *
    w_layer_step) and 1 if it holds mirrored rows (w < 0, gridded as V^H at -uvw)."""
    lib = load()
    n = ctypes.c_int64(0)
    _check(lib.idg_plan_layers(plan, None, 0, ctypes.byref(n)), "idg_plan_layers", plan)
    out = np.zeros((max(n.value, 1), 2), np.int32)
    _check(lib.idg_plan_layers(plan, _np_ptr(out), n.value, ctypes.byref(n)), "idg_plan_layers", plan)
    return out[: n.value]


def idg_plan_segments(plan) -> np.ndarray:
    lib = load()
    n = ctypes.c_int64(0)
    _check(lib.idg_plan_segments(plan, None, 0, ctypes.byref(n)), "idg_plan_segments", plan)
    out = np.zeros((max(n.value, 1), 4), np.int32)
    _check(lib.idg_plan_segments(plan, _np_ptr(out), n.value, ctypes.byref(n)), "idg_plan_segments", plan)
    return out[: n.value]


def idg_subgrid_images(plan, vis_ptr, aterms_ptr, stage, out_ptr):
    _check(load().idg_subgrid_images(plan, vis_ptr, aterms_ptr, int(stage), out_ptr), "idg_subgrid_images", plan)


def idg_synchronize(plan):
    _check(load().idg_synchronize(plan), "idg_synchronize", plan)


def idg_profile_enable(plan, on: bool):
    _check(load().idg_profile_enable(plan, 1 if on else 0), "idg_profile_enable", plan)


def idg_profile_read(plan) -> dict:
    ms = np.zeros(len(KERNEL_CLASSES), np.float64)
    n = np.zeros(len(KERNEL_CLASSES), np.int64)
    _check(load().idg_profile_read(plan, _np_ptr(ms), _np_ptr(n)), "idg_profile_read", plan)
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}


def idg_last_error(plan=None) -> str:
    return load().idg_last_error(plan).decode(errors="replace")


def idg_plan_destroy(plan):
    _check(load().idg_plan_destroy(plan), "idg_plan_destroy")


def idg_peak_rates(stream=None) -> tuple[float, float]:
    """(FP32 FMA per second, __sincosf evaluations per second) measured on the
    current device by the library's probe kernels (see idg_peak_rates in idg.h)."""
    f, s = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().idg_peak_rates(stream, ctypes.byref(f), ctypes.byref(s)), "idg_peak_rates")
    return float(f.value), float(s.value)


def _ptr_array(values):
    arr = (ctypes.c_void_p * len(values))()
    for k, v in enumerate(values):
        arr[k] = v
    return arr


def grid_many(plans, vis, aterms, grids, stream=None):
    """idg_grid_many: grid several plans' visibilities (CUDA torch tensors,
    one per plan) with their work items sharing one launch per wave on
    `stream` (default: torch's current stream)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    n = len(plans)
    _check(load().idg_grid_many(n, _ptr_array([p.handle for p in plans]), _ptr_array([_dev_ptr(v) for v in vis]),
                                _ptr_array([_dev_ptr(a) for a in aterms]), _ptr_array([_dev_ptr(g) for g in grids]),
                                stream), "idg_grid_many", plans[0].handle)
    return grids


def degrid_many(plans, grids, aterms, vis, stream=None):
    """idg_degrid_many: the degridding counterpart of grid_many."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    n = len(plans)
    _check(load().idg_degrid_many(n, _ptr_array([p.handle for p in plans]), _ptr_array([_dev_ptr(g) for g in grids]),
                                  _ptr_array([_dev_ptr(a) for a in aterms]), _ptr_array([_dev_ptr(v) for v in vis]),
                                  stream), "idg_degrid_many", plans[0].handle)
    return vis


def idg_abi_version() -> int:
    return int(load().idg_abi_version())


# ----------------------------------------------------------------- torch-facing wrapper

def make_geometry(grid_size, subgrid_size, kernel_padding, image_size, taper_beta=0.0, aterm_nodes=9, flags=0,
                  taper_user=None, degrid_channels=0, grid_chunk=0, mac_unit=0) -> tuple[Geometry, object]:
    g = Geometry()
    g.grid_size, g.subgrid_size, g.kernel_padding = int(grid_size), int(subgrid_size), int(kernel_padding)
    g.image_size = float(image_size)
    keep = None
    if taper_user is not None:
        keep = np.ascontiguousarray(taper_user, dtype=np.float64)
        g.taper_kind = IDG_TAPER_USER
        g.taper_user = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    else:
        g.taper_kind = IDG_TAPER_KB
    g.taper_beta = float(taper_beta)
    g.aterm_nodes = int(aterm_nodes)
    g.flags = int(flags)
    g.degrid_channels = int(degrid_channels)
    g.grid_chunk = int(grid_chunk)
    g.mac_unit = int(mac_unit)
    return g, keep


class Plan:
    """One observation's partition and device tables.

    grid()/degrid() take CUDA torch tensors: vis complex64 [bl, t, ch, 4],
    aterms complex64 [n_int, n_st, nodes, nodes, 4], grid complex128 [4, N, N].
    They run on the plan's stream (by default torch's current stream at
    construction)."""

    def __init__(self, obs=None, *, grid_size=None, subgrid_size=None, kernel_padding=None, image_size=None,
                 n_stations=None, baselines=None, uvw=None, freqs=None, aterm_offsets=None, aterm_nodes=9,
                 flags=0, taper_beta=0.0, taper_user=None, stream=None, degrid_channels=0, grid_chunk=0,
                 mac_unit=0):
        if obs is not None:
            grid_size = obs.grid_size if grid_size is None else grid_size
            subgrid_size = obs.subgrid_size if subgrid_size is None else subgrid_size
            kernel_padding = obs.kernel_padding if kernel_padding is None else kernel_padding
            image_size = obs.image_size if image_size is None else image_size
            n_stations, baselines, uvw = obs.n_stations, obs.baselines, obs.uvw
            freqs, aterm_offsets, aterm_nodes = obs.freqs, obs.aterm_offsets, obs.aterm_nodes
        self.geometry, self._keep = make_geometry(grid_size, subgrid_size, kernel_padding, image_size, taper_beta,
                                                  aterm_nodes, flags, taper_user, degrid_channels, grid_chunk,
                                                  mac_unit)
        if stream is None and not (flags & IDG_HOST_ONLY):
            import torch
            stream = torch.cuda.current_stream().cuda_stream  # 0 when that is the legacy default stream
        self.stream = stream
        self.handle = idg_plan_create(self.geometry, n_stations, baselines, uvw, freqs, aterm_offsets, stream)
        self.shape = (int(np.shape(uvw)[0]), int(np.shape(uvw)[1]), int(len(freqs)))

    def grid(self, vis, aterms, grid):
        idg_grid(self.handle, _dev_ptr(vis), _dev_ptr(aterms), _dev_ptr(grid))
        return grid

    def degrid(self, grid, aterms, vis):
        idg_degrid(self.handle, _dev_ptr(grid), _dev_ptr(aterms), _dev_ptr(vis))
        return vis

    def grid_graph(self, vis, aterms, grid):
        idg_grid_graph(self.handle, _dev_ptr(vis), _dev_ptr(aterms), _dev_ptr(grid))
        return grid

    def degrid_graph(self, grid, aterms, vis):
        idg_degrid_graph(self.handle, _dev_ptr(grid), _dev_ptr(aterms), _dev_ptr(vis))
        return vis

    def subgrid_images(self, vis, aterms, stage: int):
        import torch
        L = self.geometry.subgrid_size
        st = self.stats()
        out = torch.empty((st.n_subgrids, st.n_pol, L, L), dtype=torch.complex64, device=vis.device)
        idg_subgrid_images(self.handle, _dev_ptr(vis), _dev_ptr(aterms), stage, _dev_ptr(out))
        return out

    def set_stream(self, stream):
        self.stream = stream
        idg_set_stream(self.handle, stream)

    def synchronize(self):
        idg_synchronize(self.handle)

    def invert(self, vis, aterms, grid, image):
        """Dirty image [4, N, N] (pol, m, l) of `vis`; `grid` receives the uv plane."""
        idg_invert(self.handle, _dev_ptr(vis), _dev_ptr(aterms), _dev_ptr(grid), _dev_ptr(image))
        return image

    def predict(self, image, aterms, grid, vis):
        """Visibilities of `image` [4, N, N]; `grid` receives the model uv plane."""
        idg_predict(self.handle, _dev_ptr(image), _dev_ptr(aterms), _dev_ptr(grid), _dev_ptr(vis))
        return vis

    def aterm_weights(self, reset: bool = False) -> np.ndarray:
        """A-term power weights of a plan made with IDG_NORMALIZE_ATERM:
        float64 [L*L + 1], sum n_seg / ||A_p^H A_q||_F per subgrid pixel
        ([j][i] flattened) and sum n_seg last (see idg_aterm_weights)."""
        L = self.geometry.subgrid_size
        out = np.zeros(L * L + 1, np.float64)
        _check(load().idg_aterm_weights(self.handle, _np_ptr(out), int(bool(reset))), "idg_aterm_weights", self.handle)
        return out

    def wait_selftest(self, limit_us: int = 20000):
        idg_wait_selftest(self.handle, limit_us)

    def profile(self, on: bool = True):
        idg_profile_enable(self.handle, on)

    def profile_read(self) -> dict:
        return idg_profile_read(self.handle)

    def stats(self) -> PlanStats:
        return idg_plan_stats(self.handle)

    def subgrids(self) -> np.ndarray:
        return idg_plan_subgrids(self.handle)

    def segments(self) -> np.ndarray:
        return idg_plan_segments(self.handle)

    def layers(self) -> np.ndarray:
        return idg_plan_layers(self.handle)

    def grid_shape(self) -> tuple:
        """Shape of the master grid this plan grids into: [n_w_layers, n_pol, N, N],
        or [n_pol, N, N] for a plan without IDG_W_LAYERS (n_pol = 4, or 1 with
        IDG_STOKES_I)."""
        st = self.stats()
        N, npol = self.geometry.grid_size, int(st.n_pol)
        return (int(st.n_w_layers), npol, N, N) if self.geometry.flags & IDG_W_LAYERS else (npol, N, N)

    def image_shape(self) -> tuple:
        """Shape of the images of invert / predict: [n_pol, N, N]."""
        return (int(self.stats().n_pol), self.geometry.grid_size, self.geometry.grid_size)

    def close(self):
        if getattr(self, "handle", None) is not None:
            idg_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
