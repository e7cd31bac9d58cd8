"""FP64 CPU oracle for image-domain gridding -- TEST INFRASTRUCTURE ONLY.

This package wraps ``idg_oracle.c`` (plain double-precision C, OpenMP over
subgrids) with ctypes.  It is the independent reference that the GPU library
is checked against.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg and reference arm of ``bench.py`` may import it; the library never does, and it
imports nothing from the library.

Every function follows a passage of the paper (arXiv 2502.17789):
  plan()    Section 3.1 partitioning + Section 3.3 A-term constraint
  grid()    Section 2.5 imaging steps 2a-2c, Eq. 10 and Eq. 6
  degrid()  Section 2.5 prediction steps 3a-3c, Eq. 13 (adjoint reading)
  taper()   Section 4.2 Kaiser-Bessel taper
  dft2()    the subgrid Fourier transform of Eq. 8 (centred, unnormalised)
  invert()  Section 2.5 imaging step 3, Eq. 11 (w-stacked over the w layers),
            optionally with the A-term power normalisation of Section 3.3
  predict() Section 2.5 prediction step 2, Eq. 12 with w = 0 (adjoint reading)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "idg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FLAG_DROP = 1
FLAG_SPLIT_INTERVALS = 2
FLAG_W_LAYERS = 4
FLAG_STOKES_I = 8   # one Stokes-I plane instead of the 4 correlation planes (oracle-side flag; the planner ignores it)

STATUS = {0: "ok", 1: "invalid argument", 2: "unsorted frequencies", 3: "uv out of grid",
          4: "w too large", 9: "capacity"}


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: status {code} ({STATUS.get(code, '?')})")
        self.code = code


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no FMA contraction: the planner must
    round exactly like the library's planner)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, f64 = ctypes.c_int, ctypes.c_double
        lib.oracle_plan.argtypes = [i32, i32, i32, f64, i32, i32, i32, i32, P, P, P, i32,
                                    P, i32, P, P, i32, P, P, P, P]
        lib.oracle_plan.restype = i32
        common = [i32, i32, i32, f64, i32, f64, P, i32, i32, i32, i32, i32, P, P, P, i32, P, i32, P, i32,
                  P, P, f64, i32, i32]
        lib.oracle_grid.argtypes = common + [P, P, P, P, P, i32, P]
        lib.oracle_grid.restype = i32
        lib.oracle_degrid.argtypes = common + [P, P, P]
        lib.oracle_degrid.restype = i32
        lib.oracle_taper.argtypes = [i32, i32, f64, P, P]
        lib.oracle_taper.restype = i32
        lib.oracle_bessel_i0.argtypes = [f64]
        lib.oracle_bessel_i0.restype = f64
        lib.oracle_dft2.argtypes = [i32, i32, i32, P, P]
        lib.oracle_dft2.restype = i32
        lib.oracle_aterm_interp.argtypes = [i32, i32, P, P]
        lib.oracle_aterm_interp.restype = i32
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Geometry:
    """Imaging geometry: N (grid), L (subgrid), P (kernel padding), FOV."""
    grid_size: int
    subgrid_size: int
    kernel_padding: int
    image_size: float
    taper_kind: int = 0          # 0 Kaiser-Bessel, 1 user table
    taper_beta: float | None = None   # default 0.35 pi P
    taper_user: np.ndarray | None = None
    aterm_nodes: int = 9
    flags: int = 0

    @property
    def beta(self) -> float:
        # Section 4.2 fixes no beta; 0.35 pi P balances the taper kernel's aliasing
        # against the dynamic range 1/T^2 of taper-corrected models
        return float(0.35 * np.pi * self.kernel_padding) if self.taper_beta is None else float(self.taper_beta)


@dataclass
class Plan:
    subgrids: np.ndarray   # int32 [n_sg, 8]: b, t0, t1, c0, c1, x0, y0, dropped
    segments: np.ndarray   # int32 [n_seg, 4]: subgrid, interval, t_begin, t_end
    layers: np.ndarray | None = None   # int32 [n_sg]: w layer k (w0 = (k + 1/2) w_step); None: no layers, w0 = 0
    w_step: float = 0.0                # layer width 2 w_max, wavelengths
    conj: np.ndarray | None = None     # int32 [n_sg]: 1 = the subgrid holds mirrored rows (w < 0; V^H at -uvw)

    def w0(self, k: int) -> float:
        """w0 of layer k: (2k + 1) w_max = (k + 1/2) w_step (Section 2.4); 0 without layers."""
        return (k + 0.5) * self.w_step if self.layers is not None else 0.0

    @property
    def k_range(self) -> tuple[int, int]:
        """(k_min, n_layers) of the non-dropped subgrids; (0, 1) without layers."""
        if self.layers is None:
            return 0, 1
        keep = self.layers[self.subgrids[:, 7] == 0]
        if keep.size == 0:
            return 0, 1
        return int(keep.min()), int(keep.max() - keep.min() + 1)


def plan(geom: Geometry, uvw: np.ndarray, freqs: np.ndarray, aterm_offsets: np.ndarray) -> Plan:
    """Partition the visibilities into subgrids (Section 3.1)."""
    lib = _load()
    uvw = np.ascontiguousarray(uvw, dtype=np.float64)
    freqs = np.ascontiguousarray(freqs, dtype=np.float64)
    offs = np.ascontiguousarray(aterm_offsets, dtype=np.int32)
    n_bl, n_t, _ = uvw.shape
    n_ch = freqs.shape[0]
    n_int = offs.shape[0] - 1
    cap = max(64, n_bl * max(n_t, 1) * max(n_ch, 1) + 1)
    cap = min(cap, 1 << 24)
    while True:
        sg = np.zeros((cap, 8), np.int32)
        seg = np.zeros((cap, 4), np.int32)
        lay = np.zeros(cap, np.int32)
        cj = np.zeros(cap, np.int32)
        w_step = ctypes.c_double(0.0)
        nsg = ctypes.c_int(0)
        nseg = ctypes.c_int(0)
        st = lib.oracle_plan(geom.grid_size, geom.subgrid_size, geom.kernel_padding, geom.image_size,
                             geom.flags, n_bl, n_t, n_ch, _ptr(uvw), _ptr(freqs), _ptr(offs), n_int,
                             _ptr(sg), cap, ctypes.byref(nsg), _ptr(seg), cap, ctypes.byref(nseg),
                             _ptr(lay), _ptr(cj), ctypes.byref(w_step))
        if st == 9:
            cap *= 2
            continue
        if st != 0:
            raise OracleError(st, "plan")
        layered = bool(geom.flags & FLAG_W_LAYERS)
        layers = lay[: nsg.value].copy() if layered else None
        conj = cj[: nsg.value].copy() if layered else None
        return Plan(sg[: nsg.value].copy(), seg[: nseg.value].copy(), layers, float(w_step.value), conj)


def _common(geom, baselines, uvw, freqs, aterm_offsets, pl, n_st):
    uvw = np.ascontiguousarray(uvw, dtype=np.float64)
    freqs = np.ascontiguousarray(freqs, dtype=np.float64)
    bl = np.ascontiguousarray(baselines, dtype=np.int32)
    tu = None if geom.taper_user is None else np.ascontiguousarray(geom.taper_user, dtype=np.float64)
    sg = np.ascontiguousarray(pl.subgrids, dtype=np.int32)
    seg = np.ascontiguousarray(pl.segments, dtype=np.int32)
    n_bl, n_t, _ = uvw.shape
    lay = None if pl.layers is None else np.ascontiguousarray(pl.layers, dtype=np.int32)
    cj = None if pl.conj is None else np.ascontiguousarray(pl.conj, dtype=np.int32)
    k_min, _ = pl.k_range
    args = [geom.grid_size, geom.subgrid_size, geom.kernel_padding, geom.image_size, geom.taper_kind,
            geom.beta, _ptr(tu), geom.aterm_nodes, n_st, n_bl, n_t, freqs.shape[0], _ptr(bl), _ptr(uvw),
            _ptr(freqs), len(aterm_offsets) - 1, _ptr(sg), sg.shape[0], _ptr(seg), seg.shape[0],
            _ptr(lay), _ptr(cj), pl.w_step, k_min, n_pol(geom)]
    keep = (uvw, freqs, bl, tu, sg, seg, lay, cj)
    return args, keep


def n_pol(geom: Geometry) -> int:
    """Planes of the master grid and the image: 4 correlations, or 1 with
    FLAG_STOKES_I (I = (XX + YY) / 2; an unpolarised model predicts XX = YY = I)."""
    return 1 if geom.flags & FLAG_STOKES_I else 4


def grid_shape(geom: Geometry, pl: Plan) -> tuple:
    """[npol][N][N] without w layers, [n_layers][npol][N][N] with them
    (npol = 4, or 1 with FLAG_STOKES_I)."""
    N, npol = geom.grid_size, n_pol(geom)
    return (pl.k_range[1], npol, N, N) if pl.layers is not None else (npol, N, N)


def grid(geom: Geometry, n_st: int, baselines, uvw, freqs, aterm_offsets, pl: Plan, vis, aterms,
         grid_in=None, want_subgrids: bool = False, normalize: bool = False):
    """Grid visibilities (complex [n_bl][n_t][n_ch][4]) with A-terms
    (complex [n_int][n_st][nodes][nodes][4]) onto a complex128 [4][N][N] grid.
    Returns grid (and the subgrid images before / after the FFT if asked).
    normalize: A-term power normalisation (Section 3.3): every segment's
    corrected image is divided per pixel by f = ||A_p^H A_q||_F; the result
    is then (grid, weights) (plus the subgrid images if asked), weights
    float64 [L*L + 1] = sum n_seg / f on the subgrid lattice ([j][i]
    flattened) and sum n_seg in the last slot."""
    lib = _load()
    args, keep = _common(geom, baselines, uvw, freqs, aterm_offsets, pl, n_st)
    v = np.ascontiguousarray(vis, dtype=np.complex128)
    a = np.ascontiguousarray(aterms, dtype=np.complex128)
    N, L = geom.grid_size, geom.subgrid_size
    g = np.zeros(grid_shape(geom, pl), np.complex128) if grid_in is None else \
        np.array(grid_in, dtype=np.complex128, copy=True)
    img = uv = None
    if want_subgrids:
        img = np.zeros((pl.subgrids.shape[0], n_pol(geom), L, L), np.complex128)
        uv = np.zeros_like(img)
    w = np.zeros(L * L + 1, np.float64) if normalize else None
    st = lib.oracle_grid(*args, _ptr(v), _ptr(a), _ptr(g), _ptr(img), _ptr(uv), int(normalize), _ptr(w))
    if st != 0:
        raise OracleError(st, "grid")
    del keep
    out = (g, w) if normalize else (g,)
    if want_subgrids:
        out = out + (img, uv)
    return out if len(out) > 1 else g


def lattice_to_image(values: np.ndarray, N: int, L: int) -> np.ndarray:
    """Bilinear interpolation of a [L][L] map on the subgrid lattice
    (l_i = (i - L/2) FOV/L) to the N x N image (l_p = (p - N/2) FOV/N), i.e.
    at the fractional lattice index (p - N/2) L/N + L/2; beyond the last
    lattice point the map is extended flat.  Returns [q][p]."""
    v = np.asarray(values, np.float64).reshape(L, L)
    f = (np.arange(N) - N // 2) * (L / N) + L // 2
    i0 = np.clip(np.floor(f).astype(int), 0, L - 2)
    fr = np.clip(f - i0, 0.0, 1.0)
    # along i (columns) then j (rows)
    rows = v[:, i0] * (1.0 - fr)[None, :] + v[:, i0 + 1] * fr[None, :]          # [j][p]
    return rows[i0, :] * (1.0 - fr)[:, None] + rows[i0 + 1, :] * fr[:, None]    # [q][p]


def degrid(geom: Geometry, n_st: int, baselines, uvw, freqs, aterm_offsets, pl: Plan, grid_arr, aterms):
    """Predict visibilities complex128 [n_bl][n_t][n_ch][4] from a [npol][N][N]
    grid (4 correlation planes, or the Stokes-I plane with FLAG_STOKES_I)."""
    lib = _load()
    args, keep = _common(geom, baselines, uvw, freqs, aterm_offsets, pl, n_st)
    gr = np.ascontiguousarray(grid_arr, dtype=np.complex128)
    a = np.ascontiguousarray(aterms, dtype=np.complex128)
    n_bl, n_t = np.shape(uvw)[:2]
    out = np.zeros((n_bl, n_t, len(freqs), 4), np.complex128)
    st = lib.oracle_degrid(*args, _ptr(gr), _ptr(a), _ptr(out))
    if st != 0:
        raise OracleError(st, "degrid")
    del keep
    return out


def taper(L: int, beta: float, kind: int = 0, user=None) -> np.ndarray:
    lib = _load()
    out = np.zeros(L, np.float64)
    u = None if user is None else np.ascontiguousarray(user, dtype=np.float64)
    st = lib.oracle_taper(L, kind, beta, _ptr(u), _ptr(out))
    if st != 0:
        raise OracleError(st, "taper")
    return out


def bessel_i0(x: float) -> float:
    return float(_load().oracle_bessel_i0(float(x)))


def dft2(planes: np.ndarray, sign: int) -> np.ndarray:
    """Centred unnormalised 2-D DFT of [..., L, L] planes (sign -1 forward)."""
    lib = _load()
    a = np.ascontiguousarray(planes, dtype=np.complex128)
    L = a.shape[-1]
    flat = a.reshape(-1, L, L)
    out = np.zeros_like(flat)
    st = lib.oracle_dft2(L, sign, flat.shape[0], _ptr(flat), _ptr(out))
    if st != 0:
        raise OracleError(st, "dft2")
    return out.reshape(a.shape)


def aterm_interp(A: np.ndarray, L: int) -> np.ndarray:
    """Interpolate one station's [nodes][nodes][4] Jones samples to [L][L][4]."""
    lib = _load()
    a = np.ascontiguousarray(A, dtype=np.complex128)
    out = np.zeros((L, L, 4), np.complex128)
    st = lib.oracle_aterm_interp(a.shape[0], L, _ptr(a), _ptr(out))
    if st != 0:
        raise OracleError(st, "aterm_interp")
    return out


def _centre_signs(N: int) -> np.ndarray:
    """(-1)^(x+y) on an N x N plane: with it, a plain FFT of even length N is
    the centred transform sum_X f(X) e^{-+2 pi i (X - N/2)(p - N/2)/N}."""
    s = (-1.0) ** np.arange(N)
    return np.outer(s, s)


def image_taper(geom: Geometry) -> np.ndarray:
    """T(l_p) T(m_q) on the master image, l_p = (p - N/2) FOV/N ([q][p])."""
    if geom.taper_kind != 0:
        raise ValueError("the image-domain wrapper needs the Kaiser-Bessel taper")
    t = taper(geom.grid_size, geom.beta)
    return np.outer(t, t)


def _nprime_image(geom: Geometry) -> np.ndarray:
    """n'(l_p, m_q) = sqrt(1 - l^2 - m^2) - 1 on the master image ([q][p])."""
    N, fov = geom.grid_size, geom.image_size
    l = (np.arange(N) - N // 2) * fov / N
    return np.sqrt(1.0 - l[None, :] ** 2 - l[:, None] ** 2) - 1.0


def invert(geom: Geometry, n_st: int, baselines, uvw, freqs, aterm_offsets, pl: Plan, vis, aterms,
           normalize: bool = False):
    """Dirty image, complex128 [npol][N][N] indexed [pol][q][p] at (l_p, m_q):
    I = sum_layers e^{+2 pi i w0 n'} sum_{X,Y} G_w0(X,Y) e^{+2 pi i (u_X l_p + v_Y m_q)}
        / (L^2 T(l_p) T(m_q)),
    G_w0 the visibilities gridded onto layer w0 (Eq. 11; one layer w0 = 0
    without w layers).  With w layers the rows of negative w are gridded as
    their mirrors (V^H at -uvw, Section 2.4 footnote), so each contributes
    the conjugate transpose of its own term: the Hermitian part of the image
    is that of the visibilities as given.  The L^2 T T factor is what the gridder puts on every
    image point (taper once per direction, unnormalised L x L transforms);
    dividing it out is Eq. 11's 1/T correction.
    normalize (Section 3.3): the gridding divides every segment by
    f = ||A_p^H A_q||_F and the image is then divided by the weighted
    average of that factor, W = (sum n_seg / f) / (sum n_seg) on the subgrid
    lattice, interpolated to the image pixels (lattice_to_image)."""
    N, L = geom.grid_size, geom.subgrid_size
    if N % 2:
        raise ValueError("N must be even")
    if normalize:
        G, W = grid(geom, n_st, baselines, uvw, freqs, aterm_offsets, pl, vis, aterms, normalize=True)
    else:
        G = grid(geom, n_st, baselines, uvw, freqs, aterm_offsets, pl, vis, aterms)
    S = _centre_signs(N)
    layers = G[None] if pl.layers is None else G
    k_min, _ = pl.k_range
    n1 = _nprime_image(geom)
    img = np.zeros((n_pol(geom), N, N), np.complex128)
    for li, Gl in enumerate(layers):
        w0 = pl.w0(k_min + li)
        part = np.fft.ifft2(Gl * S[None], axes=(-2, -1)) * float(N) * float(N) * S[None]
        img += part * np.exp(2j * np.pi * w0 * n1)[None]
    img = img / (float(L) * float(L) * image_taper(geom)[None])
    if normalize:
        img = img / lattice_to_image(W[: L * L] / W[L * L], N, L)[None]
    return img


def predict(geom: Geometry, n_st: int, baselines, uvw, freqs, aterm_offsets, pl: Plan, image, aterms):
    """Visibilities of an image (the adjoint of invert): each layer's model
    grid G_w0(X,Y) = sum_{p,q} I e^{-2 pi i w0 n'} e^{-2 pi i (u_X l_p + v_Y m_q)}
    / (L^2 T(l_p) T(m_q)) (Eq. 12), then degrid.  With the degridder's own
    taper this predicts Eq. 1 on the image's pixels."""
    N, L = geom.grid_size, geom.subgrid_size
    if N % 2:
        raise ValueError("N must be even")
    S = _centre_signs(N)
    src = np.asarray(image, np.complex128) / (float(L) * float(L) * image_taper(geom)[None])
    k_min, n_layers = pl.k_range
    n1 = _nprime_image(geom)
    G = np.zeros(grid_shape(geom, pl), np.complex128)
    for li in range(n_layers):
        w0 = pl.w0(k_min + li)
        Gl = np.fft.fft2(src * np.exp(-2j * np.pi * w0 * n1)[None] * S[None], axes=(-2, -1)) * S[None]
        if pl.layers is None:
            G = Gl
        else:
            G[li] = Gl
    return degrid(geom, n_st, baselines, uvw, freqs, aterm_offsets, pl, G, aterms)
