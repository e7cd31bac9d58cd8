"""Independent brute-force computations used to pin the oracle.

Nothing here reuses the oracle's code: each function restates a textbook
definition (the discrete measurement equation, a Fourier sum over the grid,
bilinear interpolation through numpy.interp, scipy's Bessel I0) so that a
mistake in the oracle (a dropped term, a wrong sign or index, a transposed
operand) shows up as a mismatch.
"""
from __future__ import annotations

import numpy as np
import scipy.special

from paper_2502_17789_gb300 import synth

C = 299792458.0


def tiny_observation(seed=0, n_st=4, n_t=3, n_ch=4, N=64, L=16, P=6, fov=0.3, diameter=100.0,
                     f0=150e6, df=1e6, steps_per_interval=None, dt=8.0, enu=None):
    rng = np.random.default_rng(seed)
    enu = synth.stations_uniform_disk(rng, n_st, diameter) if enu is None else np.asarray(enu, float)
    freqs = f0 + df * np.arange(n_ch)
    spi = n_t if steps_per_interval is None else steps_per_interval
    return synth.make_observation(enu, n_t, dt, freqs, spi, N, L, P, fov)


def uvw_lambda(obs):
    """u, v, w in wavelengths, each [n_bl, n_t, n_ch]."""
    f = obs.freqs[None, None, :] / C
    return (obs.uvw[..., 0:1] * f, obs.uvw[..., 1:2] * f, obs.uvw[..., 2:3] * f)


def kb_taper(L, beta):
    x = (2.0 * np.arange(L) - L) / L
    return scipy.special.i0(beta * np.sqrt(np.clip(1.0 - x * x, 0.0, None))) / scipy.special.i0(beta)


def bilinear_at(A_nodes, fov, l, m):
    """Interpolate one station's [nodes][nodes][4] samples (node (a_m, a_l)) at
    direction (l, m) with numpy.interp along l, then along m."""
    nodes = A_nodes.shape[0]
    c = -0.5 * fov + fov * np.arange(nodes) / (nodes - 1)
    out = np.zeros(4, np.complex128)
    for e in range(4):
        rows = np.array([np.interp(l, c, A_nodes[a, :, e].real) + 1j * np.interp(l, c, A_nodes[a, :, e].imag)
                         for a in range(nodes)])
        out[e] = np.interp(m, c, rows.real) + 1j * np.interp(m, c, rows.imag)
    return out.reshape(2, 2)


def image_from_grid(G, fov, l, m):
    """Dirty image of a [4][N][N] uv grid at (l, m): sum over every grid cell
    of G e^{+2 pi i (u l + v m)}, u = (X - N/2)/FOV.  Returns 2x2."""
    N = G.shape[-1]
    u = (np.arange(N) - N // 2) / fov
    ex = np.exp(2j * np.pi * u * l)
    ey = np.exp(2j * np.pi * u * m)
    return np.einsum("pyx,y,x->p", G, ey, ex).reshape(2, 2)


def dft_image(obs, vis, aterm_nodes_per_interval, l, m, pol_sel=None):
    """Adjoint of the discrete measurement equation (Eq. 1) at one direction:
    sum_k A_p(l,m)^H V_k A_q(l,m) e^{+2 pi i (u_k l + v_k m + w_k n')}.
    aterm_nodes_per_interval: [n_int][n_st][nodes][nodes][4] complex."""
    u, v, w = uvw_lambda(obs)
    n1 = np.sqrt(1.0 - l * l - m * m) - 1.0
    ph = np.exp(2j * np.pi * (u * l + v * m + w * n1))                   # [bl, t, ch]
    out = np.zeros((2, 2), np.complex128)
    offs = obs.aterm_offsets
    for a in range(obs.n_intervals):
        t0, t1 = offs[a], offs[a + 1]
        if t1 <= t0:
            continue
        for b, (p, q) in enumerate(obs.baselines):
            Ap = bilinear_at(aterm_nodes_per_interval[a, p], obs.image_size, l, m)
            Aq = bilinear_at(aterm_nodes_per_interval[a, q], obs.image_size, l, m)
            S = np.einsum("tc,tce->e", ph[b, t0:t1], vis[b, t0:t1].astype(np.complex128)).reshape(2, 2)
            out += Ap.conj().T @ S @ Aq
    return out


def measurement_equation(obs, aterm_nodes_per_interval, l, m, B):
    """Forward Eq. 1 for one point source of brightness B (2x2) at (l, m):
    V_k = A_p B A_q^H e^{-2 pi i (u l + v m + w n')}, [n_bl, n_t, n_ch, 4]."""
    u, v, w = uvw_lambda(obs)
    n1 = np.sqrt(1.0 - l * l - m * m) - 1.0
    ph = np.exp(-2j * np.pi * (u * l + v * m + w * n1))
    out = np.zeros(ph.shape + (4,), np.complex128)
    for a in range(obs.n_intervals):
        t0, t1 = obs.aterm_offsets[a], obs.aterm_offsets[a + 1]
        for b, (p, q) in enumerate(obs.baselines):
            Ap = bilinear_at(aterm_nodes_per_interval[a, p], obs.image_size, l, m)
            Aq = bilinear_at(aterm_nodes_per_interval[a, q], obs.image_size, l, m)
            J = (Ap @ B @ Aq.conj().T).reshape(4)
            out[b, t0:t1] = ph[b, t0:t1, :, None] * J[None, None, :]
    return out


def point_source_grid(N, fov, l, m, B):
    """Unnormalised Fourier transform of a point source: G[pol][Y][X] =
    B e^{-2 pi i (u_X l + v_Y m)}, u_X = (X - N/2)/FOV."""
    u = (np.arange(N) - N // 2) / fov
    e = np.exp(-2j * np.pi * u[None, :] * l) * np.exp(-2j * np.pi * u[:, None] * m)
    return np.asarray(B, np.complex128).reshape(4)[:, None, None] * e[None]


def convolutional_grid(obs, pl, vis, aterms, T, w0=0.0):
    """Textbook convolutional gridding, visibility-major: every visibility
    adds V_k convolved with its own kernel
      K_k(dx, dy) = sum_{ij} T_i T_j A_p^H [.] A_q e^{2 pi i [dx (i-L/2) + dy (j-L/2)]/L + 2 pi i w_k n'_ij}
    sampled at the L x L cells of its subgrid's footprint (Section 2.1, Eq. 2
    written for the subgrid's pixel kernel).  O(n_vis L^4): tiny inputs only."""
    N, L, fov = obs.grid_size, obs.subgrid_size, obs.image_size
    G = np.zeros((4, N, N), np.complex128)
    u, v, w = uvw_lambda(obs)
    idx = np.arange(L) - L // 2
    lm = idx * fov / L
    n1 = np.sqrt(1.0 - lm[None, :] ** 2 - lm[:, None] ** 2) - 1.0        # [j, i]
    nodes = aterms.shape[2]
    for s, row in enumerate(pl.subgrids):
        b, t0, t1, c0, c1, x0, y0, dropped = [int(z) for z in row]
        if dropped:
            continue
        p, q = obs.baselines[b]
        segs = pl.segments[pl.segments[:, 0] == s]
        for (_, a, tb, te) in segs:
            # interpolated A on every pixel, independent evaluation
            Ap = np.array([[bilinear_at(aterms[a, p], fov, lm[i], lm[j]) for i in range(L)] for j in range(L)])
            Aq = np.array([[bilinear_at(aterms[a, q], fov, lm[i], lm[j]) for i in range(L)] for j in range(L)])
            for t in range(tb, te):
                for c in range(c0, c1):
                    xi = u[b, t, c] * fov + N // 2
                    eta = v[b, t, c] * fov + N // 2
                    V = vis[b, t, c].astype(np.complex128).reshape(2, 2)
                    # per-pixel corrected matrix  T_i T_j A_p^H V A_q
                    M = np.einsum("jira,ab,jibc->jirc", Ap.conj().transpose(0, 1, 3, 2), V, Aq)
                    M *= (T[None, :] * T[:, None])[..., None, None]
                    wph = np.exp(2j * np.pi * (w[b, t, c] - w0) * n1)            # [j, i]
                    X = np.arange(x0, x0 + L)
                    Y = np.arange(y0, y0 + L)
                    ex = np.exp(2j * np.pi * np.outer(xi - X, idx) / L)          # [X, i]
                    ey = np.exp(2j * np.pi * np.outer(eta - Y, idx) / L)         # [Y, j]
                    K = np.einsum("Yj,Xi,jirc->rcYX", ey, ex, M * wph[..., None, None])
                    G[:, y0:y0 + L, x0:x0 + L] += K.reshape(4, L, L)
    return G


def mirrored_set(obs, vis):
    """The visibility set as gridded with w layers (Section 2.4 footnote,
    V(u,v,w) = V(-u,-v,-w)^H): every timestep row with w < 0 is replaced by
    its mirror, the conjugate transpose of V on baseline (q, p) at -uvw.
    Returned as an observation with twice the baselines -- the originals
    keep the rows of w >= 0, the appended reversed baselines hold the
    mirrored rows -- and its visibilities (zero where a row is absent), so
    that dft_image and measurement_equation apply unchanged."""
    import copy
    neg = obs.uvw[..., 2] < 0.0                                           # [bl, t]
    o2 = copy.copy(obs)
    o2.baselines = np.concatenate([obs.baselines, obs.baselines[:, ::-1]]).astype(np.int32)
    o2.uvw = np.concatenate([obs.uvw, -obs.uvw])
    v = np.asarray(vis, np.complex128)
    herm = v.reshape(v.shape[:3] + (2, 2)).conj().swapaxes(-1, -2).reshape(v.shape)
    v2 = np.concatenate([np.where(neg[..., None, None], 0.0, v), np.where(neg[..., None, None], herm, 0.0)])
    return o2, v2
