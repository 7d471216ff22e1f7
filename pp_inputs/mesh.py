"""Seeded mesh generators (inputs only).

Conventions shared by every consumer (they are part of the C-ABI contract):

* ``verts``  float64 [nv, 2] reference-configuration coordinates X (chord = 1,
  leading edge at the origin, free stream along +x).
* ``tris``   int32 [nt, 3] counter-clockwise vertex indices.
* ``ftag``   int32 [nt, 3] tag of local face f = edge (v_f, v_{(f+1)%3}):
  0 interior, 1 wall (airfoil, no-slip), 2 far field.
"""
import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    verts: np.ndarray
    tris: np.ndarray
    ftag: np.ndarray
    name: str = ""

    @property
    def nt(self):
        return int(self.tris.shape[0])

    @property
    def nv(self):
        return int(self.verts.shape[0])


def _naca_half_thickness(x, t=0.12):
    # Symmetric 4-digit thickness law, closed trailing-edge variant.
    x = np.clip(x, 0.0, 1.0)
    return 5.0 * t * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x**2
                      + 0.2843 * x**3 - 0.1036 * x**4)


def _orient_ccw(verts, tris):
    a = verts[tris[:, 0]]
    b = verts[tris[:, 1]]
    c = verts[tris[:, 2]]
    area2 = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    flip = area2 < 0
    tris = tris.copy()
    tris[flip, 1], tris[flip, 2] = tris[flip, 2].copy(), tris[flip, 1].copy()
    return tris


def _tag_faces(tris, ring_of_vertex, n_r):
    ftag = np.zeros(tris.shape, dtype=np.int32)
    for f in range(3):
        a = ring_of_vertex[tris[:, f]]
        b = ring_of_vertex[tris[:, (f + 1) % 3]]
        ftag[(a == 0) & (b == 0), f] = 1
        ftag[(a == n_r) & (b == n_r), f] = 2
    return ftag


def _wall_points(n_theta, thickness, clustering):
    """n_theta wall points, counter-clockwise from the trailing edge; 'arclength' spaces
    them uniformly in arc length (LE hit exactly for even n_theta), 'cosine' uses
    x = (1 + cos(beta))/2."""
    if clustering == "cosine":
        beta = 2.0 * np.pi * np.arange(n_theta) / n_theta
    else:
        bf = np.linspace(0.0, 2.0 * np.pi, 40001)
        xf = 0.5 * (1.0 + np.cos(bf))
        yf = _naca_half_thickness(xf, thickness) * np.where(np.sin(bf) >= 0, 1.0, -1.0)
        sf = np.concatenate([[0.0], np.cumsum(np.hypot(np.diff(xf), np.diff(yf)))])
        beta = np.interp(sf[-1] * np.arange(n_theta) / n_theta, sf, bf)
        if n_theta % 2 == 0:
            beta[n_theta // 2] = np.pi
    xw = 0.5 * (1.0 + np.cos(beta))
    yw = _naca_half_thickness(xw, thickness) * np.where(np.sin(beta) >= 0, 1.0, -1.0)
    yw[np.abs(np.sin(beta)) < 1e-14] = 0.0
    return beta, np.stack([xw, yw], 1)


_M64 = (1 << 64) - 1


def splitmix64(seed, counter):
    """Output number `counter` of the SplitMix64 generator started at `seed` (Steele, Lea and
    Flood, 2014): state = seed + (counter + 1) * 0x9E3779B97F4A7C15, then the published
    xor-shift-multiply finalizer.  Counter-based, so every consumer draws the same numbers."""
    z = (seed + (counter + 1) * 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def uniform_pm1(seed, counter):
    """A double in [-1, 1) from the top 53 bits of splitmix64(seed, counter)."""
    return -1.0 + 2.0 * ((splitmix64(seed, counter) >> 11) * (1.0 / 9007199254740992.0))


def ogrid(n_theta, n_r, seed=0, r_far=10.0, jitter=0.1, thickness=0.12, clustering="arclength"):
    """O-grid of 2*n_theta*n_r triangles around a symmetric 4-digit airfoil.  Interior vertex
    (k, j) moves by jitter * h * (u1, u2), h its distance to the nearest of its four grid
    neighbours at that moment (rings j = 1 .. n_r - 1 in order, k inner), u1, u2 the next two
    numbers of uniform_pm1(seed, .)."""
    beta, wall = _wall_points(n_theta, thickness, clustering)
    far = np.stack([0.5 + r_far * np.cos(beta), r_far * np.sin(beta)], 1)
    q = 1.0 + 4.0 / n_r
    s = (q ** np.arange(n_r + 1) - 1.0) / (q ** n_r - 1.0)
    P = wall[:, None, :] + s[None, :, None] * (far - wall)[:, None, :]  # [n_theta, n_r+1, 2]

    if n_r >= 2 and jitter > 0:
        draw = 0
        for j in range(1, n_r):
            for k in range(n_theta):
                x0, y0 = float(P[k, j, 0]), float(P[k, j, 1])
                h = None
                for kk, jj in (((k + 1) % n_theta, j), ((k - 1) % n_theta, j), (k, j + 1), (k, j - 1)):
                    dx, dy = x0 - float(P[kk, jj, 0]), y0 - float(P[kk, jj, 1])
                    d = math.sqrt(dx * dx + dy * dy)
                    h = d if h is None or d < h else h
                P[k, j, 0] = x0 + jitter * h * uniform_pm1(seed, draw)
                P[k, j, 1] = y0 + jitter * h * uniform_pm1(seed, draw + 1)
                draw += 2

    vid = np.arange(n_theta * (n_r + 1)).reshape(n_theta, n_r + 1)
    ring = np.tile(np.arange(n_r + 1), n_theta)
    tris = []
    for k in range(n_theta):
        k1 = (k + 1) % n_theta
        for j in range(n_r):
            a, b, c, d = vid[k, j], vid[k1, j], vid[k1, j + 1], vid[k, j + 1]
            if (k + j) % 2 == 0:
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, b, d), (b, c, d)]
    tris = _orient_ccw(P.reshape(-1, 2), np.asarray(tris, dtype=np.int32))
    ftag = _tag_faces(tris, ring, n_r)
    return Mesh(P.reshape(-1, 2).astype(np.float64), tris.astype(np.int32), ftag,
                name=f"ogrid{n_theta}x{n_r}s{seed}")


def box(nx, ny, seed=0, x0=-1.0, x1=2.0, y0=-1.0, y1=1.0, jitter=0.1):
    """Jittered rectangle of 2*nx*ny triangles, far-field tag on every boundary face."""
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    P = np.stack(np.meshgrid(xs, ys, indexing="ij"), -1).copy()  # [nx+1, ny+1, 2]
    rng = np.random.Generator(np.random.PCG64(seed))
    h = min((x1 - x0) / nx, (y1 - y0) / ny)
    for i in range(1, nx):
        for j in range(1, ny):
            P[i, j] += jitter * h * rng.uniform(-1.0, 1.0, 2)
    vid = np.arange((nx + 1) * (ny + 1)).reshape(nx + 1, ny + 1)
    tris = []
    for i in range(nx):
        for j in range(ny):
            a, b, c, d = vid[i, j], vid[i + 1, j], vid[i + 1, j + 1], vid[i, j + 1]
            if (i + j) % 2 == 0:
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, b, d), (b, c, d)]
    verts = P.reshape(-1, 2)
    tris = _orient_ccw(verts, np.asarray(tris, dtype=np.int32))
    on_bnd = np.zeros(len(verts), dtype=bool)
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    on_bnd[((ii == 0) | (ii == nx) | (jj == 0) | (jj == ny)).reshape(-1)] = True
    side = np.full(len(verts), -1)
    # an edge is on the boundary iff both endpoints lie on the same side of the box
    side_id = np.stack([(ii == 0), (ii == nx), (jj == 0), (jj == ny)], -1).reshape(-1, 4)
    ftag = np.zeros(tris.shape, dtype=np.int32)
    for f in range(3):
        a = tris[:, f]
        b = tris[:, (f + 1) % 3]
        same = np.any(side_id[a] & side_id[b], axis=1)
        ftag[same, f] = 2
    del side, on_bnd
    return Mesh(verts.astype(np.float64), tris.astype(np.int32), ftag, name=f"box{nx}x{ny}s{seed}")
