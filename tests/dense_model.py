"""Textbook dense matrices D, B, M_k of the image-formation model y_k = D B M_k x (Eq. 1).

Each factor is built on its own, entry by entry, from its definition, and multiplied with
numpy.  Used only to pin the oracle's loop implementation on tiny grids.
"""
import numpy as np


def idx(u, v, W):
    return u * W + v


def decimation(h, w, f):
    """D: (h*w) x (H*W), D[(i,j), (f i, f j)] = 1."""
    H, W = f * h, f * w
    D = np.zeros((h * w, H * W))
    for i in range(h):
        for j in range(w):
            D[i * w + j, idx(f * i, f * j, W)] = 1.0
    return D


def binning(h, w, f):
    """D with binning: (h*w) x (H*W), D[(i,j), (f i + a, f j + b)] = 1/f^2 for a, b in [0, f)."""
    H, W = f * h, f * w
    D = np.zeros((h * w, H * W))
    for i in range(h):
        for j in range(w):
            for a in range(f):
                for b in range(f):
                    D[i * w + j, idx(f * i + a, f * j + b, W)] = 1.0 / (f * f)
    return D


def blur(H, W, psf):
    """B: convolution with the PSF, zero outside the grid:
    (B z)(u, v) = sum_{a,b} h(a, b) z(u - a, v - b)."""
    S = psf.shape[0]
    R = S // 2
    B = np.zeros((H * W, H * W))
    for u in range(H):
        for v in range(W):
            for a in range(-R, R + 1):
                for b in range(-R, R + 1):
                    uu, vv = u - a, v - b
                    if 0 <= uu < H and 0 <= vv < W:
                        B[idx(u, v, W), idx(uu, vv, W)] += psf[a + R, b + R]
    return B


def motion(H, W, ty, tx):
    """M_k: integer translation, (M x)(u, v) = x(u + ty, v + tx), zero outside the grid."""
    M = np.zeros((H * W, H * W))
    for u in range(H):
        for v in range(W):
            uu, vv = u + ty, v + tx
            if 0 <= uu < H and 0 <= vv < W:
                M[idx(u, v, W), idx(uu, vv, W)] = 1.0
    return M


def motion_frac(H, W, sy, sx):
    """M_k for a real HR shift (sy, sx): bilinear interpolation, (M x)(u, v) = sum over the
    4 pixels (floor(u + sy) + p, floor(v + sx) + q), p, q in {0, 1}, of the weights
    (1 - a_y or a_y) (1 - a_x or a_x), a = the fractional parts; zero outside the grid."""
    ny, nx = int(np.floor(sy)), int(np.floor(sx))
    ay, ax = sy - ny, sx - nx
    M = np.zeros((H * W, H * W))
    for u in range(H):
        for v in range(W):
            for p, wy in ((0, 1 - ay), (1, ay)):
                for q, wx in ((0, 1 - ax), (1, ax)):
                    uu, vv = u + ny + p, v + nx + q
                    if wy * wx != 0 and 0 <= uu < H and 0 <= vv < W:
                        M[idx(u, v, W), idx(uu, vv, W)] += wy * wx
    return M


def system_matrices(h, w, f, shifts_lr, psf, binned=False):
    """A_k = D B M_k for every frame; psf is normalised to sum 1 here."""
    H, W = f * h, f * w
    psf = np.asarray(psf, dtype=np.float64)
    psf = psf / psf.sum()
    D = binning(h, w, f) if binned else decimation(h, w, f)
    B = blur(H, W, psf)
    out = []
    for dx, dy in shifts_lr:
        sy, sx = f * dy, f * dx
        if sy == round(sy) and sx == round(sx):
            M = motion(H, W, int(round(sy)), int(round(sx)))
        else:
            M = motion_frac(H, W, sy, sx)
        out.append(D @ B @ M)
    return out
