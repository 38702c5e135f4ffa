"""Seeded synthetic inputs for the AXB = C solvers.

This module is shared by the CPU oracle tests, the GPU tests and the benchmark.
It only draws random numbers and forms the problem data (C = A X* B plus
optional noise); it holds none of the solver's arithmetic.

Shapes follow the paper's workloads (Section 5 tables, Section 6 images) and
the benchmark configurations:

* ``gaussian``          -- i.i.d. N(0, s^2) A, B, X*, consistent C (Ex. 5.2 "randn" sets)
* ``config_small``      -- A 200x100, B 80x150, X* 100x80, all N(0,1)
* ``config_scale``      -- A = U diag(sigma) V^T (Haar U, V; sigma log-spaced 1 -> 1e-2),
                           4000x1000 and 800x3000, optional rank-deficient variant
* ``config_precision``  -- A 20000x2000, B 2000x20000 with N(0, 1/cols) entries
* ``color_images`` / ``blur_systems`` -- piecewise-smooth synthetic RGB images, banded
                           Toeplitz Gaussian blurs, C = A X B + noise per channel
* ``duplicated``        -- [A;A] / [B,B] rank-deficient sets (Table 1 set 6, Table 7)
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20240810


def rng(tag: int) -> np.random.Generator:
    return np.random.default_rng(BASE_SEED + int(tag))


def gaussian(m, p, q, n, seed=0, a_scale=1.0, b_scale=1.0, x_scale=1.0, noise=0.0):
    """A (m x p), B (q x n), X* (p x q) i.i.d. Gaussian; C = A X* B (+ noise)."""
    g = rng(1000 + seed)
    A = g.standard_normal((m, p)) * a_scale
    B = g.standard_normal((q, n)) * b_scale
    Xs = g.standard_normal((p, q)) * x_scale
    C = A @ Xs @ B
    if noise > 0:
        C = C + g.standard_normal(C.shape) * noise
    return A, B, C, Xs


def config_small(seed=1):
    """A 200x100, B 80x150 i.i.d. N(0,1), X* 100x80 N(0,1), C = A X* B."""
    g = rng(seed)
    A = g.standard_normal((200, 100))
    B = g.standard_normal((80, 150))
    Xs = g.standard_normal((100, 80))
    return A, B, A @ Xs @ B, Xs


def haar(g, rows, cols):
    """rows x cols matrix with orthonormal columns, Haar distributed (QR of a
    Gaussian with the signs of R's diagonal folded into Q)."""
    Q, Rq = np.linalg.qr(g.standard_normal((rows, cols)))
    return Q * np.sign(np.diag(Rq))[None, :]


def lowrank_logspaced(g, rows, cols, rank, smax=1.0, smin=1e-2):
    U = haar(g, rows, rank)
    V = haar(g, cols, rank)
    sig = np.logspace(np.log10(smax), np.log10(smin), rank)
    return (U * sig[None, :]) @ V.T


def config_scale(rank_deficient=False, seed=2, m=4000, p=1000, q=800, n=3000):
    """A = U diag(sigma) V^T (m x p), B likewise (q x n), sigma log-spaced 1 -> 1e-2.
    The rank-deficient variant uses rank 600 for A and 500 for B."""
    g = rng(seed)
    ra = 600 if rank_deficient else min(m, p)
    rb = 500 if rank_deficient else min(q, n)
    A = lowrank_logspaced(g, m, p, ra)
    B = lowrank_logspaced(g, q, n, rb)
    Xs = g.standard_normal((p, q))
    return A, B, A @ Xs @ B, Xs


def config_precision(m=20000, p=2000, q=2000, n=20000, noise=0.0, seed=3, dtype=np.float64):
    """A m x p with N(0, 1/p) entries, B q x n with N(0, 1/n) entries, X* N(0,1),
    C = A X* B (+ N(0, noise^2)).  The full size is 20000x2000 / 2000x20000; the
    2000x200 / 200x2000 slice is the same recipe at smaller sizes."""
    g = rng(seed)
    A = (g.standard_normal((m, p), dtype=np.float64) / np.sqrt(p)).astype(dtype)
    B = (g.standard_normal((q, n), dtype=np.float64) / np.sqrt(n)).astype(dtype)
    Xs = g.standard_normal((p, q), dtype=np.float64).astype(dtype)
    C = (A @ Xs) @ B
    if noise > 0:
        C = C + (g.standard_normal(C.shape) * noise).astype(dtype)
    return A, B, C, Xs


def duplicated(m, p, q, n, seed=4, how="rows"):
    """Rank-deficient pairs by duplication: A = [A0; A0] (2m x p) and
    B = [B0, B0] (q x 2n) (how='rows'), or A = [A0, A0], B = [B0; B0] (how='cols')."""
    g = rng(5000 + seed)
    A0 = g.standard_normal((m, p))
    B0 = g.standard_normal((q, n))
    if how == "rows":
        A = np.vstack([A0, A0])
        B = np.hstack([B0, B0])
    else:
        A = np.hstack([A0, A0])
        B = np.vstack([B0, B0])
    Xs = g.standard_normal((A.shape[1], B.shape[0]))
    return A, B, A @ Xs @ B, Xs


# ---------------------------------------------------------------------------
# Colour images (Section 6 application) -- synthetic stand-ins
# ---------------------------------------------------------------------------

def _polygon_mask(yy, xx, cx, cy, radii, phase):
    """Star-shaped polygon around (cx, cy): vertex k at angle phase + 2 pi k / K
    and radius radii[k]; a pixel is inside when its radius is below the
    piecewise-linear interpolation of the vertex radii at its angle.
    yy, xx: pixel coordinates of the region to test."""
    dx, dy = xx - cx, yy - cy
    ang = (np.arctan2(dy, dx) - phase) % (2 * np.pi)
    K = len(radii)
    seg = ang / (2 * np.pi) * K
    k0 = np.floor(seg).astype(np.int64) % K
    k1 = (k0 + 1) % K
    f = seg - np.floor(seg)
    rad = radii[k0] * (1 - f) + radii[k1] * f
    return np.hypot(dx, dy) <= rad


def color_image(g, h, w):
    """h x w x 3 image in [0,1]: a linear gradient background plus 3-8 random
    star-shaped polygons of constant colour, each with its own gradient."""
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    img = np.empty((h, w, 3))
    for c in range(3):
        a, b, d = g.uniform(-0.5, 0.5, 3)
        img[:, :, c] = 0.5 + a * (xx / w - 0.5) + b * (yy / h - 0.5) + 0.2 * d
    for _ in range(int(g.integers(3, 9))):
        K = int(g.integers(3, 9))
        cx, cy = g.uniform(0, w), g.uniform(0, h)
        base = g.uniform(0.08, 0.35) * min(h, w)
        radii = base * g.uniform(0.5, 1.5, K)
        phase = g.uniform(0, 2 * np.pi)
        col = g.uniform(0, 1, 3)
        gx, gy = g.uniform(-0.3, 0.3, 2)
        # only the polygon's bounding box can be inside it
        rmax = float(np.max(radii))
        y0, y1 = max(0, int(np.floor(cy - rmax))), min(h, int(np.ceil(cy + rmax)) + 1)
        x0, x1 = max(0, int(np.floor(cx - rmax))), min(w, int(np.ceil(cx + rmax)) + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        sy, sx = yy[y0:y1, x0:x1], xx[y0:y1, x0:x1]
        mask = _polygon_mask(sy, sx, cx, cy, radii, phase)
        for c in range(3):
            region = img[y0:y1, x0:x1, c]
            region[mask] = (col[c] + gx * (sx - cx) / w + gy * (sy - cy) / h)[mask]
    return np.clip(img, 0.0, 1.0)


def gaussian_toeplitz(size, band, sigma):
    """size x size symmetric banded Toeplitz blur: taps exp(-k^2 / (2 sigma^2))
    for |k| <= band // 2, normalised to sum 1, zero boundary conditions."""
    half = band // 2
    k = np.arange(-half, half + 1)
    taps = np.exp(-(k ** 2) / (2.0 * sigma ** 2))
    taps /= taps.sum()
    T = np.zeros((size, size))
    for off, t in zip(k, taps):
        idx = np.arange(max(0, -off), min(size, size - off))
        T[idx, idx + off] = t
    return T


def _image_params(index, seed, min_side, max_side):
    """Sizes, blur and image of image `index` from its own stream
    (seed sequence [base, seed, index, 0]); the image is rounded to FP32."""
    g = np.random.default_rng([BASE_SEED, int(seed), int(index), 0])
    h = int(g.integers(min_side // 16, max_side // 16 + 1)) * 16
    w = int(g.integers(min_side // 16, max_side // 16 + 1)) * 16
    band = int(g.choice([7, 9, 11, 13, 15]))
    sig = float(g.uniform(1.5, 3.0))
    img = color_image(g, h, w).astype(np.float32)
    return h, w, band, sig, img


def _image_job(args):
    return _image_params(*args)


def _systems_from(index, seed, noise, mild, params):
    h, w, band, sig, img = params
    A = gaussian_toeplitz(h, band, sig)
    B = gaussian_toeplitz(w, band, sig)
    if mild:
        A = 0.5 * (np.eye(h) + A)
        B = 0.5 * (np.eye(w) + B)
    gn = np.random.default_rng([BASE_SEED, int(seed), int(index), 1])
    out = []
    for c in range(3):
        X = img[:, :, c].astype(np.float64)
        E = gn.standard_normal((h, w)) * noise
        out.append(dict(A=A, B=B, C=A @ X @ B + E, X=X, E=E, image=int(index), channel=c))
    return out


def blur_image_systems(index, seed=4, min_side=128, max_side=512, noise=1e-3, mild=False):
    """The three channel systems of image `index`: sides h, w uniform in
    [min_side, max_side] (multiples of 16), band b in {7, 9, ..., 15},
    sigma_blur in [1.5, 3]; A (h x h) and B (w x w) symmetric Toeplitz blurs;
    per channel C = A X B + N(0, noise^2).  Each image has its own random
    streams, so images can be generated in any order or in parallel.
    ``mild`` replaces each blur T by (I + T) / 2 (a well-conditioned control)."""
    return _systems_from(index, seed, noise, mild, _image_params(index, seed, min_side, max_side))


def blur_systems(n_images=64, seed=4, min_side=128, max_side=512, noise=1e-3, mild=False, first=0,
                 processes=1):
    """Systems of images first .. first + n_images - 1 (3 per image, see
    blur_image_systems), as a list of dicts with keys A, B, C, X (clean
    channel), E (noise), image, channel.  processes > 1 draws the images in a
    spawn-started process pool (identical result)."""
    jobs = [(first + i, seed, min_side, max_side) for i in range(n_images)]
    if processes > 1 and n_images > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            params = pool.map(_image_job, jobs, chunksize=max(1, n_images // (4 * processes)))
    else:
        params = [_image_job(j) for j in jobs]
    out = []
    for (idx, *_), pr in zip(jobs, params):
        out += _systems_from(idx, seed, noise, mild, pr)
    return out


# ---------------------------------------------------------------------------
# Sparse test matrices (Section 5, Tables 3, 5, 7: MATLAB sprandn sets)
# ---------------------------------------------------------------------------

def sprand_gaussian(g, rows, cols, density, full_rank=True, tries=50):
    """rows x cols matrix with about density * rows * cols N(0,1) nonzeros at
    uniformly random positions (a stand-in for MATLAB's sprandn, whose random
    stream and condition-number construction are not reproduced); with
    full_rank, redrawn until its rank is min(rows, cols).  Dense numpy array."""
    for _ in range(tries):
        M = np.where(g.random((rows, cols)) < density, g.standard_normal((rows, cols)), 0.0)
        if not full_rank or np.linalg.matrix_rank(M) == min(rows, cols):
            return M
    raise RuntimeError("no full-rank draw")


# (A shape, A density), (B shape, B density) of the paper's sprandn sets
SPARSE_SETS = {
    "table3_set3": ((210, 20, 0.05), (40, 270, 0.05)),
    "table3_set6": ((160, 35, 0.05), (25, 150, 0.08)),
    "table5_set3": ((25, 205, 0.08), (125, 40, 0.05)),
    "table5_set6": ((130, 320, 0.05), (435, 170, 0.02)),
}


def sparse_set(name, seed=6):
    """A, B (dense arrays with the set's sparsity), X* N(0,1), C = A X* B."""
    (m, p, da), (q, n, db) = SPARSE_SETS[name]
    g = rng(7000 + seed + 17 * sorted(SPARSE_SETS).index(name))
    A = sprand_gaussian(g, m, p, da)
    B = sprand_gaussian(g, q, n, db)
    Xs = g.standard_normal((p, q))
    return A, B, A @ Xs @ B, Xs


# ---------------------------------------------------------------------------
# Section 6 colour model: B = A X A_c^T + E, X = (vec X_r, vec X_g, vec X_b)
# ---------------------------------------------------------------------------

# cross-channel blur of Section 6
A_CROSS = np.array([[0.9, 0.05, 0.05],
                    [0.0, 0.9, 0.1],
                    [0.05, 0.1, 0.85]])

# the four test images' sizes in Section 6 (face, bird, mandril, barbara)
COLOUR_SIZES = {"face": (92, 92), "bird": (96, 96), "mandril": (125, 120), "barbara": (240, 192)}


def gaussian_psf(size=5, sigma=6.0):
    """size x size taps exp(-(x^2 + y^2) / (2 sigma^2)), x, y centred, summing to 1
    (the G(5, 6) blur of Section 6: 5 x 5 with sigma 6)."""
    h = size // 2
    x = np.arange(-h, h + 1)
    P = np.exp(-(x[:, None] ** 2 + x[None, :] ** 2) / (2.0 * sigma ** 2))
    return P / P.sum()


def blur_operator(h, w, psf):
    """The within-channel blur A (hw x hw) acting on vec(X) (columns stacked, pixel
    (r, c) at index c h + r) as the 2-D convolution with the (symmetric) psf
    under zero boundary conditions, as CSR arrays (rowptr, colind, val) with
    ascending columns; scipy is not needed."""
    k = psf.shape[0] // 2
    rows, cols, vals = [], [], []
    rr, cc = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    idx = (cc * h + rr).ravel()
    r0, c0 = rr.ravel(), cc.ravel()
    for dc in range(-k, k + 1):          # neighbour columns first: ascending column index within a row
        for dr in range(-k, k + 1):
            r1, c1 = r0 + dr, c0 + dc
            ok = (r1 >= 0) & (r1 < h) & (c1 >= 0) & (c1 < w)
            rows.append(idx[ok])
            cols.append((c1 * h + r1)[ok])
            vals.append(np.full(int(ok.sum()), psf[dr + k, dc + k]))
    rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(h * w + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr).astype(np.int64), cols.astype(np.int32), vals


def csr_to_dense(rowptr, colind, val, cols):
    D = np.zeros((len(rowptr) - 1, cols))
    for i in range(len(rowptr) - 1):
        D[i, colind[rowptr[i]:rowptr[i + 1]]] = val[rowptr[i]:rowptr[i + 1]]
    return D


def csr_matvec(rowptr, colind, val, X):
    """A X for CSR A and dense X (rows of X gathered per nonzero)."""
    out = np.zeros((len(rowptr) - 1,) + X.shape[1:])
    rows = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    np.add.at(out, rows, val[:, None] * X[colind] if X.ndim == 2 else val * X[colind])
    return out


def colour_model(h, w, seed=9, index=0, noise=0.0, psf=None):
    """One synthetic colour image (h x w x 3, as color_image) and Section 6's
    model: A = blur_operator (CSR), B = A_c^T, X = (vec X_r, vec X_g, vec X_b)
    (hw x 3), C = A X B + N(0, noise^2).  Returns a dict with A (CSR triple), B,
    C, X, E, image, h, w."""
    g = np.random.default_rng([BASE_SEED, 600 + int(seed), int(index)])
    img = color_image(g, h, w)
    X = np.stack([img[:, :, c].T.ravel() for c in range(3)], axis=1)   # vec stacks columns
    A = blur_operator(h, w, gaussian_psf() if psf is None else psf)
    B = A_CROSS.T.copy()
    E = g.standard_normal((h * w, 3)) * noise
    C = csr_matvec(*A, X) @ B + E
    return dict(A=A, B=B, C=C, X=X, E=E, image=img, h=h, w=w)


def unvec_image(X, h, w):
    """h x w x 3 image from the hw x 3 matrix of stacked columns."""
    return np.stack([X[:, c].reshape(w, h).T for c in range(3)], axis=2)
