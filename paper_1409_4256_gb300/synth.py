"""Seeded synthetic inputs for EMC (Expand-Maximize-Compress) reconstructions.

This module produces INPUTS only: detector pixel coordinates on the Ewald sphere,
a particle made of Gaussian atoms, its intensity in closed form, uniformly random
true orientations, Poisson photon counts and a perturbed starting model. It holds
none of the reconstruction's arithmetic (no rotation sampling, no interpolation,
no likelihoods, no averaging) and is shared by the CPU oracle tests and the GPU
path alike. It imports nothing from the GPU binding or from the oracle.

Reading of the paper (Sec. 2.1): a frame K_k holds photon counts K_ik on a
discrete detector, each pixel i sitting at a point q_i of the Ewald sphere; the
frame is a slice W(R_k q_i) of the object's Fourier intensity at an unknown
rotation R_k. The paper gives no detector geometry and uses real (Mimivirus)
and synthetic (icosahedron) data that are not available here; the recipe below
stands in for them:

* Detector of D x D pixels, pixel centre (u, v) = (col - D/2 + 1/2, row - D/2 + 1/2),
  sample-detector distance D (same units). Scattered direction s = (u, v, D)/|.|,
  q = R_E (s - e_z), with R_E fixed so that |q| at the middle of a detector edge
  (u = D/2, v = 0) equals q_max = N/2 - 1 grid voxels. Pixels with |q| > q_max
  (the detector corners) are dropped, so every rotated pixel keeps all eight
  trilinear corners inside an N^3 grid centred at N/2.
* Particle: n_atoms Gaussian atoms (sigma in voxels) uniform in a ball of the
  given radius. Its intensity at a frequency point p (voxel-frequency units,
  zero frequency at the grid centre) is the squared modulus of the closed-form
  Fourier transform of the atoms,
      I(p) = exp(-4 pi^2 sigma^2 |p|^2 / N^2) |sum_a exp(-2 pi i p.x_a / N)|^2,
  which equals |FFT(rho)|^2 of the sampled density up to a constant factor and
  a negligible aliasing term. It is evaluated exactly at every rotated pixel, so
  the frames carry no interpolation error of their own.
* True orientations: Haar-uniform rotation matrices (QR of a Gaussian matrix
  with the sign fix), drawn from a seeded PCG64 stream.
* Counts: K_ik ~ Poisson(phi_k * s * I(R_k q_i)), with s chosen so that the mean
  expected count over used pixels and frames is the requested mean; phi_k = 1
  unless a log-normal fluence spread is asked for (mean-one, sigma given).
* Start model: W0 = s * I(grid) * (1 + a u), u ~ U(-1, 1) per voxel (a = 0.2 is
  the "truth + 20% multiplicative noise" of the workloads).
* Mask: a central beamstop disk plus one horizontal and one vertical gap stripe
  through the centre, sized so that the requested fraction of all detector
  pixels is masked.

Seeds (fixed per purpose): atoms 1001, orientations 1002, Poisson 1003,
start-noise 1004, fluence 1005.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_ATOMS = 1001
SEED_ORIENT = 1002
SEED_POISSON = 1003
SEED_START = 1004
SEED_FLUENCE = 1005


# ----------------------------------------------------------------------------
# Detector geometry
# ----------------------------------------------------------------------------

def detector_q(D: int, N: int) -> np.ndarray:
    """All D*D pixel positions q (float64, shape [D*D, 3], row-major pixels)."""
    u = np.arange(D, dtype=np.float64) - D / 2 + 0.5
    U, V = np.meshgrid(u, u)  # U varies along columns, V along rows
    L = float(D)
    s = np.stack([U, V, np.full_like(U, L)], axis=-1)
    s /= np.linalg.norm(s, axis=-1, keepdims=True)
    s_edge = np.array([D / 2, 0.0, L])
    s_edge /= np.linalg.norm(s_edge)
    q_max = N / 2 - 1
    r_e = q_max / np.linalg.norm(s_edge - np.array([0.0, 0.0, 1.0]))
    q = r_e * (s - np.array([0.0, 0.0, 1.0]))
    return q.reshape(D * D, 3)


def detector_mask(D: int, masked_fraction: float) -> np.ndarray:
    """Boolean [D*D] array, True where a pixel is masked (beamstop or gaps)."""
    if masked_fraction <= 0:
        return np.zeros(D * D, dtype=bool)
    rows = np.arange(D)[:, None] * np.ones((1, D))
    cols = np.ones((D, 1)) * np.arange(D)[None, :]
    c = D / 2 - 0.5
    gap_w = max(1, int(round(D / 64)))  # stripes 2*gap_w pixels wide
    lo, hi = D // 2 - gap_w, D // 2 + gap_w - 1
    stripes = ((rows >= lo) & (rows <= hi)) | ((cols >= lo) & (cols <= hi))
    r = np.hypot(rows - c, cols - c)
    target = masked_fraction * D * D
    # bisection on the beamstop radius so the union covers the target count
    a, b = 0.0, float(D)
    for _ in range(60):
        mid = 0.5 * (a + b)
        cnt = np.count_nonzero(stripes | (r <= mid))
        if cnt < target:
            a = mid
        else:
            b = mid
    return (stripes | (r <= b)).reshape(D * D)


@dataclasses.dataclass
class Detector:
    D: int
    N: int
    q: np.ndarray          # [M_pix, 3] float64, used pixels only
    pixel_index: np.ndarray  # [M_pix] int64 index into the D*D detector
    masked_fraction: float


def make_detector(D: int, N: int, masked_fraction: float = 0.0) -> Detector:
    q_all = detector_q(D, N)
    q_max = N / 2 - 1
    inside = np.linalg.norm(q_all, axis=1) <= q_max
    used = inside & ~detector_mask(D, masked_fraction)
    idx = np.nonzero(used)[0]
    return Detector(D=D, N=N, q=q_all[idx].copy(), pixel_index=idx,
                    masked_fraction=masked_fraction)


# ----------------------------------------------------------------------------
# Particle and its closed-form intensity
# ----------------------------------------------------------------------------

def make_atoms(n_atoms: int, radius: float, seed: int = SEED_ATOMS) -> np.ndarray:
    """n_atoms positions uniform in a ball (voxel units, centred at 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((n_atoms, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.random(n_atoms) ** (1.0 / 3.0)
    return d * r[:, None]


def intensity(points, atoms: np.ndarray, N: int, sigma: float = 1.0,
              device: str = "cpu", chunk: int = 1 << 22) -> np.ndarray:
    """I(p) at frequency points p ([..., 3], voxel-frequency units), float64."""
    import torch

    pts = np.asarray(points, dtype=np.float64)
    shape = pts.shape[:-1]
    pts = pts.reshape(-1, 3)
    out = np.empty(pts.shape[0], dtype=np.float64)
    at = torch.as_tensor(atoms, dtype=torch.float64, device=device)
    two_pi_n = 2.0 * math.pi / N
    env_c = -4.0 * math.pi ** 2 * sigma ** 2 / N ** 2
    for s in range(0, pts.shape[0], chunk):
        p = torch.as_tensor(pts[s:s + chunk], dtype=torch.float64, device=device)
        ph = two_pi_n * (p @ at.T)
        re = torch.cos(ph).sum(1)
        im = torch.sin(ph).sum(1)
        env = torch.exp(env_c * (p * p).sum(1))
        out[s:s + chunk] = (env * (re * re + im * im)).cpu().numpy()
    return out.reshape(shape)


def grid_points(N: int) -> np.ndarray:
    """Frequency coordinates of the N^3 grid, [N, N, N, 3], index [x][y][z]."""
    c = np.arange(N, dtype=np.float64) - N / 2
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([X, Y, Z], axis=-1)


# ----------------------------------------------------------------------------
# Orientations
# ----------------------------------------------------------------------------

def random_rotations(n: int, seed: int = SEED_ORIENT) -> np.ndarray:
    """n Haar-uniform rotation matrices [n, 3, 3] (QR of Gaussian matrices)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.standard_normal((n, 3, 3))
    Q, Rr = np.linalg.qr(A)
    d = np.sign(np.diagonal(Rr, axis1=1, axis2=2))
    d[d == 0] = 1.0
    Q = Q * d[:, None, :]
    det = np.linalg.det(Q)
    Q[det < 0, :, 0] *= -1.0
    return Q


def rotated_pixels(q: np.ndarray, rot: np.ndarray) -> np.ndarray:
    """Points R_k q_i for all k, i: [n_rot, M_pix, 3]."""
    return np.einsum("kab,ib->kia", rot, q)


# ----------------------------------------------------------------------------
# Whole data sets
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Dataset:
    N: int
    detector: Detector
    atoms: np.ndarray
    rot_true: np.ndarray     # [M_data, 3, 3]
    fluence: np.ndarray      # [M_data]
    scale: float             # s: model = s * I
    K: np.ndarray            # [M_data, M_pix] int32
    model_true: np.ndarray   # [N, N, N] float64, s * I(grid)
    model_start: np.ndarray  # [N, N, N] float64

    @property
    def q(self) -> np.ndarray:
        return self.detector.q


def make_dataset(N: int, D: int, n_data: int, mean_photons: float, *,
                 n_atoms: int = 50, sigma: float = 1.0, radius: float | None = None,
                 masked_fraction: float = 0.0, start_noise: float = 0.2,
                 fluence_sigma: float = 0.0, device: str = "cpu",
                 rot_true: np.ndarray | None = None,
                 noiseless: bool = False) -> Dataset:
    """Build one seeded synthetic data set (see the module docstring)."""
    if radius is None:
        radius = 8.0 if N <= 32 else N / 4
    det = make_detector(D, N, masked_fraction)
    atoms = make_atoms(n_atoms, radius)
    if rot_true is None:
        rot_true = random_rotations(n_data)
    n_data = rot_true.shape[0]
    if fluence_sigma > 0:
        rng = np.random.Generator(np.random.PCG64(SEED_FLUENCE))
        phi = np.exp(fluence_sigma * rng.standard_normal(n_data) - 0.5 * fluence_sigma ** 2)
    else:
        phi = np.ones(n_data)
    lam = np.empty((n_data, det.q.shape[0]), dtype=np.float64)
    step = max(1, (1 << 22) // max(1, det.q.shape[0]))
    for s in range(0, n_data, step):
        lam[s:s + step] = intensity(rotated_pixels(det.q, rot_true[s:s + step]),
                                    atoms, N, sigma, device=device)
    scale = mean_photons / lam.mean() if lam.size else 1.0
    lam *= scale * phi[:, None]
    if noiseless:
        K = lam.astype(np.float64)
    else:
        rng = np.random.Generator(np.random.PCG64(SEED_POISSON))
        K = rng.poisson(lam).astype(np.int32)
    model_true = scale * intensity(grid_points(N), atoms, N, sigma, device=device)
    rng = np.random.Generator(np.random.PCG64(SEED_START))
    u = rng.uniform(-1.0, 1.0, size=model_true.shape)
    model_start = model_true * (1.0 + start_noise * u)
    return Dataset(N=N, detector=det, atoms=atoms, rot_true=rot_true, fluence=phi,
                   scale=scale, K=K, model_true=model_true, model_start=model_start)


# The five workloads: grid side N, detector side D, quaternion subdivision n,
# frame count, mean photons per pixel, masked fraction, fluence spread.
WORKLOADS = {
    "emc32": dict(N=32, D=32, n_quat=4, n_data=1000, mean_photons=0.5,
                  masked_fraction=0.0, fluence_sigma=0.0),
    "emc64": dict(N=64, D=64, n_quat=10, n_data=20000, mean_photons=1.0,
                  masked_fraction=0.10, fluence_sigma=0.0),
    "emc128": dict(N=128, D=128, n_quat=16, n_data=100000, mean_photons=0.3,
                   masked_fraction=0.0, fluence_sigma=0.0),
    "emc160": dict(N=160, D=160, n_quat=20, n_data=200000, mean_photons=0.2,
                   masked_fraction=0.0, fluence_sigma=0.3),
}
