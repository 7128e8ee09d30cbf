"""Host-side model assembly for the CUDA library: mass moments of the link
bodies (Eq. ATOM's precomputed integral int rho [p;1][p;1]^T dp) and rest
transforms, from a plain body description (``inputs.BodySpec``).

Link bodies run along the local -z axis from the joint (origin) to (0,0,-L).
"""
from __future__ import annotations

import numpy as np

from .inputs import CAPSULE, ROD, BodySpec


def rod_moment(m: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Thin uniform rod: int z^2 dm = m L^2/3, int z dm = -m L/2."""
    m = np.asarray(m, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    out = np.zeros(m.shape + (10,))
    out[..., 5] = m * L * L / 3.0
    out[..., 8] = -m * L / 2.0
    out[..., 9] = m
    return out


def capsule_moment(m: np.ndarray, L: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Solid capsule (cylinder of radius r over z in [-L, 0], hemispherical
    caps centred at 0 and -L), uniform density, total mass m. Second moments
    summed piecewise from the three solids' own integrals:
      cylinder:     int x^2 = m_c r^2/4, int z^2 = m_c L^2/3, int z = -m_c L/2
      hemisphere:   int x^2 = m_h r^2/5, int z'^2 = m_h r^2/5, int z' = +-3 r m_h/8
    (z' measured from the cap centre, shifted to 0 or -L)."""
    m = np.asarray(m, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    vc = np.pi * r * r * L
    vh = 2.0 / 3.0 * np.pi * r ** 3  # one hemisphere
    rho = m / (vc + 2 * vh)
    mc, mh = rho * vc, rho * vh
    sxx = mc * r * r / 4 + 2 * mh * r * r / 5
    # top cap: z in [0, r]; bottom cap: z = -L + z', z' in [-r, 0]
    szz = mc * L * L / 3 + mh * r * r / 5 + mh * (r * r / 5 + 2 * L * 3 * r / 8 + L * L)
    sz = -mc * L / 2 + mh * 3 * r / 8 + mh * (-L - 3 * r / 8)
    out = np.zeros(m.shape + (10,))
    out[..., 0] = sxx
    out[..., 3] = sxx
    out[..., 5] = szz
    out[..., 8] = sz
    out[..., 9] = m
    return out


def mass_moments(spec: BodySpec) -> np.ndarray:
    """(count, N, 10) mass moments of every link of every instance."""
    out = np.zeros((spec.count, spec.n_links, 10))
    for l in range(spec.n_links):
        if spec.shape[l] == ROD:
            out[:, l] = rod_moment(spec.mass[:, l], spec.length[:, l])
        elif spec.shape[l] == CAPSULE:
            out[:, l] = capsule_moment(spec.mass[:, l], spec.length[:, l], spec.radius[:, l])
        else:
            raise ValueError(f"unknown link shape {spec.shape[l]}")
    return out


def rest_transforms(spec: BodySpec) -> np.ndarray:
    """(count, N, 12) rest transforms [R_rest | attach] row-major."""
    out = np.zeros((spec.count, spec.n_links, 3, 4))
    out[:, :, :, :3] = spec.rest_rot[None]
    out[:, :, :, 3] = spec.attach
    return out.reshape(spec.count, spec.n_links, 12)
