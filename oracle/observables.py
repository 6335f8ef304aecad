"""Observables of the paper's evaluation (Sec. 4.2): radial distribution function pair counts and
the virial pressure -- TEST INFRASTRUCTURE ONLY (see the package docstring).

``rdf_counts``: number of unordered pairs {i, j} whose minimum-image distance r falls in bin b,
edges[b] <= r < edges[b + 1], edges[b] = b * (r_max / nbins) in IEEE double; r is computed as
sqrt((dx*dx + dy*dy) + dz*dz) with d = x_j - x_i folded by d - L * rint(d / L) per axis.  The
histogram is the raw material of g(r) (Sec. 4.2.2, the RDF of the aluminium runs):
g(r_b) = counts[b] / (N / 2 * rho * 4/3 pi (edges[b+1]^3 - edges[b]^3)).

``pressure``: P = (2 E_kin + W) / (3 V) with W = sum over interactions of sum_a r_a . F_a (the
virial), the pressure of Sec. 4.2.2.
"""
from __future__ import annotations

import numpy as np


def bin_edges(nbins: int, r_max: float) -> np.ndarray:
    """edges[b] = b * (r_max / nbins), each a single IEEE double product."""
    dr = float(r_max) / int(nbins)
    return np.arange(nbins + 1, dtype=np.float64) * dr


def rdf_counts(x, L: float, nbins: int, r_max: float, chunk: int = 256) -> np.ndarray:
    """Pair counts per distance bin, brute force over all pairs i < j (O(N^2), chunked rows)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    edges = bin_edges(nbins, r_max)
    counts = np.zeros(nbins, dtype=np.int64)
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        d = x[None, :, :] - x[i0:i1, None, :]          # d = x_j - x_i
        d = d - L * np.rint(d / L)
        r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
        r = np.sqrt(r2)
        jj = np.arange(n)[None, :]
        ii = np.arange(i0, i1)[:, None]
        rr = r[jj > ii]                                  # each unordered pair once
        rr = rr[rr < edges[-1]]
        b = np.searchsorted(edges, rr, side="right") - 1
        counts += np.bincount(b, minlength=nbins)[:nbins]
    return counts


def rdf_normalise(counts: np.ndarray, n: int, L: float, r_max: float) -> np.ndarray:
    """g(r) per bin from the pair counts: ideal-gas pair count of each spherical shell in the
    denominator."""
    edges = bin_edges(len(counts), r_max)
    shell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    rho = n / L ** 3
    return counts / (0.5 * n * rho * shell)


def pressure(e_kin: float, virial: float, L: float) -> float:
    """P = (2 E_kin + W) / (3 V), V = L^3 (k_B = 1)."""
    return (2.0 * e_kin + virial) / (3.0 * L ** 3)
