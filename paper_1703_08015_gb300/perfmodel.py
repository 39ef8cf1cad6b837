"""Memory and bandwidth overhead model of tiles (Secs. 2.2-3.1 and 4.2).

Host-side analysis only: the benchmark uses it to set the measured traffic of
the step kernel beside the paper's predictions.  Every function follows one
numbered equation of Tomczak & Szafran (arXiv:1703.08015); symbols keep the
paper's names:

  q     PDFs per node            s_d   bytes per PDF value
  s_t   bytes per node type      s_ti  bytes per tileMap index
  a     nodes per tile edge      d     space dimension, n_tn = a^d
  phi   porosity (Eq. 11)        phi_t average tile porosity (Eq. 17)
  alpha_M, alpha_B  fraction of ghost buffers allocated / transferred
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class LatticeCounts:
    """q and the ghost-buffer link classes of Sec. 3.1.1.2."""
    q: int
    d: int
    q_s: int  # links toward faces (3D) / edges (2D): one ghost-buffer set
    q_d: int  # links toward edges (3D) / corners (2D): two sets
    q_t: int  # links toward corners (3D): three sets


D2Q9 = LatticeCounts(q=9, d=2, q_s=4, q_d=4, q_t=0)
D3Q19 = LatticeCounts(q=19, d=3, q_s=6, q_d=12, q_t=0)
D3Q27 = LatticeCounts(q=27, d=3, q_s=6, q_d=12, q_t=8)


def M_node(q, s_d):
    """Eq. 9: minimum bytes stored per node."""
    return q * s_d


def B_node(q, s_d):
    """Eq. 10: minimum bytes moved per node and time step."""
    return 2 * q * s_d


def porosity(n_fnodes, n_nodes):
    """Eq. 11."""
    return n_fnodes / n_nodes


def solidity(n_snodes, n_nodes):
    """Eq. 12."""
    return n_snodes / n_nodes


def dM_CM(q, s_d, s_idx=4):
    """Eq. 13: connectivity-matrix memory overhead."""
    return (q - 1) * s_idx / M_node(q, s_d) + 1


def dB_CM(q, s_d, s_idx=4):
    """Eq. 14: connectivity-matrix bandwidth overhead."""
    return (q - 1) * s_idx / B_node(q, s_d)


def dM_FIA(q, s_d, phi, s_idx=4):
    """Eq. 15: fluid-index-array memory overhead."""
    return s_idx / (phi * M_node(q, s_d)) + 1


def dB_FIA(q, s_d, phi, s_idx=4):
    """Eq. 16: fluid-index-array bandwidth overhead."""
    return s_idx / (phi * B_node(q, s_d)) + 1


def M_tile(n_tn, phi_t, q, s_d):
    """Eq. 18."""
    return n_tn * phi_t * M_node(q, s_d)


def B_tile(n_tn, phi_t, q, s_d):
    """Eq. 19."""
    return n_tn * phi_t * B_node(q, s_d)


def dM_T2C(q, s_d, a, d, phi_t, tiles_ratio=1.0, s_t=2, s_ti=4):
    """Eq. 24: memory overhead of tiles with two copies.

    Sum of Eq. 20 (solid nodes in tiles), Eq. 21 (node types), Eq. 22 (second
    copy) and Eq. 23 (tileMap), with tiles_ratio = N_tiles / N_ftiles."""
    n_tn = a ** d
    M = M_node(q, s_d)
    return (1.0 / phi_t) * (2 - phi_t + (s_t + tiles_ratio * s_ti / n_tn) / M)


def T2C_memory_constants(q, s_d, a, d, s_t=2, s_ti=4):
    """Eqs. 25/26: Delta^M_T2C = (c0 + c1 * N_tiles/N_ftiles) / phi_t - 1."""
    M = M_node(q, s_d)
    return 2 + s_t / M, s_ti / (a ** d * M)


def C_gb(lat: LatticeCounts):
    """Ghost buffers per PDF (Eq. 28's constant)."""
    return (lat.q_s + 2 * lat.q_d + 3 * lat.q_t) / lat.q


def C_gbi(lat: LatticeCounts):
    """Ghost-buffer indices per tile (Eq. 29's constant)."""
    return 2 * lat.q_s + 5 * lat.q_d + 10 * lat.q_t


def dM_TGB(lat: LatticeCounts, s_d, a, phi_t, alpha_M, s_t=2, s_gbi=4):
    """Eq. 30: memory overhead of tiles with ghost buffers."""
    n_tn = a ** lat.d
    M = M_node(lat.q, s_d)
    return (1.0 / phi_t) * (1 - phi_t + (s_t + C_gbi(lat) * s_gbi / n_tn) / M
                            + 2 * alpha_M * C_gb(lat) / a)


def TGB_memory_constants(lat: LatticeCounts, s_d, a, s_t=2, s_gbi=4):
    """Eqs. 31/32: Delta^M_TGB = (c0 + c1 * alpha_M) / phi_t - 1."""
    M = M_node(lat.q, s_d)
    return 1 + (s_t + C_gbi(lat) * s_gbi / a ** lat.d) / M, 2 * C_gb(lat) / a


def dB_nt(q, s_d, a, d, phi_t, s_t=2):
    """Eq. 33: node types of a tile and its one-node halo."""
    return (a + 2) ** d * s_t / B_tile(a ** d, phi_t, q, s_d)


def dB_T2C(q, s_d, a, d, phi_t, s_t=2, s_ti=4):
    """Eq. 35 (= Eq. 33 + Eq. 34): bandwidth overhead of two copies."""
    return ((a + 2) ** d * s_t + (q - 1) * s_ti) / B_tile(a ** d, phi_t, q, s_d)


def dB_TGB(lat: LatticeCounts, s_d, a, phi_t, s_t=2, s_gbi=4):
    """Eq. 37 (= Eq. 33 + Eq. 36): bandwidth overhead of ghost buffers."""
    return (((a + 2) ** lat.d * s_t + C_gbi(lat) * s_gbi)
            / B_tile(a ** lat.d, phi_t, lat.q, s_d))


def dB_ftd(phi_t):
    """Eq. 38: whole-tile transfers when tiles hold solid nodes."""
    return 1.0 / phi_t - 1


def dB_T2C_bt(q, s_d, a, d, phi_t, s_t=2, s_ti=4):
    """Eq. 41: pessimistic burst-transaction overhead of two copies."""
    return dB_T2C(q, s_d, a, d, phi_t, s_t, s_ti) + dB_ftd(phi_t)


def dB_TGB_bt(lat: LatticeCounts, s_d, a, phi_t, alpha_B, s_b=32, s_t=2, s_gbi=4):
    """Eq. 42 with Eqs. 39/40 (q_c = q_d in 2D, q_t in 3D)."""
    n_tn = a ** lat.d
    q_c = lat.q_d if lat.d == 2 else lat.q_t
    B_gbnc = (C_gbi(lat) - q_c) * (n_tn / a) * s_d
    B_gbc = q_c * s_b
    return (dB_TGB(lat, s_d, a, phi_t, s_t, s_gbi) + dB_ftd(phi_t)
            + (B_gbnc + B_gbc) / B_tile(n_tn, phi_t, lat.q, s_d) * alpha_B)


def bandwidth_utilisation(mlups, q, s_d, B_gpu_GBs):
    """Eq. 43: BU = P * B_node / B_GPU (P in MLUPS over non-solid nodes)."""
    return mlups * 1e6 * B_node(q, s_d) / (B_gpu_GBs * 1e9)


def predictions(q, s_d, a, d, phi, phi_t, tiles_ratio):
    """Overheads the model predicts for one tiled geometry (T2C)."""
    return {
        "dM_T2C": dM_T2C(q, s_d, a, d, phi_t, tiles_ratio),
        "dB_T2C": dB_T2C(q, s_d, a, d, phi_t),
        "dB_T2C_bt": dB_T2C_bt(q, s_d, a, d, phi_t),
        "dB_CM": dB_CM(q, s_d),
        "dB_FIA": dB_FIA(q, s_d, phi),
    }
