"""The overhead model (Secs. 2.2-4.2) against every number the paper prints.

Inputs printed with 2 decimals (phi, phi_t, alpha_M) are known only to
+-0.005, so each check evaluates the model over that interval and asks the
printed value to lie inside the resulting range widened by half a unit of
its own last printed digit.
"""
import itertools
import json
import os

import pytest

from paper_1703_08015_gb300 import perfmodel as pm

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_overheads.json")))


def _within(fn, printed, decimals, **ranges):
    keys = list(ranges)
    vals = [fn(**dict(zip(keys, corner))) for corner in itertools.product(*(ranges[k] for k in keys))]
    half = 0.5 * 10 ** (-decimals) + 1e-12
    assert min(vals) - half <= printed <= max(vals) + half, (printed, min(vals), max(vals))


def _r(v, h=0.005):
    return (v - h, v + h)


def test_B_node():
    g = GOLD["B_node"]
    assert pm.B_node(9, 8) == g["D2Q9_f64"]
    assert pm.B_node(19, 8) == g["D3Q19_f64"]
    assert pm.M_node(19, 8) * 2 == pm.B_node(19, 8)


def test_eq25_eq26_T2C_constants():
    c0, c1 = pm.T2C_memory_constants(9, 8, 16, 2)
    assert round(c0, 3) == GOLD["eq25_T2C_D2Q9_16"]["c0"]
    assert round(c1, 5) == GOLD["eq25_T2C_D2Q9_16"]["c1"]
    c0, c1 = pm.T2C_memory_constants(19, 8, 4, 3)
    assert round(c0, 3) == GOLD["eq26_T2C_D3Q19_4"]["c0"]
    assert round(c1, 5) == GOLD["eq26_T2C_D3Q19_4"]["c1"]
    # Eq. 24 written out equals the constants form of Eq. 26
    for phi_t, r in [(0.5, 3.0), (0.9, 8.6)]:
        assert pm.dM_T2C(19, 8, 4, 3, phi_t, r) == pytest.approx((c0 + c1 * r) / phi_t - 1)


def test_eq31_eq32_TGB_constants():
    c0, c1 = pm.TGB_memory_constants(pm.D2Q9, 8, 16)
    assert round(c0, 3) == GOLD["eq31_TGB_D2Q9_16"]["c0"] and round(c1, 3) == GOLD["eq31_TGB_D2Q9_16"]["c1"]
    c0, c1 = pm.TGB_memory_constants(pm.D3Q19, 8, 4)
    assert round(c0, 3) == GOLD["eq32_TGB_D3Q19_4"]["c0"] and round(c1, 3) == GOLD["eq32_TGB_D3Q19_4"]["c1"]


def test_C_gb_C_gbi():
    for name, lat in (("D2Q9", pm.D2Q9), ("D3Q19", pm.D3Q19), ("D3Q27", pm.D3Q27)):
        num, den = GOLD["C_gb"][name]
        assert pm.C_gb(lat) == pytest.approx(num / den)
        assert pm.C_gbi(lat) == GOLD["C_gbi"][name]
        assert lat.q == lat.q_s + lat.q_d + lat.q_t + 1


def test_bandwidth_constants():
    g = GOLD["dB_T2C_times_phi_t"]
    assert round(pm.dB_T2C(9, 8, 16, 2, 1.0), 4) == g["D2Q9_16"]
    assert round(pm.dB_T2C(19, 8, 4, 3, 1.0), 4) == g["D3Q19_4"]
    g = GOLD["dB_TGB_times_phi_t"]
    assert round(pm.dB_TGB(pm.D2Q9, 8, 16, 1.0), 4) == g["D2Q9_16"]
    assert round(pm.dB_TGB(pm.D3Q19, 8, 4, 1.0), 4) == g["D3Q19_4"]


@pytest.mark.parametrize("row", GOLD["table1"]["rows"], ids=[r[0] for r in GOLD["table1"]["rows"]])
def test_table1(row):
    case, lat, phi, phi_t, aM, dM_TGB, dM_T2C, dM_FIA, dM_CM, dB_TGB, dB_T2C, dB_FIA, dB_CM = row
    L = pm.D3Q19 if lat == "D3Q19" else pm.D2Q9
    a = 4 if lat == "D3Q19" else 16
    q, d = L.q, L.d
    _within(lambda phi_t, aM: pm.dM_TGB(L, 8, a, phi_t, aM), dM_TGB, 2, phi_t=_r(phi_t), aM=_r(aM))
    # N_tiles/N_ftiles lies in (2.3, 8.6) for the paper's geometries (Sec. 3.1.1.1)
    _within(lambda phi_t, r: pm.dM_T2C(q, 8, a, d, phi_t, r), dM_T2C, 2, phi_t=_r(phi_t), r=(2.3, 8.6))
    _within(lambda phi: pm.dM_FIA(q, 8, phi), dM_FIA, 2, phi=_r(phi))
    assert round(pm.dM_CM(q, 8), 2) == dM_CM
    _within(lambda phi_t: pm.dB_TGB(L, 8, a, phi_t), dB_TGB, 3, phi_t=_r(phi_t))
    _within(lambda phi_t: pm.dB_T2C(q, 8, a, d, phi_t), dB_T2C, 3, phi_t=_r(phi_t))
    _within(lambda phi: pm.dB_FIA(q, 8, phi), dB_FIA, 3, phi=_r(phi))
    assert round(pm.dB_CM(q, 8), 2) == dB_CM


@pytest.mark.parametrize("row", GOLD["table5_3d"]["rows"], ids=[r[0] for r in GOLD["table5_3d"]["rows"]])
def test_table5_T2C_burst(row):
    case, phi_t, dB, dB_bt = row
    _within(lambda phi_t: pm.dB_T2C(19, 8, 4, 3, phi_t), dB, 3, phi_t=_r(phi_t))
    _within(lambda phi_t: pm.dB_T2C_bt(19, 8, 4, 3, phi_t), dB_bt, 3, phi_t=_r(phi_t))


def test_coarctation_transactions():
    g = GOLD["coarctation_transactions"]
    # 659105 * 304 / 32 = 6261497.5, printed rounded up
    assert round(g["n_fnodes"] * pm.B_node(19, 8) / 32 + 0.5) == g["min_32B_transactions"]
    assert round(g["observed"] / g["min_32B_transactions"] - 1, 3) == g["overhead"]


def test_headline_bandwidth_utilisation():
    g = GOLD["table2_headline"]
    # BU = 0.719 at 682 MLUPS fixes the GTX Titan peak the paper used: ~288.4 GB/s
    b_gpu = g["mlups"] * 1e6 * pm.B_node(19, 8) / g["BU"] / 1e9
    assert 288.0 < b_gpu < 288.6
    assert round(pm.bandwidth_utilisation(g["mlups"], 19, 8, 288.4), 3) == g["BU"]
