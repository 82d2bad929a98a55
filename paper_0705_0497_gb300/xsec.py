"""Cross-section data for the reactions of the paper's Table 1 (data only).

The paper's own cross-section set is semi-empirical and published elsewhere
(Sec. 2), so it is not available.  What the paper does give is used exactly:

* Eq. 1, associative detachment (20) on O2(a1Dg):
  sigma_ad(E) = 5.96e-16 cm^2 / sqrt(E[eV]), no threshold;
* the two-channel Landau-Zener form of ion-ion neutralization (17):
  sigma_n(E) = 4 pi R_x^2 (1 + 1/(R_x E)) in atomic units, i.e. in SI
  sigma_n = 4 pi R_x^2 (1 + E_c/E) with E_c = e^2 / (4 pi eps0 R_x);
* the charge-exchange rule for (9): sigma_cx = sigma_m / 2, sigma_m taken from
  (here: placeholder) empirical branches below 0.251 eV and above 8.5 eV and
  linearly interpolated in between;
* the thresholds of (12), 6.4 eV, and (13), 8.6 eV.

Every other curve below is a PLACEHOLDER of plausible magnitude, not the
paper's data: smooth analytic shapes with textbook O2 thresholds.  They make
the simulation exercise every reaction path; they do not reproduce the
paper's figures.

Each process is a dict(species, kind, target, threshold_eV, E, sigma) with
E in eV (strictly increasing) and sigma in m^2, the layout the C ABI takes.
"""
import math

import numpy as np

from .inputs import EPS0, QE

# species
E, OM, OP = 0, 1, 2
# process kinds (same numbering as the C ABI)
ELASTIC, EXCITE, IONIZE, ATTACH, DETACH, CX, NEUTRALIZE, RECOMBINE, EDETACH = range(9)
KIND_NAMES = ("elastic", "excite", "ionize", "attach", "detach", "cx", "neutralize", "recombine", "edetach")
# targets
T_O2, T_O2_META, T_ION, T_ELECTRON = 0, 1, 2, 3
# electron affinity of O [eV]: the threshold of (22) e + O- -> O + 2e
O_AFFINITY_EV = 1.461

# Rate-table grid used by both implementations: 32 points per octave on
# [2^-10, 2^12] eV.  Curves given exactly at these energies interpolate without
# error on that grid.
GRID = np.array([math.ldexp(1.0 + (i % 32) / 32.0, i // 32 - 10) for i in range(22 * 32 + 1)])

SIGMA_AD_CM2 = 5.96e-16          # Eq. 1 prefactor [cm^2 eV^1/2]
CX_LOW_EV, CX_HIGH_EV = 0.251, 8.5


def _energies(thr=0.0, lo=1e-3, hi=4096.0, n=240):
    """A log-spaced energy axis; for threshold processes it starts at thr."""
    if thr > 0:
        e = np.geomspace(thr, hi, n)
        e[0] = thr
    else:
        e = np.geomspace(lo, hi, n)
    return e


def _bump(E, thr, peak, smax):
    """Resonance shape y exp(1-y), y = (E-thr)/(peak-thr): 0 at thr, smax at peak."""
    y = np.clip((E - thr) / (peak - thr), 0.0, None)
    s = smax * y * np.exp(1.0 - y)
    return np.where(s < smax * 1e-30, 0.0, s)


def _rise(E, thr, peak, smax):
    """Broad shape 2y/(1+y^2): 0 at thr, smax at peak, ~1/E far above."""
    y = np.clip((E - thr) / (peak - thr), 0.0, None)
    return smax * 2.0 * y / (1.0 + y * y)


def sigma_ad(E_eV):
    """Eq. 1: associative detachment O- + O2(a1Dg) -> O3 + e  [m^2]."""
    return SIGMA_AD_CM2 * 1e-4 / np.sqrt(E_eV)


def landau_zener_Ec(R_x_m):
    """E_c = e^2 / (4 pi eps0 R_x) in eV."""
    return QE / (4.0 * math.pi * EPS0 * R_x_m)


def sigma_n(E_eV, R_x_m=1.0e-9):
    """Two-channel Landau-Zener ion-ion neutralization cross section [m^2]."""
    return 4.0 * math.pi * R_x_m ** 2 * (1.0 + landau_zener_Ec(R_x_m) / E_eV)


def sigma_m_o2plus(E_eV, s_low=1.0e-18, s_high=6.0e-19):
    """Momentum-transfer cross section of O2+ on O2 used for the cx rule:
    placeholder empirical branches below 0.251 eV (~E^-1/2) and above 8.5 eV
    (~E^-0.1), linear in E in between."""
    E_eV = np.asarray(E_eV, dtype=np.float64)
    lo = s_low * (E_eV / CX_LOW_EV) ** -0.5
    hi = s_high * (E_eV / CX_HIGH_EV) ** -0.1
    mid = s_low + (s_high - s_low) * (E_eV - CX_LOW_EV) / (CX_HIGH_EV - CX_LOW_EV)
    return np.where(E_eV <= CX_LOW_EV, lo, np.where(E_eV >= CX_HIGH_EV, hi, mid))


def sigma_cx(E_eV):
    """(9) charge exchange: sigma_cx = sigma_m / 2."""
    return 0.5 * sigma_m_o2plus(E_eV)


def _proc(species, kind, target, thr, E_ax, sig, name):
    return dict(species=species, kind=kind, target=target, threshold_eV=float(thr),
                E=np.ascontiguousarray(E_ax, dtype=np.float64),
                sigma=np.ascontiguousarray(sig, dtype=np.float64), name=name)


def electron_processes():
    """e + O2 processes (7), (10)-(15), (18), (21) — placeholder shapes."""
    out = []
    Ea = _energies()
    # (7) elastic momentum transfer
    x = Ea / 12.0
    el = 1.0e-19 * (0.4 + 0.6 * x / (1.0 + x * x)) / (1.0 + Ea / 300.0)
    out.append(_proc(E, ELASTIC, T_O2, 0.0, Ea, el, "(7) e+O2 elastic"))
    # (10) vibrational nu = 1..4
    for v, (thr, smax) in enumerate(((0.193, 1.5e-21), (0.383, 8.0e-22), (0.570, 5.0e-22), (0.753, 3.0e-22)), 1):
        Ex = _energies(thr)
        out.append(_proc(E, EXCITE, T_O2, thr, Ex, _bump(Ex, thr, thr + 1.0, smax), f"(10) vib v={v}"))
    # (11) Rydberg
    Ex = _energies(8.4)
    out.append(_proc(E, EXCITE, T_O2, 8.4, Ex, _rise(Ex, 8.4, 25.0, 2.0e-21), "(11) Rydberg"))
    # (12) dissociation O(3P)+O(3P), 6.4 eV (paper's threshold)
    Ex = _energies(6.4)
    out.append(_proc(E, EXCITE, T_O2, 6.4, Ex, _rise(Ex, 6.4, 14.0, 6.0e-21), "(12) diss 3P+3P"))
    # (13) dissociation O(3P)+O(1D), 8.6 eV (paper's threshold)
    Ex = _energies(8.6)
    out.append(_proc(E, EXCITE, T_O2, 8.6, Ex, _rise(Ex, 8.6, 20.0, 1.2e-20), "(13) diss 3P+1D"))
    # (14) a1Dg, (15) b1Sg
    Ex = _energies(0.977)
    out.append(_proc(E, EXCITE, T_O2, 0.977, Ex, _rise(Ex, 0.977, 6.0, 1.0e-22), "(14) a1Dg"))
    Ex = _energies(1.627)
    out.append(_proc(E, EXCITE, T_O2, 1.627, Ex, _rise(Ex, 1.627, 6.5, 4.0e-23), "(15) b1Sg"))
    # (18) dissociative attachment, resonance near 6.5 eV
    Ex = _energies(4.2)
    out.append(_proc(E, ATTACH, T_O2, 4.2, Ex, 1.4e-22 * np.exp(-((Ex - 6.5) / 1.3) ** 2), "(18) attachment"))
    # (21) ionization, 12.06 eV
    Ex = _energies(12.06)
    out.append(_proc(E, IONIZE, T_O2, 12.06, Ex, _rise(Ex, 12.06, 100.0, 2.7e-20), "(21) ionization"))
    return out


def om_processes(include_ad=True, direct_thr=1.465):
    """O- processes: (8) elastic, (19) direct detachment, (20) associative
    detachment on O2(a) with Eq. 1 exactly (given on the table grid)."""
    out = []
    Ea = _energies()
    out.append(_proc(OM, ELASTIC, T_O2, 0.0, Ea, 3.0e-19 / np.sqrt(Ea), "(8) O-+O2 elastic"))
    Ex = _energies(direct_thr)
    out.append(_proc(OM, DETACH, T_O2, direct_thr, Ex, _rise(Ex, direct_thr, 30.0, 1.0e-19), "(19) direct detachment"))
    if include_ad:
        out.append(_proc(OM, DETACH, T_O2_META, 0.0, GRID, sigma_ad(GRID), "(20) associative detachment (Eq. 1)"))
    return out


def op_processes():
    """O2+ + O2 (9) charge exchange, sigma_cx = sigma_m / 2; the table holds
    the two junction energies 0.251 and 8.5 eV exactly."""
    Ea = np.union1d(_energies(), [CX_LOW_EV, CX_HIGH_EV])
    return [_proc(OP, CX, T_O2, 0.0, Ea, sigma_cx(Ea), "(9) charge exchange")]


def neutralization_process(R_x_m=1.0e-9):
    """(17) O- + O2+ -> O + O2, Landau-Zener, given on the table grid."""
    return _proc(OM, NEUTRALIZE, T_ION, 0.0, GRID, sigma_n(GRID, R_x_m), "(17) neutralization")


def sigma_r(E_eV):
    """(16) e + O2+ -> O + O dissociative recombination: placeholder
    sigma_r = 3.4e-19 m^2 (1 eV / E), i.e. a rate coefficient sigma_r g of
    2e-13 m^3/s at 1 eV that grows as E^-1/2 towards low energies.  The
    paper lists (16) in Table 1 without its cross section."""
    return 3.4e-19 / np.asarray(E_eV, dtype=np.float64)


def recombination_process():
    """(16) e + O2+ -> O + O, binary and cell-local like (17), on the grid."""
    return _proc(E, RECOMBINE, T_ION, 0.0, GRID, sigma_r(GRID), "(16) recombination")


def sigma_edetach(E_eV, thr=O_AFFINITY_EV):
    """(22) e + O- -> O + 2e electron-impact detachment: placeholder shape with
    the O electron affinity as threshold, rising to 5e-20 m^2 near 20 eV
    (the paper lists (22) in Table 1 without its cross section)."""
    return _rise(np.asarray(E_eV, dtype=np.float64), thr, 20.0, 5.0e-20)


def edetach_process(thr=O_AFFINITY_EV):
    """(22) e + O- -> O + 2e, binary and cell-local like (17) (species O-,
    partner the electrons), on ion steps before (16) and (17)."""
    Ex = _energies(thr)
    return _proc(OM, EDETACH, T_ELECTRON, thr, Ex, sigma_edetach(Ex, thr), "(22) electron detachment")


def oxygen_set(include_ad=True, R_x_m=1.0e-9, include_rec=False, include_edet=False):
    """The full 3-species set used by the workloads ((16), (22) on request)."""
    out = electron_processes() + om_processes(include_ad) + op_processes() + [neutralization_process(R_x_m)]
    if include_rec:
        out.append(recombination_process())
    if include_edet:
        out.append(edetach_process())
    return out


def constant_rate_process(species, kind, nu0, n_target, mu, target=T_O2, thr=0.0):
    """A test process with sigma ~ 1/g, i.e. a constant collision frequency nu0
    at target density n_target (reduced mass mu), on the table grid."""
    g = np.sqrt(2.0 * QE * GRID / mu)
    return _proc(species, kind, target, thr, GRID, nu0 / (n_target * g), "constant-rate test")
