"""CPU oracle of the 1D3V PIC-MCC oxygen-discharge step — TEST INFRASTRUCTURE.

ctypes binding of ``oracle/o2pic_oracle.cpp``.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import this
package.  It imports nothing from the CUDA package; both receive the same
seeded inputs from ``paper_0705_0497_gb300.inputs`` / ``.xsec`` (data only).
"""
import ctypes

import numpy as np

from . import build as _build

NSP = 3
SPECIES = ("e", "O-", "O2+")
MAXPROC = 16

_lib = None


class OracleConfig(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("L", "f", "U", "p", "T_gas", "C_meta", "dt", "weight", "area",
                 "m_e", "m_OM", "m_OP", "M_gas")] + [
        ("n_cells", ctypes.c_int32), ("ion_subcycle", ctypes.c_int32),
        ("seed", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class OracleProcess(ctypes.Structure):
    _fields_ = [("species", ctypes.c_int32), ("kind", ctypes.c_int32), ("target", ctypes.c_int32),
                ("n", ctypes.c_int32), ("threshold_eV", ctypes.c_double),
                ("E_eV", ctypes.POINTER(ctypes.c_double)), ("sigma_m2", ctypes.POINTER(ctypes.c_double))]


COUNTER_NAMES = ([f"events_{s}_{k}" for s in range(NSP) for k in range(MAXPROC)] +
                 [f"absorbed_{s}_{w}" for s in range(NSP) for w in range(2)] +
                 [f"born_{s}" for s in range(NSP)] +
                 ["neutralized", "pair_candidates", "particle_steps", "warn_emax", "warn_tries",
                  "warn_pair_gt1", "id_overflow", "recombined", "rec_candidates", "edetached", "edet_candidates", "coulomb_pairs", "warn_numax"])


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, u64, i32, u32, dbl = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, ctypes.c_double
        P = ctypes.POINTER
        L.oracle_create.restype = vp
        L.oracle_create.argtypes = [P(OracleConfig), i32]
        L.oracle_destroy.argtypes = [vp]
        L.oracle_set_processes.argtypes = [vp, P(OracleProcess), i32]
        L.oracle_load.argtypes = [vp, i32, vp, vp, vp, vp, vp, u64]
        L.oracle_set_next_id.argtypes = [vp, i32, u32]
        L.oracle_set_coulomb.argtypes = [vp, u32, dbl]
        L.oracle_set_majorant_cap.argtypes = [vp, vp]
        L.oracle_set_threads.argtypes = [vp, i32]
        L.oracle_set_threads.restype = i32
        L.oracle_step.argtypes = [vp, u64]
        L.oracle_set_step.argtypes = [vp, u64]
        L.oracle_get_step.restype = u64
        L.oracle_get_step.argtypes = [vp]
        L.oracle_count.restype = u64
        L.oracle_count.argtypes = [vp, i32]
        L.oracle_read.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        L.oracle_next_id.restype = u64
        L.oracle_next_id.argtypes = [vp, i32]
        L.oracle_read_field.argtypes = [vp, vp, vp, vp]
        L.oracle_read_charge.restype = u64
        L.oracle_read_charge.argtypes = [vp, vp, vp]
        L.oracle_reset_moments.argtypes = [vp]
        L.oracle_counters.argtypes = [vp, vp, i32]
        L.oracle_currents.argtypes = [vp, u64, u64, vp]
        L.oracle_table.argtypes = [vp, i32, vp, vp, vp, vp]
        L.oracle_neutral_table.argtypes = [vp, vp]
        L.oracle_update_particle.argtypes = [vp, i32, u64, vp, vp, u32, vp, i32, vp, vp]
        L.oracle_load_flight.argtypes = [vp, i32, vp, u64]
        L.oracle_read_flight.argtypes = [vp, i32, vp]
        L.oracle_flight_gap.restype = u32
        L.oracle_flight_gap.argtypes = [vp, i32, u32]
        L.oracle_philox.argtypes = [vp, vp, vp]
        L.oracle_ln_f32.restype = ctypes.c_float
        L.oracle_ln_f32.argtypes = [ctypes.c_float]
        L.oracle_sample.argtypes = [i32, i32, u32, u64, vp]
        L.oracle_solve_field.argtypes = [i32, dbl, dbl, dbl, dbl, vp, vp, vp]
        L.oracle_solve_field_thomas.argtypes = [i32, dbl, dbl, dbl, dbl, vp, vp, vp]
        L.oracle_deposit.argtypes = [i32, dbl, vp, u64, vp]
        L.oracle_lookup.restype = dbl
        L.oracle_lookup.argtypes = [vp, i32, i32, dbl]
        L.oracle_grid_energy.restype = dbl
        L.oracle_grid_energy.argtypes = [i32]
        L.oracle_ngrid.restype = i32
        L.oracle_ncounters.restype = i32
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cfg_struct(cfg):
    c = OracleConfig()
    for name, _ in OracleConfig._fields_:
        if name == "reserved":
            continue
        setattr(c, name, cfg[name])
    return c


class Oracle:
    """One discharge in the oracle.  precision = 32 (FP32 mirror) or 64."""

    def set_majorant_cap(self, caps):
        """Majorant caps in eV per species (None: the whole grid), taking
        effect at the next set_processes: nu_max = the largest total rate over
        the grid points up to the first one at or above the cap."""
        c = np.array([np.nan if v is None else float(v) for v in caps], np.float64)
        if lib().oracle_set_majorant_cap(self.h, _ptr(c)) != 0:
            raise ValueError("majorant cap must be positive")

    def set_coulomb(self, mask, ln_lambda=10.0):
        """Coulomb collisions (1)-(6): bit r-1 of mask enables reaction r."""
        lib().oracle_set_coulomb(self.h, int(mask), float(ln_lambda))

    def set_threads(self, n):
        """Host threads of the particle loop and the deposit (the results do
        not depend on it); returns the threads OpenMP offers."""
        return int(lib().oracle_set_threads(self.h, int(n)))

    def __init__(self, cfg, precision=32):
        self.cfg = dict(cfg)
        self.precision = precision
        self._c = _cfg_struct(cfg)
        self.h = lib().oracle_create(ctypes.byref(self._c), precision)
        if not self.h:
            raise ValueError("oracle_create rejected the configuration")
        self.Ng = int(cfg["n_cells"]) + 1
        self._keep = []

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_destroy(self.h)
            self.h = None

    def set_processes(self, procs):
        arr = (OracleProcess * len(procs))()
        keep = []
        for i, p in enumerate(procs):
            E = np.ascontiguousarray(p["E"], dtype=np.float64)
            s = np.ascontiguousarray(p["sigma"], dtype=np.float64)
            keep += [E, s]
            arr[i].species, arr[i].kind, arr[i].target = p["species"], p["kind"], p["target"]
            arr[i].n = len(E)
            arr[i].threshold_eV = p.get("threshold_eV", 0.0)
            arr[i].E_eV = E.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            arr[i].sigma_m2 = s.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        rc = lib().oracle_set_processes(self.h, arr, len(procs))
        if rc != 0:
            raise ValueError("oracle_set_processes rejected the tables")

    def load(self, species, x, vx, vy, vz, ids):
        a = [np.ascontiguousarray(v, dtype=np.float32) for v in (x, vx, vy, vz)]
        i = np.ascontiguousarray(ids, dtype=np.uint32)
        lib().oracle_load(self.h, species, *[_ptr(v) for v in a], _ptr(i), len(i))

    def load_flight(self, species, tc):
        """Set the free flights (step of the next collision candidate) of the
        loaded particles of a species, in array order."""
        t = np.ascontiguousarray(tc, dtype=np.uint32)
        if lib().oracle_load_flight(self.h, species, _ptr(t), len(t)) != 0:
            raise ValueError("flight count differs from the particle count")

    def flight(self, species):
        """Step of each particle's next collision candidate, in array order."""
        out = np.zeros(self.count(species), np.uint32)
        lib().oracle_read_flight(self.h, species, _ptr(out))
        return out

    def flight_gap(self, species, word):
        return int(lib().oracle_flight_gap(self.h, species, int(word) & 0xFFFFFFFF))

    def set_next_id(self, species, v):
        lib().oracle_set_next_id(self.h, species, v)

    def step(self, n=1):
        lib().oracle_step(self.h, n)

    def set_step(self, n):
        lib().oracle_set_step(self.h, n)

    @property
    def step_count(self):
        return lib().oracle_get_step(self.h)

    def count(self, species):
        return lib().oracle_count(self.h, species)

    def next_id(self, species):
        return lib().oracle_next_id(self.h, species)

    def particles(self, species):
        n = self.count(species)
        out = {k: np.zeros(n, np.float64) for k in ("x", "vx", "vy", "vz")}
        out["id"] = np.zeros(n, np.uint32)
        lib().oracle_read(self.h, species, _ptr(out["x"]), _ptr(out["vx"]), _ptr(out["vy"]),
                          _ptr(out["vz"]), _ptr(out["id"]))
        return out

    def field(self):
        phi, E, Eg = (np.zeros(self.Ng) for _ in range(3))
        lib().oracle_read_field(self.h, _ptr(phi), _ptr(E), _ptr(Eg))
        return phi, E, Eg

    def charge(self):
        Q = np.zeros((NSP, self.Ng), np.uint64)
        Qa = np.zeros((NSP, self.Ng), np.uint64)
        steps = lib().oracle_read_charge(self.h, _ptr(Q), _ptr(Qa))
        return Q, Qa, steps

    def reset_moments(self):
        lib().oracle_reset_moments(self.h)

    def counters(self):
        n = lib().oracle_ncounters()
        buf = np.zeros(n, np.uint64)
        lib().oracle_counters(self.h, _ptr(buf), n)
        return dict(zip(COUNTER_NAMES, (int(v) for v in buf)))

    def current_sums(self, step0, n):
        """Conduction-current sums [n][3] (int64) of steps step0 .. step0+n-1:
        sum over the particles pushed in the step of trunc(256 v_x^{n+1/2})."""
        out = np.zeros((n, 3), np.int64)
        rc = lib().oracle_currents(self.h, step0, n, _ptr(out))
        if rc != 0:
            raise ValueError("steps not recorded since the last load")
        return out

    def table(self, species):
        G = ngrid()
        cum = np.zeros(G * MAXPROC)
        nu = np.zeros(G * MAXPROC)
        numax = ctypes.c_double()
        pmax = ctypes.c_double()
        np_ = lib().oracle_table(self.h, species, _ptr(cum), _ptr(nu), ctypes.byref(numax), ctypes.byref(pmax))
        return (cum[:G * np_].reshape(G, np_), nu[:G * np_].reshape(G, np_), numax.value, pmax.value)

    def lookup(self, which, k, E):
        """The tabulated rate at energy E as the collision step reads it:
        which = species (cumulative column k), 3 = (17) table, 4 = (16),
        5 = (22)."""
        return lib().oracle_lookup(self.h, which, k, float(E))

    def neutral_table(self):
        K = np.zeros(ngrid())
        lib().oracle_neutral_table(self.h, _ptr(K))
        return K

    def update_particle(self, species, step, Ef, state, pid, tc=None):
        """One particle through push + absorb + MCC with gather field Ef; tc =
        the step of its next collision candidate (default: a free flight
        drawn at this step as for a freshly loaded particle, so a candidate
        with probability P_max).  Returns (alive, state, births, tc after)."""
        Ef = np.ascontiguousarray(Ef, dtype=np.float64)
        st = np.ascontiguousarray(state, dtype=np.float64).copy()
        births = np.zeros(5 * 4)
        nb = ctypes.c_int()
        t = ctypes.c_uint32(0 if tc is None else int(tc) & 0xFFFFFFFF)
        alive = lib().oracle_update_particle(self.h, species, step, _ptr(Ef), _ptr(st), pid, ctypes.byref(t),
                                             1 if tc is None else 0, _ptr(births), ctypes.byref(nb))
        return bool(alive), st, births[:5 * nb.value].reshape(nb.value, 5), int(t.value)


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def ln_f32(x):
    return lib().oracle_ln_f32(float(x))


def sample(kind, precision, seed, n):
    width = 3 if kind == 0 else 2
    out = np.zeros(n * width)
    lib().oracle_sample(kind, precision, seed, n, _ptr(out))
    return out.reshape(n, width)


def solve_field(n_cells, dx, weight, area, V0, Rnet, method="closed"):
    """Field of net node charges Rnet (2^16 per particle): the method's closed
    form ("closed") or the Thomas algorithm ("thomas")."""
    R = np.ascontiguousarray(Rnet, dtype=np.int64)
    phi = np.zeros(n_cells + 1)
    E = np.zeros(n_cells + 1)
    f = lib().oracle_solve_field if method == "closed" else lib().oracle_solve_field_thomas
    f(n_cells, dx, weight, area, V0, _ptr(R), _ptr(phi), _ptr(E))
    return phi, E


def deposit(n_cells, L, x):
    xx = np.ascontiguousarray(x, dtype=np.float32)
    Q = np.zeros(n_cells + 1, np.uint64)
    lib().oracle_deposit(n_cells, L, _ptr(xx), len(xx), _ptr(Q))
    return Q


def grid_energy(i):
    return lib().oracle_grid_energy(i)


def ngrid():
    return lib().oracle_ngrid()
