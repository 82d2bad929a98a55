"""ctypes binding of libo2pic (C ABI in include/o2pic.h) — argument marshalling only.

Every step of the particle loop runs in the library's CUDA kernels; this
module converts Python/numpy/torch arguments to pointers and back.  There is
no CPU fallback: if the library is missing the import of this module fails.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libo2pic.so")

NSP = 3
MAXPROC = 16
E, OM, OP = 0, 1, 2
HOST, DEVICE = 0, 1
KERNEL_KINDS = ("push_e", "push_om", "push_op", "pair_hist", "pair", "field", "compact", "deposit",
                "cand_e", "cand_om", "cand_op", "recomb", "filter_om", "filter_op", "coulomb")

OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CAPACITY", -3: "ID_OVERFLOW", -4: "NONFINITE", -5: "CUDA", -6: "TIMEOUT",
          -7: "STATE"}


class O2picError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({lib().o2pic_strerror(code).decode()})")


class Config(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("L", "f", "U", "p", "T_gas", "C_meta", "dt", "weight", "area", "m_e", "m_OM", "m_OP", "M_gas")] + [
        ("n_cells", ctypes.c_int32), ("ion_subcycle", ctypes.c_int32),
        ("seed", ctypes.c_uint32), ("compact_check", ctypes.c_uint32),
        ("capacity", ctypes.c_uint64 * NSP), ("device", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Process(ctypes.Structure):
    _fields_ = [("species", ctypes.c_int32), ("kind", ctypes.c_int32), ("target", ctypes.c_int32),
                ("n", ctypes.c_int32), ("threshold_eV", ctypes.c_double),
                ("E_eV", ctypes.POINTER(ctypes.c_double)), ("sigma_m2", ctypes.POINTER(ctypes.c_double))]


TUNE_MAX = 8


class TuneReport(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("particles_per_warp", ctypes.c_int32 * TUNE_MAX),
                ("ms", ctypes.c_double * TUNE_MAX), ("chosen", ctypes.c_int32), ("fused", ctypes.c_int32),
                ("other_mode_ms", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("events", (ctypes.c_uint64 * MAXPROC) * NSP), ("absorbed", (ctypes.c_uint64 * 2) * NSP),
                ("born", ctypes.c_uint64 * NSP), ("neutralized", ctypes.c_uint64),
                ("pair_candidates", ctypes.c_uint64), ("particle_steps", ctypes.c_uint64),
                ("warn_emax", ctypes.c_uint64), ("warn_tries", ctypes.c_uint64), ("warn_pair_gt1", ctypes.c_uint64),
                ("id_overflow", ctypes.c_uint64), ("step", ctypes.c_uint64), ("live", ctypes.c_uint64 * NSP),
                ("slots", ctypes.c_uint64 * NSP), ("next_id", ctypes.c_uint64 * NSP),
                ("error_flags", ctypes.c_uint64), ("particle_steps_species", ctypes.c_uint64 * NSP),
                ("recombined", ctypes.c_uint64), ("rec_candidates", ctypes.c_uint64),
                ("edetached", ctypes.c_uint64), ("edet_candidates", ctypes.c_uint64),
                ("coulomb_pairs", ctypes.c_uint64), ("warn_numax", ctypes.c_uint64)]

    def as_dict(self):
        d = {}
        for s in range(NSP):
            for k in range(MAXPROC):
                d[f"events_{s}_{k}"] = int(self.events[s][k])
            for w in range(2):
                d[f"absorbed_{s}_{w}"] = int(self.absorbed[s][w])
            d[f"born_{s}"] = int(self.born[s])
            d[f"live_{s}"] = int(self.live[s])
            d[f"slots_{s}"] = int(self.slots[s])
            d[f"next_id_{s}"] = int(self.next_id[s])
            d[f"particle_steps_{s}"] = int(self.particle_steps_species[s])
        for n in ("neutralized", "pair_candidates", "particle_steps", "warn_emax", "warn_tries", "warn_pair_gt1",
                  "id_overflow", "step", "error_flags", "recombined", "rec_candidates", "edetached",
                  "edet_candidates", "coulomb_pairs", "warn_numax"):
            d[n] = int(getattr(self, n))
        return d


_lib = None

# (name, restype, argtypes) for every function of include/o2pic.h
_vp, _u64, _i32, _u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
_P = ctypes.POINTER
SIGNATURES = [
    ("o2pic_config_init", _i32, [_P(Config)]),
    ("o2pic_create", _i32, [_P(Config), _P(_vp)]),
    ("o2pic_set_processes", _i32, [_vp, _P(Process), _i32]),
    ("o2pic_load_particles", _i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _u64, _i32, _vp]),
    ("o2pic_set_next_id", _i32, [_vp, _i32, _u32]),
    ("o2pic_load_flight", _i32, [_vp, _i32, _vp, _u64, _i32, _vp]),
    ("o2pic_set_coulomb", _i32, [_vp, _u32, ctypes.c_double]),
    ("o2pic_set_majorant_cap", _i32, [_vp, _vp]),
    ("o2pic_read_flight", _i32, [_vp, _i32, _vp, _u64, _P(_u64), _i32]),
    ("o2pic_step", _i32, [_vp, _u64, _vp]),
    ("o2pic_synchronize", _i32, [_vp]),
    ("o2pic_read_particles", _i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _u64, _P(_u64), _i32]),
    ("o2pic_read_field", _i32, [_vp, _vp, _vp]),
    ("o2pic_read_charge", _i32, [_vp, _vp, _vp, _P(_u64)]),
    ("o2pic_read_currents", _i32, [_vp, _u64, _u64, _vp]),
    ("o2pic_read_moments", _i32, [_vp, _vp, _P(_u64), _i32]),
    ("o2pic_get_stats", _i32, [_vp, _P(Stats)]),
    ("o2pic_set_step", _i32, [_vp, _u64]),
    ("o2pic_set_timing", _i32, [_vp, _i32]),
    ("o2pic_get_timing", _i32, [_vp, _vp, _vp, _vp, _i32]),
    ("o2pic_launch_count", _u64, [_vp]),
    ("o2pic_philox", _i32, [_vp, _vp, _vp, _u64, _vp]),
    ("o2pic_ln_f32", _i32, [_vp, _vp, _u64, _vp]),
    ("o2pic_compact_particles", _i32, [_vp, _vp, _vp, _vp, _vp, _u64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("o2pic_compact_particles_noalloc", _i32, [_vp, _vp, _vp, _vp, _vp, _u64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("o2pic_check_bounded_wait", _i32, [_P(ctypes.c_double), _vp]),
    ("o2pic_set_launch_shape", _i32, [_vp, _P(ctypes.c_int32)]),
    ("o2pic_get_launch_shape", _i32, [_vp, _P(ctypes.c_int32)]),
    ("o2pic_batch_create", _i32, [_P(_vp), ctypes.c_int32, _u64, _P(_vp)]),
    ("o2pic_batch_step", _i32, [_vp, _u64]),
    ("o2pic_batch_synchronize", _i32, [_vp]),
    ("o2pic_batch_stream", _vp, [_vp]),
    ("o2pic_batch_autotune", _i32, [_vp, _vp]),
    ("o2pic_batch_destroy", None, [_vp]),
    ("o2pic_mlp_create", _i32, [_P(ctypes.c_int32), ctypes.c_int32, _u64, _P(_vp)]),
    ("o2pic_mlp_num_params", _u64, [_vp]),
    ("o2pic_mlp_set_params", _i32, [_vp, _vp]),
    ("o2pic_mlp_get_params", _i32, [_vp, _vp]),
    ("o2pic_mlp_forward", _i32, [_vp, _vp, _vp, ctypes.c_int32, _vp]),
    ("o2pic_mlp_gradients", _i32, [_vp, _vp, _vp, ctypes.c_int32, _vp, _vp, _vp]),
    ("o2pic_mlp_train_step", _i32, [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_float, _vp, _vp]),
    ("o2pic_mlp_destroy", None, [_vp]),
    ("o2pic_strerror", ctypes.c_char_p, [_i32]),
    ("o2pic_destroy", None, [_vp]),
    ("o2pic_version", _i32, []),
]


def lib():
    """The loaded libo2pic.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with paper_0705_0497_gb300.build.build() "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc, what):
    if rc != OK:
        raise O2picError(rc, what)


def _host_f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _is_torch_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def make_config(cfg, capacity, device=0, compact_check=0):
    c = Config()
    for name in ("L", "f", "U", "p", "T_gas", "C_meta", "dt", "weight", "area", "m_e", "m_OM", "m_OP", "M_gas"):
        setattr(c, name, float(cfg[name]))
    c.n_cells = int(cfg["n_cells"])
    c.ion_subcycle = int(cfg["ion_subcycle"])
    c.seed = int(cfg["seed"])
    c.compact_check = int(compact_check)
    for s in range(NSP):
        c.capacity[s] = int(capacity[s])
    c.device = int(device)
    return c


class Discharge:
    """One discharge on one GPU (a libo2pic context)."""

    def __init__(self, cfg, capacity, device=0, compact_check=0):
        self.cfg = dict(cfg)
        self.Ng = int(cfg["n_cells"]) + 1
        self._c = make_config(cfg, capacity, device, compact_check)
        h = ctypes.c_void_p()
        _check(lib().o2pic_create(ctypes.byref(self._c), ctypes.byref(h)), "o2pic_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().o2pic_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_processes(self, procs):
        arr = (Process * max(len(procs), 1))()
        keep = []
        for i, p in enumerate(procs):
            Ev = np.ascontiguousarray(p["E"], dtype=np.float64)
            sv = np.ascontiguousarray(p["sigma"], dtype=np.float64)
            keep += [Ev, sv]
            arr[i].species, arr[i].kind, arr[i].target, arr[i].n = p["species"], p["kind"], p["target"], len(Ev)
            arr[i].threshold_eV = float(p.get("threshold_eV", 0.0))
            arr[i].E_eV = Ev.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            arr[i].sigma_m2 = sv.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib().o2pic_set_processes(self.h, arr, len(procs)), "o2pic_set_processes")

    def load(self, species, x, vx, vy, vz, ids, stream=None):
        """Host numpy arrays or CUDA torch tensors (float32 / int32-or-uint32 ids)."""
        if _is_torch_cuda(x):
            n = int(x.numel())
            ptrs = [ctypes.c_void_p(t.data_ptr()) for t in (x, vx, vy, vz, ids)]
            kind = DEVICE
        else:
            arrs = [_host_f32(v) for v in (x, vx, vy, vz)] + [np.ascontiguousarray(ids, dtype=np.uint32)]
            n = len(arrs[0])
            ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in arrs]
            kind = HOST
        _check(lib().o2pic_load_particles(self.h, species, *ptrs, n, kind, _stream_ptr(stream)), "o2pic_load_particles")

    def load_state(self, state, stream=None):
        """Load all species; a species dict with "tc" (saved free flights)
        restores them, else fresh flights are drawn at the next step."""
        for s, p in enumerate(state):
            self.load(s, p["x"], p["vx"], p["vy"], p["vz"], p["id"], stream)
            if "tc" in p:
                self.load_flight(s, p["tc"])

    def load_flight(self, species, tc):
        """Free flights (step of each particle's next collision candidate) of
        the particles just loaded into `species` (host array or CUDA tensor)."""
        if _is_torch_cuda(tc):
            ptr, n, kind = ctypes.c_void_p(tc.data_ptr()), int(tc.numel()), DEVICE
        else:
            a = np.ascontiguousarray(tc, dtype=np.uint32)
            ptr, n, kind = a.ctypes.data_as(ctypes.c_void_p), len(a), HOST
        _check(lib().o2pic_load_flight(self.h, species, ptr, n, kind, None), "o2pic_load_flight")

    def flight(self, species):
        """Step of each live particle's next collision candidate, array order."""
        n = self.count(species)
        out = np.zeros(n, np.uint32)
        m = ctypes.c_uint64()
        _check(lib().o2pic_read_flight(self.h, species, out.ctypes.data_as(ctypes.c_void_p), n, ctypes.byref(m), HOST),
               "o2pic_read_flight")
        return out

    def step(self, n=1, stream=None):
        _check(lib().o2pic_step(self.h, int(n), _stream_ptr(stream)), "o2pic_step")

    def synchronize(self):
        _check(lib().o2pic_synchronize(self.h), "o2pic_synchronize")

    def count(self, species):
        n = ctypes.c_uint64()
        _check(lib().o2pic_read_particles(self.h, species, None, None, None, None, None, 0, ctypes.byref(n), HOST),
               "o2pic_read_particles")
        return int(n.value)

    def particles(self, species, flight=False):
        """Live particles of a species in array order (host arrays); with
        flight=True also "tc", their free flights (a saved state that
        load_state resumes bit for bit)."""
        n = self.count(species)
        out = {k: np.zeros(n, np.float32) for k in ("x", "vx", "vy", "vz")}
        out["id"] = np.zeros(n, np.uint32)
        m = ctypes.c_uint64()
        _check(lib().o2pic_read_particles(self.h, species, *[out[k].ctypes.data_as(ctypes.c_void_p)
                                                             for k in ("x", "vx", "vy", "vz", "id")],
                                          n, ctypes.byref(m), HOST), "o2pic_read_particles")
        if flight:
            out["tc"] = self.flight(species)
        return out

    def read_into(self, species, d):
        """Live particles into preallocated host arrays d["x"], ... d["id"]; returns the count."""
        m = ctypes.c_uint64()
        _check(lib().o2pic_read_particles(self.h, species, *[d[k].ctypes.data_as(ctypes.c_void_p)
                                                             for k in ("x", "vx", "vy", "vz", "id")],
                                          len(d["x"]), ctypes.byref(m), HOST), "o2pic_read_particles")
        if m.value > len(d["x"]):
            raise O2picError(-1, "read_into: host arrays too small")
        return int(m.value)

    def particles_into(self, species, x, vx, vy, vz, ids):
        """Live particles into caller CUDA tensors (device to device); returns the live count."""
        m = ctypes.c_uint64()
        _check(lib().o2pic_read_particles(self.h, species, *[ctypes.c_void_p(t.data_ptr()) for t in (x, vx, vy, vz, ids)],
                                          int(x.numel()), ctypes.byref(m), DEVICE), "o2pic_read_particles")
        return int(m.value)

    def field(self):
        phi = np.zeros(self.Ng)
        Ef = np.zeros(self.Ng, np.float32)
        _check(lib().o2pic_read_field(self.h, phi.ctypes.data_as(ctypes.c_void_p), Ef.ctypes.data_as(ctypes.c_void_p)),
               "o2pic_read_field")
        return phi, Ef

    def currents(self, first_step, n):
        """Current densities [n][5] in A/m^2 of steps first_step ..: conduction
        current of e, O-, O2+, displacement current, total (o2pic_read_currents)."""
        out = np.zeros((n, 5))
        _check(lib().o2pic_read_currents(self.h, int(first_step), int(n), out.ctypes.data_as(ctypes.c_void_p)),
               "o2pic_read_currents")
        return out

    def charge(self):
        Q = np.zeros((NSP, self.Ng), np.uint64)
        Qa = np.zeros((NSP, self.Ng), np.uint64)
        steps = ctypes.c_uint64()
        _check(lib().o2pic_read_charge(self.h, Q.ctypes.data_as(ctypes.c_void_p), Qa.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.byref(steps)), "o2pic_read_charge")
        return Q, Qa, int(steps.value)

    def moments(self, reset=False):
        d = np.zeros((NSP, self.Ng))
        steps = ctypes.c_uint64()
        _check(lib().o2pic_read_moments(self.h, d.ctypes.data_as(ctypes.c_void_p), ctypes.byref(steps), int(reset)),
               "o2pic_read_moments")
        return d, int(steps.value)

    def stats(self):
        st = Stats()
        _check(lib().o2pic_get_stats(self.h, ctypes.byref(st)), "o2pic_get_stats")
        return st.as_dict()

    def set_majorant_cap(self, caps):
        """Majorant caps in eV per species (None: the whole grid), taking
        effect at the next set_processes (o2pic_set_majorant_cap)."""
        c = np.array([np.nan if v is None else float(v) for v in caps], np.float64)
        _check(lib().o2pic_set_majorant_cap(self.h, c.ctypes.data), "o2pic_set_majorant_cap")

    def set_coulomb(self, mask, ln_lambda=10.0):
        """Coulomb collisions (1)-(6): bit r-1 of mask enables reaction r."""
        _check(lib().o2pic_set_coulomb(self.h, int(mask), float(ln_lambda)), "o2pic_set_coulomb")

    def set_step(self, n):
        _check(lib().o2pic_set_step(self.h, int(n)), "o2pic_set_step")

    def set_next_id(self, species, next_id):
        _check(lib().o2pic_set_next_id(self.h, int(species), int(next_id)), "o2pic_set_next_id")

    def set_timing(self, on):
        _check(lib().o2pic_set_timing(self.h, int(bool(on))), "o2pic_set_timing")

    def timing(self):
        k = len(KERNEL_KINDS)
        ms = np.zeros(k)
        n = np.zeros(k, np.uint64)
        _check(lib().o2pic_get_timing(self.h, ms.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p),
                                      None, k), "o2pic_get_timing")
        return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(KERNEL_KINDS)}

    def set_launch_shape(self, push_blocks):
        arr = (ctypes.c_int32 * NSP)(*[int(b) for b in push_blocks])
        _check(lib().o2pic_set_launch_shape(self.h, arr), "o2pic_set_launch_shape")

    def launch_shape(self):
        arr = (ctypes.c_int32 * NSP)()
        _check(lib().o2pic_get_launch_shape(self.h, arr), "o2pic_get_launch_shape")
        return tuple(arr)

    def launch_count(self):
        return int(lib().o2pic_launch_count(self.h))


def philox(ctr, key, stream=None):
    """Philox4x32-10 on the device: ctr (n,4), key (n,2) uint32 torch CUDA tensors -> (n,4)."""
    import torch
    out = torch.empty_like(ctr)
    _check(lib().o2pic_philox(ctypes.c_void_p(ctr.data_ptr()), ctypes.c_void_p(key.data_ptr()),
                              ctypes.c_void_p(out.data_ptr()), int(ctr.shape[0]), _stream_ptr(stream)), "o2pic_philox")
    return out


def _ptrs(ts):
    return [ctypes.c_void_p(t.data_ptr()) for t in ts]


def compact_particles(x, vx, vy, vz, ids, stream=None, out=None, noalloc=False):
    """Stable removal of the particles with x = NaN from CUDA tensors; returns
    tensors holding the kept particles in their input order.  `out` = five
    caller tensors to write into (else new ones); noalloc=True uses the entry
    point with static scratch (o2pic_compact_particles_noalloc)."""
    import torch
    n = int(x.numel())
    outs = out if out is not None else [torch.empty(max(n, 1), dtype=t.dtype, device=t.device)
                                        for t in (x, vx, vy, vz, ids)]
    n_out = torch.zeros(1, dtype=torch.int64, device=x.device)
    f = lib().o2pic_compact_particles_noalloc if noalloc else lib().o2pic_compact_particles
    _check(f(*_ptrs((x, vx, vy, vz, ids)), n, *_ptrs(outs), ctypes.c_void_p(n_out.data_ptr()), _stream_ptr(stream)),
           "o2pic_compact_particles" + ("_noalloc" if noalloc else ""))
    m = int(n_out.item())
    return [o[:m] for o in outs]


def ln_f32(x, stream=None):
    import torch
    out = torch.empty_like(x)
    _check(lib().o2pic_ln_f32(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), int(x.numel()),
                              _stream_ptr(stream)), "o2pic_ln_f32")
    return out


class Batch:
    """Many discharges (Discharge objects, borrowed) advanced together by one
    CUDA graph of `steps_per_launch` steps each (o2pic_batch_*)."""

    def __init__(self, discharges, steps_per_launch):
        self.discharges = list(discharges)
        self.K = int(steps_per_launch)
        arr = (ctypes.c_void_p * len(self.discharges))(*[d.h for d in self.discharges])
        h = ctypes.c_void_p()
        _check(lib().o2pic_batch_create(arr, len(self.discharges), self.K, ctypes.byref(h)), "o2pic_batch_create")
        self.h = h

    def step(self, launches=1):
        _check(lib().o2pic_batch_step(self.h, int(launches)), "o2pic_batch_step")

    def synchronize(self):
        _check(lib().o2pic_batch_synchronize(self.h), "o2pic_batch_synchronize")

    def stream(self):
        """The batch's CUDA stream as a torch stream (for events)."""
        import torch
        return torch.cuda.ExternalStream(lib().o2pic_batch_stream(self.h))

    def timed_step(self, launches):
        """step(launches) bracketed by CUDA events on the batch's stream;
        returns the elapsed milliseconds."""
        import torch
        s = self.stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        self.step(launches)
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1)

    def autotune(self):
        r = TuneReport()
        _check(lib().o2pic_batch_autotune(self.h, ctypes.byref(r)), "o2pic_batch_autotune")
        return {"particles_per_warp": [int(r.particles_per_warp[i]) for i in range(r.n)],
                "ms": [float(r.ms[i]) for i in range(r.n)], "chosen": int(r.chosen),
                "fused": bool(r.fused), "other_mode_ms": float(r.other_mode_ms)}

    def close(self):
        if getattr(self, "h", None):
            lib().o2pic_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The warm-start MLP (o2pic_mlp_*): bf16 weights, fp32 accumulation; the
    tensors passed in are CUDA float32 tensors."""

    def __init__(self, widths, seed=0):
        self.widths = [int(w) for w in widths]
        arr = (ctypes.c_int32 * len(self.widths))(*self.widths)
        h = ctypes.c_void_p()
        _check(lib().o2pic_mlp_create(arr, len(self.widths), int(seed), ctypes.byref(h)), "o2pic_mlp_create")
        self.h = h
        self.n = int(lib().o2pic_mlp_num_params(self.h))

    def params(self):
        out = np.zeros(self.n, np.float32)
        _check(lib().o2pic_mlp_get_params(self.h, out.ctypes.data_as(ctypes.c_void_p)), "o2pic_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.n
        _check(lib().o2pic_mlp_set_params(self.h, p.ctypes.data_as(ctypes.c_void_p)), "o2pic_mlp_set_params")

    def forward(self, X, stream=None):
        import torch
        X = X.contiguous()
        Y = torch.empty((X.shape[0], self.widths[-1]), dtype=torch.float32, device=X.device)
        _check(lib().o2pic_mlp_forward(self.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                       int(X.shape[0]), _stream_ptr(stream)), "o2pic_mlp_forward")
        return Y

    def gradients(self, X, T, stream=None):
        import torch
        X, T = X.contiguous(), T.contiguous()
        g = torch.empty(self.n, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(lib().o2pic_mlp_gradients(self.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                         int(X.shape[0]), ctypes.c_void_p(g.data_ptr()),
                                         ctypes.c_void_p(loss.data_ptr()), _stream_ptr(stream)),
               "o2pic_mlp_gradients")
        return g, loss

    def train_step(self, X, T, lr, loss=None, stream=None):
        import torch
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(lib().o2pic_mlp_train_step(self.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                          int(X.shape[0]), float(lr), ctypes.c_void_p(loss.data_ptr()),
                                          _stream_ptr(stream)), "o2pic_mlp_train_step")
        return loss

    def close(self):
        if getattr(self, "h", None):
            lib().o2pic_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
