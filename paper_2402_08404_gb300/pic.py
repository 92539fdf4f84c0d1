"""Thin ctypes binding of libpic.so (C ABI in include/pic.h).  Argument marshalling only: every
step of the computation runs in the library's CUDA kernels.  PyTorch provides the device memory
(caching-allocator callbacks) and the stream.  Importing this module raises if the library was
not built; there is no CPU fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpic.so")

PIC_OK, PIC_E_INVALID, PIC_E_CAPACITY, PIC_E_NOCONV, PIC_E_TIMEOUT, PIC_E_CUDA = 0, -1, -2, -3, -4, -5
ELECTRON, NEUTRAL, ION, ION2 = 0, 1, 2, 3
F_EMISSION, F_EVAP, F_SPUTTER, F_IMPACT_ION, F_DFI, F_HEAT, F_SURROGATE, F_MIXED_MG = (
    0x01, 0x02, 0x04, 0x08, 0x10, 0x20, 0x40, 0x80)
F_ALL = 0xFF
F_FAST_INTEGRAL = 0x100
F_GRAPH = 0x200
F_CIRCUIT = 0x400
F_ELASTIC = 0x800
F_EXTRAPOLATE = 0x1000
F_COULOMB = 0x2000
F_MERGE = 0x4000
F_ION2 = 0x8000
F_PRODUCTION = F_ALL | F_FAST_INTEGRAL     # surrogate, FP32 Gamow quadrature for its fallback, mixed MG

QE = 1.602176634e-19
ME = 9.1093837015e-31
MCU = 63.546 * 1.66053906660e-27


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libpic error {code}: {msg}")
        self.code = code


class Geometry(C.Structure):
    _fields_ = [("tip_radius", C.c_double), ("tip_height", C.c_double)]


class GridT(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double)]


class HostSpeciesT(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("x", "y", "z", "vx", "vy", "vz", "w", "id")] + [("n", C.c_int64)]


class SpeciesT(C.Structure):
    _fields_ = [("charge_e", C.c_int), ("mass", C.c_double), ("capacity", C.c_int64)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("apex_field", C.c_double), ("V0", C.c_double), ("T0", C.c_double),
                ("work_function", C.c_double), ("w_min", C.c_double), ("w_max_units", C.c_int),
                ("n_heat", C.c_int), ("seed", C.c_uint64), ("flags", C.c_uint32), ("mg_tol", C.c_double),
                ("mg_max_cycles", C.c_int), ("mg_sweeps", C.c_int), ("circuit_R", C.c_double),
                ("circuit_C", C.c_double), ("sigma_el_en", C.c_double), ("sigma_el_nn", C.c_double),
                ("sigma_cx", C.c_double), ("coulomb_log", C.c_double), ("merge_max", C.c_int)]


class Diag(C.Structure):
    _fields_ = [("step", C.c_int64), ("next_id", C.c_int64), ("count", C.c_int64 * 4), ("weight", C.c_int64 * 4),
                ("emitted", C.c_int64), ("evaporated", C.c_int64), ("sputtered", C.c_int64),
                ("impact_ionizations", C.c_int64), ("field_ionizations", C.c_int64), ("removed", C.c_int64 * 4),
                ("ion_impacts", C.c_int64), ("total_charge_fixed", C.c_int64), ("mg_cycles", C.c_int),
                ("mg_residual", C.c_double), ("V0", C.c_double), ("max_face_field", C.c_double),
                ("max_J", C.c_double), ("max_T", C.c_double), ("emitted_current", C.c_double),
                ("ms", C.c_double * 8), ("kernel_launches", C.c_int64), ("emission_evals", C.c_int64),
                ("surrogate_faces", C.c_int64), ("V_gap", C.c_double), ("I_gap", C.c_double),
                ("I_tot", C.c_double), ("elastic_en", C.c_int64), ("elastic_nn", C.c_int64),
                ("charge_exchanges", C.c_int64), ("mg_cycles_total", C.c_int64), ("coulomb_ee", C.c_int64),
                ("coulomb_ei", C.c_int64), ("coulomb_ii", C.c_int64), ("merged", C.c_int64),
                ("fallback_range", C.c_int64), ("fallback_bin", C.c_int64), ("double_ionizations", C.c_int64),
                ("ion_ionizations", C.c_int64), ("coulomb_ej", C.c_int64), ("coulomb_ij", C.c_int64),
                ("coulomb_jj", C.c_int64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2402_08404_gb300._build")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, dp, fp = C.c_void_p, C.c_int64, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_float)
        L.pic_create.argtypes = [C.POINTER(Geometry), C.POINTER(GridT), C.POINTER(SpeciesT), i32, C.POINTER(Params),
                                 ALLOC_FN, FREE_FN, vp, vp, C.POINTER(vp)]
        L.pic_destroy.argtypes = [vp]
        L.pic_destroy.restype = None
        L.pic_last_error.argtypes = [vp]
        L.pic_last_error.restype = C.c_char_p
        for name in ("pic_emit", "pic_push", "pic_sort", "pic_collide", "pic_deposit", "pic_solve_field", "pic_heat",
                     "pic_circuit", "pic_merge"):
            getattr(L, name).argtypes = [vp]
        L.pic_step.argtypes = [vp, i32]
        L.pic_load_particles.argtypes = [vp, i32] + [vp] * 8 + [i64]
        L.pic_get_particles.argtypes = [vp, i32] + [vp] * 8 + [i64, C.POINTER(i64)]
        L.pic_load_all.argtypes = [vp, C.POINTER(HostSpeciesT), i32]
        L.pic_set_clock.argtypes = [vp, i64, i64]
        L.pic_save.argtypes = [vp, C.c_char_p]
        L.pic_load.argtypes = [vp, C.c_char_p]
        for name in ("pic_set_potential", "pic_get_potential", "pic_get_efield", "pic_get_charge",
                     "pic_set_temperature", "pic_get_temperature"):
            getattr(L, name).argtypes = [vp, vp]
        L.pic_num_solid.argtypes = [vp, C.POINTER(i64)]
        L.pic_num_faces.argtypes = [vp, C.POINTER(i64)]
        L.pic_get_faces.argtypes = [vp, vp, vp, vp]
        L.pic_get_face_emission.argtypes = [vp, vp, vp, vp]
        L.pic_get_face_accumulators.argtypes = [vp] * 7
        L.pic_set_face_accumulators.argtypes = [vp] * 7
        L.pic_diagnostics.argtypes = [vp, C.POINTER(Diag)]
        L.pic_emission_eval.argtypes = [vp] * 7 + [i64]
        L.pic_emission_eval_noalloc.argtypes = [vp] * 7 + [i64]
        L.pic_set_flags.argtypes = [vp, C.c_uint32]
        L.pic_set_solver.argtypes = [vp, C.c_double, i32]
        L.pic_mlp_num_params.argtypes = []
        L.pic_mlp_set_params.argtypes = [vp, vp]
        L.pic_mlp_get_params.argtypes = [vp, vp]
        L.pic_mlp_forward_backward.argtypes = [vp, vp, vp, i64, vp, vp, vp]
        L.pic_surrogate_train.argtypes = [vp, i64, i32, i32, C.c_double, C.c_uint64, vp]
        L.pic_surrogate_eval.argtypes = [vp] * 8 + [i64]
        L.pic_batch_create.argtypes = [C.POINTER(vp), i32, C.POINTER(vp)]
        L.pic_batch_step.argtypes = [vp, i32]
        L.pic_batch_ms.argtypes = [vp, dp]
        L.pic_batch_last_error.argtypes = [vp]
        L.pic_batch_last_error.restype = C.c_char_p
        L.pic_batch_destroy.argtypes = [vp]
        L.pic_batch_destroy.restype = None
        L.pic_autotune.argtypes = [vp, C.POINTER(i32), i32]
        L.pic_surrogate_copy.argtypes = [vp, vp]
        L.pic_num_kernels.argtypes = []
        L.pic_kernel_name.argtypes = [i32]
        L.pic_kernel_name.restype = C.c_char_p
        L.pic_set_kernel_timing.argtypes = [vp, C.c_uint64]
        L.pic_get_kernel_timing.argtypes = [vp, i32, C.POINTER(i64), dp, dp]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, on the handle's stream."""

    def __init__(self):
        import torch
        self.torch = torch
        self.live = {}

        def alloc(nbytes, stream, user):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream)
            except Exception:
                return None
            self.live[p] = nbytes
            return p

        def free(ptr, nbytes, stream, user):
            if ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = ALLOC_FN(alloc)
        self.free_fn = FREE_FN(free)


def species_table(cap, ion2=False):
    """e-, Cu, Cu+, Cu2+ entries; Cu2+ room: cap[3] if given, else Cu+'s with F_ION2, else 1024 SPs."""
    if np.isscalar(cap):
        cap = (cap, cap, cap)
    cap_j = cap[3] if len(cap) > 3 else (cap[2] if ion2 else 1024)
    return (SpeciesT * 4)(SpeciesT(-1, ME, int(cap[0])), SpeciesT(0, MCU, int(cap[1])), SpeciesT(1, MCU, int(cap[2])),
                          SpeciesT(2, MCU, int(cap_j)))


class Pic:
    """One vacuum-arc PIC-MCC instance on the current CUDA device."""

    def __init__(self, cfg, capacity, flags=F_ALL, mg_tol=1e-8, mg_max_cycles=60, V0=0.0, stream=None,
                 torch_memory=True, mg_sweeps=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libpic needs a CUDA device")
        L = lib()
        self.cfg = dict(cfg)
        self._alloc = _TorchAllocator() if torch_memory else None
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        geo = Geometry(cfg["tip_radius"], cfg["tip_height"])
        grid = GridT(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"])
        prm = Params(cfg["dt"], cfg["apex_field"], V0, cfg["T0"], cfg["work_function"], cfg["w_min"],
                     int(cfg["w_max_units"]), int(cfg.get("n_heat", 0)), int(cfg.get("seed", 1)), int(flags),
                     float(mg_tol), int(mg_max_cycles), int(mg_sweeps), float(cfg.get("circuit_R", 0.0)),
                     float(cfg.get("circuit_C", 0.0)), float(cfg.get("sigma_el_en", 0.0)),
                     float(cfg.get("sigma_el_nn", 0.0)), float(cfg.get("sigma_cx", 0.0)),
                     float(cfg.get("coulomb_log", 0.0)), int(cfg.get("merge_max", 0)))
        h = C.c_void_p()
        a = self._alloc.alloc_fn if self._alloc else ALLOC_FN(0)
        f = self._alloc.free_fn if self._alloc else FREE_FN(0)
        rc = L.pic_create(C.byref(geo), C.byref(grid), species_table(capacity, bool(flags & F_ION2)), 4,
                          C.byref(prm), a, f, None,
                          C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != PIC_OK:
            raise PicError(rc, "pic_create failed")
        self.h = h
        n = C.c_int64()
        L.pic_num_faces(self.h, C.byref(n))
        self.nface = n.value
        L.pic_num_solid(self.h, C.byref(n))
        self.nsolid = n.value
        self.nnode = (cfg["nx"] + 1) * (cfg["ny"] + 1) * (cfg["nz"] + 1)
        self.node_shape = (cfg["nz"] + 1, cfg["ny"] + 1, cfg["nx"] + 1)

    def close(self):
        if getattr(self, "h", None):
            lib().pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != PIC_OK:
            raise PicError(rc, lib().pic_last_error(self.h).decode())

    # -- state ---------------------------------------------------------------------------------
    def load_particles(self, species, sp):
        arrs = [np.ascontiguousarray(sp[k], dtype=t) for k, t in
                (("x", np.float32), ("y", np.float32), ("z", np.float32), ("vx", np.float32), ("vy", np.float32),
                 ("vz", np.float32), ("w", np.int32), ("id", np.uint64))]
        self._check(lib().pic_load_particles(self.h, species, *[_ptr(a) for a in arrs], len(arrs[0])))

    def load_all(self, pops):
        """pic_load_all: pops[s] holds the SoA arrays of species s (pinned host memory copies at full
        bandwidth); the next species' copies overlap the current one's check and sort."""
        keep, tab = [], (HostSpeciesT * len(pops))()
        for s, sp in enumerate(pops):
            arrs = [np.ascontiguousarray(sp[k], dtype=t) for k, t in
                    (("x", np.float32), ("y", np.float32), ("z", np.float32), ("vx", np.float32), ("vy", np.float32),
                     ("vz", np.float32), ("w", np.int32), ("id", np.uint64))]
            keep.append(arrs)
            tab[s] = HostSpeciesT(*[_ptr(a) for a in arrs], len(arrs[0]))
        self._check(lib().pic_load_all(self.h, tab, len(pops)))

    def get_particles(self, species, cap=None):
        n = C.c_int64()
        lib().pic_get_particles(self.h, species, *([None] * 8), 0, C.byref(n))
        m = n.value
        out = {k: np.zeros(m, dtype=t) for k, t in (("x", np.float32), ("y", np.float32), ("z", np.float32),
                                                      ("vx", np.float32), ("vy", np.float32), ("vz", np.float32),
                                                      ("w", np.int32), ("id", np.uint64))}
        self._check(lib().pic_get_particles(self.h, species, *[_ptr(out[k]) for k in
                                                               ("x", "y", "z", "vx", "vy", "vz", "w", "id")],
                                            m, C.byref(n)))
        return out

    def set_clock(self, step, next_id):
        self._check(lib().pic_set_clock(self.h, int(step), int(next_id)))

    def save(self, path):
        """pic_save: the whole evolving state to a file (between steps or after a sort)."""
        self._check(lib().pic_save(self.h, os.fsencode(path)))

    def load(self, path):
        """pic_load: state from a pic_save file into this handle (same creation inputs)."""
        self._check(lib().pic_load(self.h, os.fsencode(path)))

    def set_potential(self, phi):
        a = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        assert a.size == self.nnode
        self._check(lib().pic_set_potential(self.h, _ptr(a)))

    def get_potential(self):
        a = np.zeros(self.nnode)
        self._check(lib().pic_get_potential(self.h, _ptr(a)))
        return a.reshape(self.node_shape)

    def get_efield(self):
        a = np.zeros(self.nnode * 3, dtype=np.float32)
        self._check(lib().pic_get_efield(self.h, _ptr(a)))
        return a.reshape(self.node_shape + (3,))

    def get_charge(self):
        a = np.zeros(self.nnode, dtype=np.int64)
        self._check(lib().pic_get_charge(self.h, _ptr(a)))
        return a.reshape(self.node_shape)

    def set_temperature(self, T):
        a = np.ascontiguousarray(T, dtype=np.float64)
        assert a.size == self.nsolid
        self._check(lib().pic_set_temperature(self.h, _ptr(a)))

    def get_temperature(self):
        a = np.zeros(self.nsolid)
        self._check(lib().pic_get_temperature(self.h, _ptr(a)))
        return a

    def faces(self):
        v = np.zeros(self.nface, np.int64)
        d = np.zeros(self.nface, np.int32)
        o = np.zeros(self.nface, np.int64)
        self._check(lib().pic_get_faces(self.h, _ptr(v), _ptr(d), _ptr(o)))
        return v, d, o

    def face_emission(self):
        F, J, P = (np.zeros(self.nface) for _ in range(3))
        self._check(lib().pic_get_face_emission(self.h, _ptr(F), _ptr(J), _ptr(P)))
        return F, J, P

    def face_accumulators(self):
        ev, he, ch = (np.zeros(self.nface) for _ in range(3))
        sp_, eb, es = (np.zeros(self.nface, np.int64) for _ in range(3))
        self._check(lib().pic_get_face_accumulators(self.h, *[_ptr(a) for a in (ev, he, ch, sp_, eb, es)]))
        return {"evap": ev, "heat": he, "charge": ch, "sput": sp_, "Eb": eb, "Es": es}

    def set_face_accumulators(self, acc):
        arrs = [np.ascontiguousarray(acc[k], dtype=t) for k, t in (("evap", np.float64), ("heat", np.float64),
                                                                    ("charge", np.float64), ("sput", np.int64),
                                                                    ("Eb", np.int64), ("Es", np.int64))]
        self._check(lib().pic_set_face_accumulators(self.h, *[_ptr(a) for a in arrs]))

    def set_flags(self, flags):
        self._check(lib().pic_set_flags(self.h, int(flags)))

    def set_solver(self, mg_tol, mg_max_cycles):
        self._check(lib().pic_set_solver(self.h, float(mg_tol), int(mg_max_cycles)))

    # -- stages --------------------------------------------------------------------------------
    def emit(self):
        self._check(lib().pic_emit(self.h))

    def push(self):
        self._check(lib().pic_push(self.h))

    def sort(self):
        self._check(lib().pic_sort(self.h))

    def merge(self):
        self._check(lib().pic_merge(self.h))

    def circuit(self):
        self._check(lib().pic_circuit(self.h))

    def collide(self):
        self._check(lib().pic_collide(self.h))

    def deposit(self):
        self._check(lib().pic_deposit(self.h))

    def solve_field(self):
        self._check(lib().pic_solve_field(self.h))

    def heat(self):
        self._check(lib().pic_heat(self.h))

    def step(self, nsteps=1):
        self._check(lib().pic_step(self.h, int(nsteps)))

    def diagnostics(self):
        d = Diag()
        self._check(lib().pic_diagnostics(self.h, C.byref(d)))
        out = {}
        for name, _ in Diag._fields_:
            v = getattr(d, name)
            out[name] = list(v) if isinstance(v, C.Array) else v
        return out

    # -- autotuner ------------------------------------------------------------------------------------
    def autotune(self):
        """pic_autotune: {"particle_blocks_per_sm": b, "residual_planes_per_thread": r,
        "smoother_planes_per_thread": [per level]}."""
        buf = (C.c_int * 18)()
        n = lib().pic_autotune(self.h, buf, 18)
        if n < 0:
            self._check(n)
        return {"particle_blocks_per_sm": buf[0], "residual_planes_per_thread": buf[1],
                "smoother_planes_per_thread": list(buf[2:n])}

    # -- kernel timing (diagnostics) ----------------------------------------------------------------
    @staticmethod
    def kernel_names():
        return [lib().pic_kernel_name(k).decode() for k in range(lib().pic_num_kernels())]

    def set_kernel_timing(self, names=()):
        """Time every launch of the named kernels (CUDA events on the library stream); () = off."""
        idx = {n: k for k, n in enumerate(self.kernel_names())}
        mask = 0
        for n in names:
            mask |= 1 << idx[n]
        self._check(lib().pic_set_kernel_timing(self.h, C.c_uint64(mask)))

    def kernel_timing(self):
        """{name: (launches, ms, units)} of the kernels timed since the last set_kernel_timing."""
        out = {}
        for k, n in enumerate(self.kernel_names()):
            cnt, ms, un = C.c_int64(), C.c_double(), C.c_double()
            self._check(lib().pic_get_kernel_timing(self.h, k, C.byref(cnt), C.byref(ms), C.byref(un)))
            if cnt.value:
                out[n] = (cnt.value, ms.value, un.value)
        return out

    # -- emission surrogate ------------------------------------------------------------------------
    def mlp_params(self):
        p = np.zeros(lib().pic_mlp_num_params(), dtype=np.float32)
        self._check(lib().pic_mlp_get_params(self.h, _ptr(p)))
        return p

    def set_mlp_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == lib().pic_mlp_num_params()
        self._check(lib().pic_mlp_set_params(self.h, _ptr(p)))

    def mlp_forward_backward(self, x, t=None):
        """y (n x 2); with targets t also (loss, flat gradient in the public parameter layout)."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        n = x.shape[0]
        y = np.zeros((n, 2), dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        g = np.zeros(lib().pic_mlp_num_params(), dtype=np.float32)
        tt = None if t is None else np.ascontiguousarray(t, dtype=np.float32)
        self._check(lib().pic_mlp_forward_backward(self.h, _ptr(x), _ptr(tt), n, _ptr(y),
                                                   _ptr(loss) if t is not None else None,
                                                   _ptr(g) if t is not None else None))
        return (y,) if t is None else (y, float(loss[0]), g)

    def surrogate_train(self, nsamples=2_000_000, epochs=60, batch=8192, lr=2e-3, seed=1):
        st = np.zeros(8)
        self._check(lib().pic_surrogate_train(self.h, int(nsamples), int(epochs), int(batch), float(lr), int(seed),
                                              _ptr(st)))
        keys = ("train_loss", "val_rms_dlog10J", "val_max_dlog10J", "valid_bin_fraction", "valid_sample_fraction",
                "ms_data", "ms_train", "steps")
        return dict(zip(keys, st.tolist()))

    def surrogate_eval(self, F, T, W, R):
        F, T, W, R = (np.ascontiguousarray(np.broadcast_to(a, np.shape(F)), dtype=np.float64) for a in (F, T, W, R))
        J = np.zeros(F.size)
        P = np.zeros(F.size)
        v = np.zeros(F.size, dtype=np.uint8)
        self._check(lib().pic_surrogate_eval(self.h, _ptr(F), _ptr(T), _ptr(W), _ptr(R), _ptr(J), _ptr(P), _ptr(v),
                                             F.size))
        return J, P, v.astype(bool)

    def surrogate_copy_from(self, other):
        """Install the trained surrogate of another instance (pic_surrogate_copy)."""
        self._check(lib().pic_surrogate_copy(self.h, other.h))

    def emission_eval_noalloc(self, F, T, W, R):
        """pic_emission_eval_noalloc: the same evaluation staged through the library's fixed
        device array (no device allocation; at most PIC_NOALLOC_MAX_TUPLES tuples per call)."""
        F, T, W, R = (np.ascontiguousarray(np.broadcast_to(a, np.shape(F)), dtype=np.float64) for a in (F, T, W, R))
        J = np.zeros(F.size)
        P = np.zeros(F.size)
        self._check(lib().pic_emission_eval_noalloc(self.h, _ptr(F), _ptr(T), _ptr(W), _ptr(R), _ptr(J), _ptr(P),
                                                    F.size))
        return J, P

    def emission_eval(self, F, T, W, R):
        F, T, W, R = (np.ascontiguousarray(np.broadcast_to(a, np.shape(F)), dtype=np.float64) for a in (F, T, W, R))
        J = np.zeros(F.size)
        P = np.zeros(F.size)
        self._check(lib().pic_emission_eval(self.h, _ptr(F), _ptr(T), _ptr(W), _ptr(R), _ptr(J), _ptr(P), F.size))
        return J, P


class Batch:
    """pic_batch_*: independent instances (sharing one stream) stepped by one graph launch per step."""

    def __init__(self, sims):
        self.sims = list(sims)
        arr = (C.c_void_p * len(self.sims))(*[x.h.value for x in self.sims])
        b = C.c_void_p()
        rc = lib().pic_batch_create(arr, len(self.sims), C.byref(b))
        if rc != PIC_OK:
            raise PicError(rc, "pic_batch_create failed (distinct handles on one stream required)")
        self.b = b

    def step(self, nsteps=1):
        rc = lib().pic_batch_step(self.b, int(nsteps))
        if rc != PIC_OK:
            raise PicError(rc, lib().pic_batch_last_error(self.b).decode())

    def ms(self):
        v = C.c_double()
        lib().pic_batch_ms(self.b, C.byref(v))
        return v.value

    def close(self):
        if getattr(self, "b", None):
            lib().pic_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
