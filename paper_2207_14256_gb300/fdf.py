"""Python binding of libfdf.so (include/fdf.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Host arrays are
numpy arrays; device arrays are CUDA torch tensors (their data_ptr is passed
with the on-device flag set).  Errors raise FdfError carrying the C return code
and the library's last message.  There is no fallback: if libfdf.so is missing
or fails to load, every call raises.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfdf.so")

FDF_OK, FDF_EINVAL, FDF_ENOMEM, FDF_ECUDA, FDF_ESTATE, FDF_ETIMEOUT, FDF_ENAN, FDF_ENOSYS = 0, -1, -2, -3, -4, -5, -6, -7
FDF_PREC_F64, FDF_PREC_F32, FDF_PREC_BF16, FDF_PREC_F32_FIXED, FDF_PREC_BF16_FIXED = 0, 1, 2, 3, 4
FDF_FLAG_FIXED_AMPLITUDE, FDF_FLAG_LEGENDRE_DIPOLE = 1, 2
FDF_Q_W_EPS, FDF_Q_W, FDF_Q_EPS, FDF_Q_COUNT, FDF_Q_W_QX, FDF_Q_W_QY, FDF_Q_W_QZ = 0, 1, 2, 3, 4, 5, 6
FDF_EOM_GEODESIC, FDF_EOM_CANONICAL, FDF_EOM_SR_NEWTON, FDF_EOM_Q_SIMPLE, FDF_EOM_NEWTONIAN = 0, 1, 2, 3, 4
FDF_EOM_EXACT = 5
FDF_K_PUSH, FDF_K_FIELDS_Z, FDF_K_FIELDS_Y, FDF_K_FIELDS_X, FDF_K_OTHER, FDF_K_SORT = 0, 1, 2, 3, 4, 5
KERNEL_CLASSES = {"push": 0, "fields_z": 1, "fields_y": 2, "fields_x": 3, "other": 4, "sort": 5}


class FdfError(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__("%s failed: %s (%d): %s" % (where, fdf_error_string(code), code, msg))
        self.code = code


class fdf_params(C.Structure):
    _fields_ = [
        ("box_mpc", C.c_double),
        ("n_part", C.c_int64),
        ("n_grid", C.c_int32),
        ("n_species", C.c_int32),
        ("m_ev", C.c_double * 4),
        ("T_nu_K", C.c_double),
        ("z_start", C.c_double),
        ("z_end", C.c_double),
        ("n_steps", C.c_int32),
        ("precision", C.c_int32),
        ("seed", C.c_uint64),
        ("h", C.c_double),
        ("omega_m", C.c_double),
        ("omega_r", C.c_double),
        ("A_s", C.c_double),
        ("n_s", C.c_double),
        ("k_pivot", C.c_double),
        ("flags", C.c_int32),
        ("n_gl", C.c_int32),
        ("sort_every", C.c_int32),
        ("steps_per_pass", C.c_int32),
        ("sort_tile", C.c_int32),
        ("sort_cells", C.c_int32),
        ("interp_order", C.c_int32),
        ("superstep_tol", C.c_double),
        ("eom", C.c_int32),
        ("pass_blocks", C.c_int32),
        ("gather_tile", C.c_int32),
        ("deposit_presum", C.c_int32),
    ]


class fdf_tables(C.Structure):
    _fields_ = [
        ("nk", C.c_int32),
        ("na", C.c_int32),
        ("lnk", C.POINTER(C.c_double)),
        ("lna", C.POINTER(C.c_double)),
        ("T_psi", C.POINTER(C.c_double)),
        ("T_phi", C.POINTER(C.c_double)),
        ("dTphi_dlna", C.POINTER(C.c_double)),
        ("ncdf", C.c_int32),
        ("cdf_t", C.POINTER(C.c_double)),
        ("cdf_F", C.POINTER(C.c_double)),
    ]


FDF_REQ_QUEUED, FDF_REQ_RUNNING, FDF_REQ_DONE, FDF_REQ_FAILED = 0, 1, 2, 3
FDF_SERVER_MERGE_PASSES = 1


class fdf_request_info(C.Structure):
    _fields_ = [
        ("id", C.c_int64),
        ("status", C.c_int32),
        ("error", C.c_int32),
        ("t_submit", C.c_double),
        ("t_admit", C.c_double),
        ("t_done", C.c_double),
        ("footprint", C.c_size_t),
        ("particle_steps", C.c_int64),
        ("message", C.c_char * 160),
    ]


_lib = None
_V = C.c_void_p
_D = C.POINTER(C.c_double)


def lib():
    """Load libfdf.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfdf.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        P = C.POINTER(fdf_params)
        T = C.POINTER(fdf_tables)
        sig = {
            "fdf_footprint": (C.c_int, [P, C.POINTER(C.c_size_t)]),
            "fdf_create": (C.c_int, [P, T, _V, _V, C.c_size_t, C.POINTER(_V)]),
            "fdf_sample": (C.c_int, [_V]),
            "fdf_step": (C.c_int, [_V, C.c_int32]),
            "fdf_run_graph": (C.c_int, [_V, C.c_int32]),
            "fdf_accel_terms": (C.c_int, [_V, C.c_int32, _D]),
            "fdf_deposit": (C.c_int, [_V, C.c_int32, C.c_int32, _V, C.c_int32]),
            "fdf_deposit_subset": (C.c_int, [_V, C.c_int32, C.c_int32, C.c_int32, _V, C.c_int32]),
            "fdf_get": (C.c_int, [_V, C.c_int32, _V, _V, _V, C.c_int32]),
            "fdf_get_initial": (C.c_int, [_V, C.c_int32, _V, _V, _V, C.c_int32]),
            "fdf_build_fields": (C.c_int, [_V, C.c_double, _V, C.c_int32]),
            "fdf_set_fields": (C.c_int, [_V, _V, C.c_int32]),
            "fdf_build_fields_noalloc": (C.c_int, [P, T, C.c_double, _V, _V]),
            "fdf_supersteps": (C.c_int, [_V, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32)]),
            "fdf_state": (C.c_int, [_V, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
            "fdf_pass_info": (C.c_int, [_V, C.POINTER(C.c_int32)]),
            "fdf_timing": (C.c_int, [_V, C.c_int32]),
            "fdf_kernel_time": (C.c_int, [_V, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
            "fdf_launch_count": (C.c_int64, [_V]),
            "fdf_pipe_rates": (C.c_int, [_V, _D, _D, _D]),
            "fdf_error_string": (C.c_char_p, [C.c_int]),
            "fdf_last_error": (C.c_char_p, []),
            "fdf_destroy": (None, [_V]),
            "fdf_tune": (C.c_int, [P, T, _V, P, C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
            "fdf_server_create": (C.c_int, [C.c_size_t, C.c_int32, C.c_int32, C.POINTER(_V)]),
            "fdf_server_create_opts": (C.c_int, [C.c_size_t, C.c_int32, C.c_int32, C.c_int32, C.POINTER(_V)]),
            "fdf_server_merged_launches": (C.c_int, [_V, C.POINTER(C.c_int64)]),
            "fdf_server_submit": (C.c_int, [_V, P, T, C.POINTER(C.c_int64)]),
            "fdf_server_wait": (C.c_int, [_V, C.c_int32, C.POINTER(C.c_int64)]),
            "fdf_server_info": (C.c_int, [_V, C.c_int64, C.POINTER(fdf_request_info)]),
            "fdf_server_get": (C.c_int, [_V, C.c_int64, C.c_int32, _V, _V, _V, C.c_int32]),
            "fdf_server_deposit": (C.c_int, [_V, C.c_int64, _V, C.c_int32]),
            "fdf_server_release": (C.c_int, [_V, C.c_int64]),
            "fdf_server_clock": (C.c_double, [_V]),
            "fdf_server_load": (C.c_int, [_V, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_size_t)]),
            "fdf_server_destroy": (None, [_V]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc, where):
    if rc != FDF_OK:
        raise FdfError(rc, where, fdf_last_error())


def _ptr(a):
    """(pointer, on_device) for a numpy array, a CUDA torch tensor or None."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"] or not a.flags["WRITEABLE"]:
            raise ValueError("host arrays must be C-contiguous and writeable")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor, got %r" % type(a))


def _same_side(ptrs):
    dev = {d for p, d in ptrs if p is not None}
    if len(dev) > 1:
        raise ValueError("outputs must all be on the host or all on the device")
    return dev.pop() if dev else 0


def make_params(d):
    """fdf_params from a dict with the keys of inputs.config() (box, n_part, n_grid, ...)."""
    p = fdf_params()
    m = list(d["m_ev"]) + [0.0] * (4 - len(d["m_ev"]))
    p.box_mpc = d["box"]
    p.n_part = int(d["n_part"])
    p.n_grid = int(d["n_grid"])
    p.n_species = int(d.get("n_species", 1))
    p.m_ev = (C.c_double * 4)(*m)
    p.T_nu_K = d["T_K"]
    p.z_start = d["z_start"]
    p.z_end = d["z_end"]
    p.n_steps = int(d["n_steps"])
    p.precision = int(d.get("precision", FDF_PREC_F32))
    p.seed = int(d["seed"])
    p.h, p.omega_m, p.omega_r = d["h"], d["omega_m"], d["omega_r"]
    p.A_s, p.n_s, p.k_pivot = d["A_s"], d["n_s"], d["k_pivot"]
    p.flags = int(d.get("flags", 0))
    p.n_gl = int(d.get("n_gl", 0))
    p.sort_every = int(d.get("sort_every", 0))
    p.steps_per_pass = int(d.get("steps_per_pass", 0))
    p.sort_tile = int(d.get("sort_tile", 0))
    p.sort_cells = int(d.get("sort_cells", 0))
    p.interp_order = int(d.get("interp_order", 0))
    p.superstep_tol = float(d.get("superstep_tol", 0.0))
    p.eom = int(d.get("eom", 0))
    p.pass_blocks = int(d.get("pass_blocks", 0))
    p.gather_tile = int(d.get("gather_tile", 0))
    p.deposit_presum = int(d.get("deposit_presum", 0))
    return p


def knobs(p):
    """The schedule knobs of an fdf_params as a dict (for reports)."""
    return {k: int(getattr(p, k)) for k in ("sort_every", "sort_cells", "sort_tile", "steps_per_pass", "pass_blocks",
                                             "gather_tile", "n_gl")}


def make_tables(d):
    """(fdf_tables, keep-alive list) from a dict of float64 arrays (inputs.transfer_tables())."""
    keep = []
    t = fdf_tables()
    for k in ("lnk", "lna", "T_psi", "T_phi", "dTphi_dlna", "cdf_t", "cdf_F"):
        a = np.ascontiguousarray(d[k], dtype=np.float64)
        keep.append(a)
        setattr(t, k, a.ctypes.data_as(_D))
    t.nk = len(d["lnk"])
    t.na = len(d["lna"])
    t.ncdf = len(d["cdf_t"])
    return t, keep


# ---- entry points ------------------------------------------------------------------------
def fdf_footprint(params):
    b = C.c_size_t(0)
    _check(lib().fdf_footprint(C.byref(params), C.byref(b)), "fdf_footprint")
    return b.value


def fdf_create(params, tables, stream=None, arena=None, arena_bytes=0):
    """stream: a torch.cuda.Stream, an int cudaStream_t or None; arena: a CUDA tensor or None."""
    s = getattr(stream, "cuda_stream", stream)
    ap, _ = _ptr(arena)
    if arena is not None and not arena_bytes:
        arena_bytes = arena.numel() * arena.element_size()
    ctx = _V()
    _check(lib().fdf_create(C.byref(params), C.byref(tables), s, ap, arena_bytes, C.byref(ctx)), "fdf_create")
    return ctx


def fdf_sample(ctx):
    _check(lib().fdf_sample(ctx), "fdf_sample")


def fdf_step(ctx, n):
    _check(lib().fdf_step(ctx, int(n)), "fdf_step")


def fdf_accel_terms(ctx, species=-1):
    """RMS of the four terms of eq:releq and of their sum at the current step (Fig. 2)."""
    out = np.zeros(5)
    _check(lib().fdf_accel_terms(ctx, int(species), out.ctypes.data_as(C.POINTER(C.c_double))), "fdf_accel_terms")
    return out


def fdf_run_graph(ctx, n):
    """fdf_sample + fdf_step(n) as one CUDA graph, recorded on the first call for n."""
    _check(lib().fdf_run_graph(ctx, int(n)), "fdf_run_graph")


def fdf_deposit(ctx, species, quantity, out):
    p, dev = _ptr(out)
    _check(lib().fdf_deposit(ctx, species, quantity, p, dev), "fdf_deposit")
    return out


def fdf_deposit_subset(ctx, species, quantity, parity, out):
    p, dev = _ptr(out)
    _check(lib().fdf_deposit_subset(ctx, species, quantity, parity, p, dev), "fdf_deposit_subset")
    return out


def fdf_get(ctx, species, x=None, q=None, w=None):
    ptrs = [_ptr(a) for a in (x, q, w)]
    dev = _same_side(ptrs)
    _check(lib().fdf_get(ctx, species, ptrs[0][0], ptrs[1][0], ptrs[2][0], dev), "fdf_get")
    return x, q, w


def fdf_get_initial(ctx, species, X=None, q_sampled=None, p=None):
    ptrs = [_ptr(a) for a in (X, q_sampled, p)]
    dev = _same_side(ptrs)
    _check(lib().fdf_get_initial(ctx, species, ptrs[0][0], ptrs[1][0], ptrs[2][0], dev), "fdf_get_initial")
    return X, q_sampled, p


def fdf_build_fields(ctx, lna, out):
    p, dev = _ptr(out)
    _check(lib().fdf_build_fields(ctx, float(lna), p, dev), "fdf_build_fields")
    return out


def fdf_build_fields_noalloc(params, tables, lna, out, stream=None):
    """out: a contiguous float64 CUDA tensor of 8 N^3 elements on the current device (the
    entry point allocates nothing and writes all of it).  Anything else raises before the
    library is called."""
    if not (hasattr(out, "data_ptr") and hasattr(out, "is_cuda")):
        raise TypeError("fdf_build_fields_noalloc writes device memory: pass a torch tensor")
    if str(out.dtype) != "torch.float64":
        raise ValueError("out must be float64, got %s" % out.dtype)
    N = int(params.n_grid)
    if out.numel() != 8 * N ** 3:
        raise ValueError("out must hold 8 n_grid^3 = %d doubles, got %d" % (8 * N ** 3, out.numel()))
    if not out.is_contiguous():
        raise ValueError("out must be contiguous")
    if not out.is_cuda:
        raise ValueError("fdf_build_fields_noalloc writes device memory: pass a CUDA tensor")
    import torch

    if out.device.index != torch.cuda.current_device():
        raise ValueError("out is on cuda:%d but the current device is cuda:%d"
                         % (out.device.index, torch.cuda.current_device()))
    p = out.data_ptr()
    s = getattr(stream, "cuda_stream", stream)
    _check(lib().fdf_build_fields_noalloc(C.byref(params), C.byref(tables), float(lna), p, s),
           "fdf_build_fields_noalloc")
    return out


def fdf_set_fields(ctx, fields):
    if fields is None:
        _check(lib().fdf_set_fields(ctx, None, 0), "fdf_set_fields")
        return
    if isinstance(fields, np.ndarray):
        fields = np.ascontiguousarray(fields, dtype=np.float64)
    p, dev = _ptr(fields)
    _check(lib().fdf_set_fields(ctx, p, dev), "fdf_set_fields")


def fdf_supersteps(ctx, n_steps):
    """(is_super array of n_steps + 1, count)."""
    out = np.zeros(n_steps + 1, np.int32)
    cnt = C.c_int32(0)
    _check(lib().fdf_supersteps(ctx, out.ctypes.data_as(C.POINTER(C.c_int32)), len(out), C.byref(cnt)),
           "fdf_supersteps")
    return out, cnt.value


def fdf_pass_info(ctx):
    """dict(form, series, passes, steps_per_pass) of the last fdf_step or fdf_run_graph run."""
    info = np.zeros(4, np.int32)
    _check(lib().fdf_pass_info(ctx, info.ctypes.data_as(C.POINTER(C.c_int32))), "fdf_pass_info")
    return dict(form=int(info[0]), series=int(info[1]), passes=int(info[2]), steps_per_pass=int(info[3]))


def fdf_state(ctx):
    k = C.c_int32(0)
    l = C.c_double(0)
    _check(lib().fdf_state(ctx, C.byref(k), C.byref(l)), "fdf_state")
    return k.value, l.value


def fdf_timing(ctx, enable):
    _check(lib().fdf_timing(ctx, 1 if enable else 0), "fdf_timing")


def fdf_kernel_time(ctx, which):
    ms = C.c_double(0)
    n = C.c_int64(0)
    _check(lib().fdf_kernel_time(ctx, which, C.byref(ms), C.byref(n)), "fdf_kernel_time")
    return ms.value, n.value


def fdf_pipe_rates(stream=None):
    """(FP64 FMA/s, FP32 FMA/s, FP64->FP32->FP64 round trips/s) measured on the current device."""
    s = getattr(stream, "cuda_stream", stream)
    d, f, c = C.c_double(0), C.c_double(0), C.c_double(0)
    _check(lib().fdf_pipe_rates(s, C.byref(d), C.byref(f), C.byref(c)), "fdf_pipe_rates")
    return d.value, f.value, c.value


def fdf_launch_count(ctx):
    return int(lib().fdf_launch_count(ctx))


def fdf_error_string(code):
    return lib().fdf_error_string(code).decode()


def fdf_last_error():
    return lib().fdf_last_error().decode()


def fdf_destroy(ctx):
    if ctx:
        lib().fdf_destroy(ctx)


def fdf_tune(params, tables, stream=None):
    """Returns (tuned fdf_params, best run ms, timed runs)."""
    s = getattr(stream, "cuda_stream", stream)
    out = fdf_params()
    ms = C.c_double(0)
    n = C.c_int32(0)
    _check(lib().fdf_tune(C.byref(params), C.byref(tables), s, C.byref(out), C.byref(ms), C.byref(n)), "fdf_tune")
    return out, ms.value, n.value


def fdf_server_create(hbm_budget, max_active, slice_steps):
    srv = _V()
    _check(lib().fdf_server_create(int(hbm_budget), int(max_active), int(slice_steps), C.byref(srv)),
           "fdf_server_create")
    return srv


def fdf_server_create_opts(hbm_budget, max_active, slice_steps, options):
    srv = _V()
    _check(lib().fdf_server_create_opts(int(hbm_budget), int(max_active), int(slice_steps), int(options),
                                        C.byref(srv)), "fdf_server_create_opts")
    return srv


def fdf_server_merged_launches(srv):
    n = C.c_int64(0)
    _check(lib().fdf_server_merged_launches(srv, C.byref(n)), "fdf_server_merged_launches")
    return n.value


def fdf_server_submit(srv, params, tables):
    rid = C.c_int64(0)
    _check(lib().fdf_server_submit(srv, C.byref(params), C.byref(tables), C.byref(rid)), "fdf_server_submit")
    return rid.value


def fdf_server_wait(srv, timeout_ms=-1):
    """Id of the next finished request, or None on timeout."""
    rid = C.c_int64(0)
    rc = lib().fdf_server_wait(srv, int(timeout_ms), C.byref(rid))
    if rc == FDF_ETIMEOUT:
        return None
    _check(rc, "fdf_server_wait")
    return rid.value


def fdf_server_info(srv, rid):
    info = fdf_request_info()
    _check(lib().fdf_server_info(srv, int(rid), C.byref(info)), "fdf_server_info")
    return info


def fdf_server_get(srv, rid, species, x=None, q=None, w=None):
    ptrs = [_ptr(a) for a in (x, q, w)]
    dev = _same_side(ptrs)
    _check(lib().fdf_server_get(srv, int(rid), species, ptrs[0][0], ptrs[1][0], ptrs[2][0], dev), "fdf_server_get")
    return x, q, w


def fdf_server_deposit(srv, rid, out):
    p, dev = _ptr(out)
    _check(lib().fdf_server_deposit(srv, int(rid), p, dev), "fdf_server_deposit")
    return out


def fdf_server_release(srv, rid):
    _check(lib().fdf_server_release(srv, int(rid)), "fdf_server_release")


def fdf_server_clock(srv):
    return lib().fdf_server_clock(srv)


def fdf_server_load(srv):
    q, r, b = C.c_int32(0), C.c_int32(0), C.c_size_t(0)
    _check(lib().fdf_server_load(srv, C.byref(q), C.byref(r), C.byref(b)), "fdf_server_load")
    return q.value, r.value, b.value


def fdf_server_destroy(srv):
    if srv:
        lib().fdf_server_destroy(srv)


class Run:
    """One context: ``with Run(params_dict, tables_dict) as r: r.sample(); r.step(n); x, q, w = r.get(0)``."""

    def __init__(self, params, tables, stream=None, arena=None):
        self.params = dict(params)
        self._p = make_params(self.params)
        self._t, self._keep = make_tables(tables)
        self.ctx = fdf_create(self._p, self._t, stream, arena)
        self.n_part = int(self.params["n_part"])
        self.N = int(self.params["n_grid"])

    def close(self):
        if self.ctx:
            fdf_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sample(self):
        fdf_sample(self.ctx)

    def step(self, n):
        fdf_step(self.ctx, n)

    def run_graph(self, n):
        fdf_run_graph(self.ctx, n)

    def accel_terms(self, species=-1):
        return fdf_accel_terms(self.ctx, species)

    def get(self, species=0):
        n = self.n_part
        x = np.zeros((3, n))
        q = np.zeros((3, n))
        w = np.zeros(n)
        fdf_get(self.ctx, species, x, q, w)
        return x, q, w

    def get_initial(self, species=0):
        n = self.n_part
        X = np.zeros((3, n), np.uint32)
        qs = np.zeros((3, n))
        p = np.zeros(n)
        fdf_get_initial(self.ctx, species, X, qs, p)
        return X, qs, p

    def deposit(self, species=-1, quantity=FDF_Q_W_EPS, parity=-1):
        out = np.zeros((self.N, self.N, self.N))
        fdf_deposit_subset(self.ctx, species, quantity, parity, out)
        return out

    def build_fields(self, lna):
        out = np.zeros((8, self.N, self.N, self.N))
        fdf_build_fields(self.ctx, lna, out)
        return out

    def set_fields(self, fields):
        fdf_set_fields(self.ctx, fields)

    def state(self):
        return fdf_state(self.ctx)

    def supersteps(self):
        return fdf_supersteps(self.ctx, int(self.params["n_steps"]))[0]


class Server:
    """The request server: ``with Server(budget_bytes) as s: rid = s.submit(p, t); s.wait(); s.get(rid)``."""

    def __init__(self, hbm_budget, max_active=8, slice_steps=8, merge=False):
        self.srv = fdf_server_create_opts(hbm_budget, max_active, slice_steps,
                                          FDF_SERVER_MERGE_PASSES if merge else 0)
        self.params = {}

    def close(self):
        if self.srv:
            fdf_server_destroy(self.srv)
            self.srv = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, params, tables):
        P = make_params(params)
        T, keep = make_tables(tables)
        rid = fdf_server_submit(self.srv, P, T)
        self.params[rid] = dict(params)
        return rid

    def wait(self, timeout_ms=-1):
        return fdf_server_wait(self.srv, timeout_ms)

    def info(self, rid):
        return fdf_server_info(self.srv, rid)

    def clock(self):
        return fdf_server_clock(self.srv)

    def load(self):
        return fdf_server_load(self.srv)

    def merged_launches(self):
        return fdf_server_merged_launches(self.srv)

    def get(self, rid, species=0):
        n = int(self.params[rid]["n_part"])
        x = np.zeros((3, n))
        q = np.zeros((3, n))
        w = np.zeros(n)
        fdf_server_get(self.srv, rid, species, x, q, w)
        return x, q, w

    def deposit(self, rid):
        N = int(self.params[rid]["n_grid"])
        out = np.zeros((N, N, N))
        fdf_server_deposit(self.srv, rid, out)
        return out

    def release(self, rid):
        fdf_server_release(self.srv, rid)
        self.params.pop(rid, None)
