"""Python binding of the C ABI in include/cgdem.h (argument marshalling only).

Every step of the method runs in the CUDA library ``_build/libcgdem.so``;
this module only converts arguments.  PyTorch supplies the device workspace
and the stream.  There is no CPU fallback: if the library is missing or no
GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcgdem.so")

CGDEM_OK = 0
CGDEM_E_INVALID = -1
CGDEM_E_CAPACITY = -2
CGDEM_E_CUDA = -3
CGDEM_E_NONFINITE = -4
CGDEM_E_TIMEOUT = -5
CGDEM_E_STATE = -6
MLP_NPARAMS = 8844
PSD_MAX = 16  # size classes of the produced-sand accumulators
FP64, MIXED = 0, 1
PERIODIC_BOX, CYLINDER = 0, 1
CG_NONE, CG_SSW, CG_SSP = 0, 1, 2

# every symbol that include/cgdem.h declares
EXPORTS = [
    "cgdem_rayleigh_dt", "cgdem_cg_scale_diameters", "cgdem_workspace_size", "cgdem_create",
    "cgdem_destroy", "cgdem_last_error", "cgdem_status_sync", "cgdem_init_particles",
    "cgdem_set_fluid_velocity", "cgdem_build_contacts", "cgdem_couple_fluid",
    "cgdem_compute_forces", "cgdem_integrate", "cgdem_step", "cgdem_prepare", "cgdem_fp64_math_check",
    "cgdem_get_state",
    "cgdem_get_contacts", "cgdem_get_contact_springs", "cgdem_get_voidfrac", "cgdem_get_diagnostics", "cgdem_get_removed_step", "cgdem_set_psd_classes", "cgdem_get_produced_psd", "cgdem_get_fluid",
    "cgdem_get_counters", "cgdem_get_launch_counts", "cgdem_profile_step", "cgdem_touching_pairs_noalloc",
    "cgdem_mlp_workspace_size", "cgdem_mlp_forward", "cgdem_mlp_train_step", "cgdem_mlp_status",
    "cgdem_set_closure", "cgdem_closure_record", "cgdem_get_closure_data",
    "cgdem_set_stage", "cgdem_get_boundaries", "cgdem_bond_touching",
]


class Stage(C.Structure):
    """cgdem_stage: contact model and moving boundaries of a preparation stage."""
    _fields_ = [
        ("jkr_mode", C.c_int),
        ("plate_mode", C.c_int), ("plate_H", C.c_double), ("plate_stress", C.c_double),
        ("plate_gain", C.c_double), ("plate_vmax", C.c_double),
        ("pen_mode", C.c_int), ("pen_radius", C.c_double), ("pen_speed", C.c_double),
        ("pen_z_start", C.c_double), ("pen_z_stop", C.c_double), ("pen_force", C.c_double),
        ("outlet_closed", C.c_int),
    ]


def stage(**kw) -> Stage:
    """A Stage from keyword arguments (missing ones are zero)."""
    st = Stage()
    for k, v in kw.items():
        setattr(st, k, v)
    return st


class CgdemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cgdem error {code}: {msg}")
        self.code = code


class SampleParams(C.Structure):
    _fields_ = [
        ("rho", C.c_double), ("E", C.c_double), ("nu", C.c_double), ("e", C.c_double),
        ("mu", C.c_double), ("gamma", C.c_double),
        ("k_cg", C.c_double), ("cg_scheme", C.c_int),
        ("rho_f", C.c_double), ("mu_f", C.c_double),
        ("use_drag", C.c_int), ("use_buoyancy", C.c_int),
        ("kind", C.c_int), ("L", C.c_double * 3), ("Rc", C.c_double), ("H", C.c_double),
        ("r_out", C.c_double), ("g", C.c_double * 3), ("dt", C.c_double),
        ("coulomb_mode", C.c_int),
        ("nf", C.c_int * 3), ("f_lo", C.c_double * 3), ("hf", C.c_double * 3),
        ("inv_hf", C.c_double * 3), ("V_cell", C.c_double), ("n_min", C.c_double),
        ("vf_mode", C.c_int), ("couple_every", C.c_int), ("skin", C.c_double),
        ("r_max", C.c_double),
        ("fluid_mode", C.c_int), ("p_inlet", C.c_double), ("perm_d", C.c_double),
        ("jkr_mode", C.c_int),
    ]


class Config(C.Structure):
    _fields_ = [
        ("precision", C.c_int), ("n_samples", C.c_int), ("max_neighbors", C.c_int),
        ("block_size", C.c_int), ("cell_scale", C.c_double), ("steps_per_graph", C.c_int),
        ("closure", C.c_int), ("particles_per_warp", C.c_int),
        ("fluid_iters", C.c_int), ("fluid_tol", C.c_double), ("fluid_kernels", C.c_int),
    ]


class ClosureParams(C.Structure):
    _fields_ = [("lo", C.c_float * 5), ("hi", C.c_float * 5), ("cd_log_max", C.c_float),
                ("cg_log_max", C.c_float)]


CL_COLS = 12


_lib = None


def lib():
    """Load libcgdem.so (build it first with build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        vp, i, i64, d = C.c_void_p, C.c_int, C.c_int64, C.c_double
        sig = {
            "cgdem_rayleigh_dt": (d, [d, d, d, d]),
            "cgdem_cg_scale_diameters": (i, [vp, i64, d, i, vp, vp]),
            "cgdem_workspace_size": (i, [vp, vp, vp, vp]),
            "cgdem_create": (i, [vp, vp, vp, vp, C.c_size_t, vp]),
            "cgdem_destroy": (None, [vp]),
            "cgdem_last_error": (C.c_char_p, [vp]),
            "cgdem_status_sync": (i, [vp, vp]),
            "cgdem_init_particles": (i, [vp, vp, vp, vp, vp, i, vp]),
            "cgdem_set_fluid_velocity": (i, [vp, vp, vp]),
            "cgdem_build_contacts": (i, [vp, vp]),
            "cgdem_couple_fluid": (i, [vp, vp]),
            "cgdem_compute_forces": (i, [vp, vp]),
            "cgdem_integrate": (i, [vp, i, vp]),
            "cgdem_step": (i, [vp, i64, vp]),
            "cgdem_prepare": (i, [vp, vp]),
            "cgdem_fp64_math_check": (i, [vp, i64, vp, vp]),
            "cgdem_get_state": (i, [vp, vp, vp, vp, vp, vp, vp]),
            "cgdem_get_contacts": (i, [vp, vp, vp, vp, i64, vp, vp]),
            "cgdem_get_contact_springs": (i, [vp, vp, vp, vp, i64, vp, vp]),
            "cgdem_get_voidfrac": (i, [vp, vp, i64, vp]),
            "cgdem_get_diagnostics": (i, [vp, vp, i64, vp]),
            "cgdem_get_removed_step": (i, [vp, vp, vp]),
            "cgdem_set_psd_classes": (i, [vp, vp, i, vp]),
            "cgdem_set_stage": (i, [vp, i, vp, vp]),
            "cgdem_bond_touching": (i, [vp, vp]),
            "cgdem_get_boundaries": (i, [vp, vp, i64, vp]),
            "cgdem_get_fluid": (i, [vp, vp, vp, vp, vp, vp, vp]),
            "cgdem_get_produced_psd": (i, [vp, vp, vp, i64, vp]),
            "cgdem_get_counters": (i, [vp, vp, vp, vp, vp, vp]),
            "cgdem_get_launch_counts": (i, [vp, vp, vp]),
            "cgdem_profile_step": (i, [vp, i64, vp, vp]),
            "cgdem_touching_pairs_noalloc": (i, [vp, vp, i64, vp, vp, i, d, d, vp, i64, vp, vp]),
            "cgdem_mlp_workspace_size": (i, [vp]),
            "cgdem_mlp_forward": (i, [vp, vp, i64, vp, vp, C.c_size_t, vp]),
            "cgdem_mlp_train_step": (i, [vp, vp, vp, i64, d, vp, vp, vp, i64, vp, vp, vp, C.c_size_t,
                                         vp]),
            "cgdem_mlp_status": (i, [vp, vp]),
            "cgdem_set_closure": (i, [vp, vp, vp, i, vp]),
            "cgdem_closure_record": (i, [vp, i, vp]),
            "cgdem_get_closure_data": (i, [vp, vp, i64, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data if a is not None else None


# ---- host-only helpers ----

def cgdem_rayleigh_dt(Rbar, rho, E, nu):
    return lib().cgdem_rayleigh_dt(Rbar, rho, E, nu)


def cgdem_cg_scale_diameters(d_fine, k, scheme):
    d_fine = np.ascontiguousarray(d_fine, dtype=np.float64)
    out = np.zeros(max(len(d_fine), 1))
    n = C.c_int64(0)
    r = lib().cgdem_cg_scale_diameters(_ptr(d_fine), len(d_fine), float(k), int(scheme), _ptr(out),
                                       C.byref(n))
    if r:
        raise CgdemError(r, "cg_scale_diameters")
    return out[: n.value].copy()


def fp64_math_check(x):
    """The FP64 step's reciprocal and cube root beside CUDA's, on the GPU:
    returns (nr_rcp(x), 1/x, nr_cbrt(|x|), cbrt(|x|)) as numpy arrays."""
    import torch

    xd = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")
    out = torch.empty(4 * xd.numel(), dtype=torch.float64, device="cuda")
    r = lib().cgdem_fp64_math_check(C.c_void_p(xd.data_ptr()), xd.numel(), C.c_void_p(out.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if r:
        raise CgdemError(r, "fp64_math_check")
    o = out.view(-1, 4).cpu().numpy()
    return o[:, 0], o[:, 1], o[:, 2], o[:, 3]


def cgdem_touching_pairs_noalloc(x_dev, R_dev, n, box_lo, box_hi, periodic, r_max, skin,
                                 pairs_dev, cap, count_dev, stream=None):
    """Pair search that allocates no device memory (device pointers in and out)."""
    lo = np.ascontiguousarray(box_lo, dtype=np.float64)
    hi = np.ascontiguousarray(box_hi, dtype=np.float64)
    r = lib().cgdem_touching_pairs_noalloc(C.c_void_p(x_dev), C.c_void_p(R_dev), int(n), _ptr(lo),
                                           _ptr(hi), int(periodic), float(r_max), float(skin),
                                           C.c_void_p(pairs_dev), int(cap), C.c_void_p(count_dev),
                                           C.c_void_p(stream))
    if r:
        raise CgdemError(r, "touching_pairs_noalloc")


def cgdem_mlp_workspace_size():
    n = C.c_size_t(0)
    r = lib().cgdem_mlp_workspace_size(C.byref(n))
    if r:
        raise CgdemError(r, "mlp_workspace_size")
    return n.value


def cgdem_mlp_forward(theta_dev, X_dev, n, out_dev, ws_dev, ws_bytes, stream=None):
    r = lib().cgdem_mlp_forward(C.c_void_p(theta_dev), C.c_void_p(X_dev), int(n), C.c_void_p(out_dev),
                                C.c_void_p(ws_dev), int(ws_bytes), C.c_void_p(stream))
    if r:
        raise CgdemError(r, "mlp_forward")


def cgdem_mlp_train_step(theta_dev, m_dev, v_dev, t, lr, X_dev, Y_dev, M_dev, n, grad_dev, loss_dev,
                         ws_dev, ws_bytes, stream=None):
    r = lib().cgdem_mlp_train_step(C.c_void_p(theta_dev), C.c_void_p(m_dev), C.c_void_p(v_dev), int(t),
                                   float(lr), C.c_void_p(X_dev), C.c_void_p(Y_dev), C.c_void_p(M_dev),
                                   int(n), C.c_void_p(grad_dev), C.c_void_p(loss_dev), C.c_void_p(ws_dev),
                                   int(ws_bytes), C.c_void_p(stream))
    if r:
        raise CgdemError(r, "mlp_train_step")


def cgdem_mlp_status(ws_dev, stream=None):
    r = lib().cgdem_mlp_status(C.c_void_p(ws_dev), C.c_void_p(stream))
    if r:
        raise CgdemError(r, "mlp kernel")


class Closure:
    """The closure network on one GPU: FP32 parameters, Adam moments and the
    kernels' workspace as torch tensors; every computation runs in the
    library's tensor-core kernels."""

    def __init__(self, theta, device="cuda:0"):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("cgdem needs a CUDA GPU")
        self.torch = torch
        self.device = torch.device(device)
        theta = np.asarray(theta, dtype=np.float32)
        if theta.shape != (MLP_NPARAMS,):
            raise ValueError("theta must hold %d floats" % MLP_NPARAMS)
        self.theta = torch.tensor(theta, device=self.device)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.t = 0
        self.ws_bytes = cgdem_mlp_workspace_size()
        self.ws = torch.zeros(self.ws_bytes // 4 + 1, dtype=torch.float32, device=self.device)
        self.grad = torch.zeros_like(self.theta)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)

    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def _dev(self, a, cols):
        t = self.torch
        if isinstance(a, t.Tensor):
            a = a.to(device=self.device, dtype=t.float32).contiguous()
        else:
            a = t.tensor(np.ascontiguousarray(a, dtype=np.float32), device=self.device)
        return a.reshape(-1, cols)

    def forward(self, X):
        X = self._dev(X, 5)
        out = self.torch.empty((len(X), 2), dtype=self.torch.float32, device=self.device)
        cgdem_mlp_forward(self.theta.data_ptr(), X.data_ptr(), len(X), out.data_ptr(), self.ws.data_ptr(),
                          self.ws_bytes, self._stream())
        cgdem_mlp_status(self.ws.data_ptr(), self._stream())
        return out

    def gradient(self, X, Y, M):
        X, Y, M = self._dev(X, 5), self._dev(Y, 2), self._dev(M, 2)
        cgdem_mlp_train_step(self.theta.data_ptr(), None, None, 0, 0.0, X.data_ptr(), Y.data_ptr(),
                             M.data_ptr(), len(X), self.grad.data_ptr(), self.loss.data_ptr(),
                             self.ws.data_ptr(), self.ws_bytes, self._stream())
        cgdem_mlp_status(self.ws.data_ptr(), self._stream())
        return float(self.loss.item()), self.grad.clone()

    def train(self, X, Y, M, steps, lr, check_every=50):
        """`steps` full-batch Adam steps; returns the loss before each step."""
        X, Y, M = self._dev(X, 5), self._dev(Y, 2), self._dev(M, 2)
        hist = self.torch.zeros(steps, dtype=self.torch.float32, device=self.device)
        for k in range(steps):
            self.t += 1
            cgdem_mlp_train_step(self.theta.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.t, lr,
                                 X.data_ptr(), Y.data_ptr(), M.data_ptr(), len(X), None,
                                 hist[k:].data_ptr(), self.ws.data_ptr(), self.ws_bytes, self._stream())
            if (k + 1) % check_every == 0 or k + 1 == steps:
                cgdem_mlp_status(self.ws.data_ptr(), self._stream())
        return hist.cpu().numpy()

    def params(self):
        return self.theta.cpu().numpy()


def spheres_per_warp_for(n, device="cuda:0"):
    """Spheres per warp of the force kernel for a context of n spheres run
    without the autotuner: 16 when 32 per warp would leave the GPU with fewer
    than two blocks of 128 threads per SM (the step is then bound by one
    warp's chain of rounds; on the 25,000-parcel coarse cylinder 16 per warp
    is 16 % faster), else 32."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    return 16 if n < 2 * 128 * sms else 32


def sample_params(s, dt, skin, k=1.0, scheme=CG_NONE, use_drag=1, use_buoyancy=1,
                  coulomb_mode=0, vf_mode=0, couple_every=1, n_min=0.2, r_max=None,
                  gamma_fine=None, fluid_mode=0, p_inlet=0.0, perm_d=None, jkr_mode=0) -> SampleParams:
    """SampleParams from an inputs.Sample-like object (material at fine scale)."""
    p = SampleParams()
    m = s.material
    p.rho, p.E, p.nu, p.e, p.mu = m["rho"], m["E"], m["nu"], m["e"], m["mu"]
    p.gamma = m["gamma"] if gamma_fine is None else gamma_fine
    p.k_cg, p.cg_scheme = float(k), int(scheme)
    p.rho_f, p.mu_f = s.fluid["rho_f"], s.fluid["mu_f"]
    p.use_drag, p.use_buoyancy = int(use_drag), int(use_buoyancy)
    dom = s.domain
    p.kind = int(dom["kind"])
    for i in range(3):
        p.L[i] = dom["L"][i]
        p.g[i] = s.g[i]
        p.nf[i] = s.grid.nf[i]
        p.f_lo[i] = s.grid.lo[i]
        p.hf[i] = s.grid.h[i]
        p.inv_hf[i] = s.grid.inv_h[i]
    p.Rc, p.H, p.r_out = dom["Rc"], dom["H"], dom["r_out"]
    p.dt = float(dt)
    p.coulomb_mode = int(coulomb_mode)
    p.V_cell = s.grid.V_cell
    p.n_min = n_min
    p.vf_mode = int(vf_mode)
    p.couple_every = int(couple_every)
    p.skin = float(skin)
    p.r_max = float(r_max if r_max is not None else np.max(s.R))
    p.fluid_mode = int(fluid_mode)
    p.p_inlet = float(p_inlet)
    # Kozeny-Carman diameter: the volume-mean grain diameter unless given
    p.perm_d = float(perm_d if perm_d is not None else np.mean((2 * np.asarray(s.R)) ** 3) ** (1 / 3))
    p.jkr_mode = int(jkr_mode)
    return p


class Context:
    """A library context over one or more samples on one GPU."""

    def __init__(self, params, counts, precision=MIXED, max_neighbors=48, block_size=128,
                 cell_scale=0.0, steps_per_graph=32, device="cuda:0", stream=None, closure=False,
                 particles_per_warp=32, fluid_iters=0, fluid_tol=0.0, fluid_kernels=0, prepare=True):
        """prepare: capture the step graphs on the context's stream now
        (cgdem_prepare), so that the first step() replays them."""
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("cgdem needs a CUDA GPU")
        self.torch = torch
        self.device = torch.device(device)
        self.n_samples = len(params)
        self._params = (SampleParams * self.n_samples)(*params)
        self.counts = np.ascontiguousarray(counts, dtype=np.int64)
        self.N = int(self.counts.sum())
        self.cfg = Config(precision, self.n_samples, max_neighbors, block_size, cell_scale,
                          steps_per_graph, int(bool(closure)), int(particles_per_warp), int(fluid_iters),
                          float(fluid_tol), int(fluid_kernels))
        nbytes = C.c_size_t(0)
        r = lib().cgdem_workspace_size(C.byref(self.cfg), self._params, _ptr(self.counts),
                                       C.byref(nbytes))
        if r:
            raise CgdemError(r, "workspace_size: invalid configuration")
        self.workspace_bytes = nbytes.value
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8,
                                         device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        h = C.c_void_p()
        r = lib().cgdem_create(C.byref(self.cfg), self._params, _ptr(self.counts),
                               C.c_void_p(aligned), self.workspace_bytes, C.byref(h))
        if r:
            raise CgdemError(r, "create failed")
        self.h = h
        self.stream = stream
        if prepare:
            self.prepare()

    def _s(self):
        if self.stream is not None:
            return C.c_void_p(self.stream)
        return C.c_void_p(self.torch.cuda.current_stream(self.device).cuda_stream)

    def _check(self, r, what):
        if r != CGDEM_OK:
            msg = lib().cgdem_last_error(self.h)
            raise CgdemError(r, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            lib().cgdem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- verbs ----
    def init_particles(self, x, v, w, R, bond_touching=True):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1, 3)
        R = np.ascontiguousarray(R, dtype=np.float64).reshape(-1)
        if len(R) != self.N:
            raise ValueError("particle count mismatch")
        self._check(lib().cgdem_init_particles(self.h, _ptr(x), _ptr(v), _ptr(w), _ptr(R),
                                               int(bond_touching), self._s()), "init_particles")

    def set_fluid_velocity(self, Us):
        Us = np.ascontiguousarray(Us, dtype=np.float64).reshape(-1, 3)
        self._check(lib().cgdem_set_fluid_velocity(self.h, _ptr(Us), self._s()), "set_fluid_velocity")

    def build_contacts(self):
        self._check(lib().cgdem_build_contacts(self.h, self._s()), "build_contacts")

    def couple_fluid(self):
        self._check(lib().cgdem_couple_fluid(self.h, self._s()), "couple_fluid")

    def compute_forces(self):
        self._check(lib().cgdem_compute_forces(self.h, self._s()), "compute_forces")

    def integrate(self, half):
        self._check(lib().cgdem_integrate(self.h, int(half), self._s()), "integrate")

    def step(self, n=1):
        self._check(lib().cgdem_step(self.h, int(n), self._s()), "step")

    def prepare(self):
        """Capture and upload the step graphs on the context's stream."""
        self._check(lib().cgdem_prepare(self.h, self._s()), "prepare")

    # ---- readback ----
    def get_state(self, out=None):
        """x, v, w, F, T in id order.  out: a dict of five (N, 3) float64
        C-contiguous arrays to fill (pinned host memory makes the copies
        several times faster than fresh pageable arrays)."""
        keys = ["x", "v", "w", "F", "T"]
        if out is None:
            arrs = [np.zeros((self.N, 3)) for _ in keys]
        else:
            arrs = [out[k] for k in keys]
            for a in arrs:
                if a.dtype != np.float64 or a.shape != (self.N, 3) or not a.flags["C_CONTIGUOUS"]:
                    raise ValueError("get_state: out arrays must be float64, C-contiguous, of shape (N, 3)")
        self._check(lib().cgdem_get_state(self.h, *[_ptr(a) for a in arrs], self._s()), "get_state")
        return dict(zip(keys, arrs))

    def get_contacts(self):
        n = C.c_int64(0)
        self._check(lib().cgdem_get_contacts(self.h, None, None, None, 0, C.byref(n), self._s()),
                    "get_contacts")
        cap = max(n.value, 1)
        i = np.zeros(cap, np.int32)
        j = np.zeros(cap, np.int32)
        b = np.zeros(cap, np.uint8)
        self._check(lib().cgdem_get_contacts(self.h, _ptr(i), _ptr(j), _ptr(b), cap, C.byref(n),
                                             self._s()), "get_contacts")
        k = n.value
        return i[:k], j[:k], b[:k]

    def get_contact_springs(self):
        """(id_i, id_j, xi [n,3]) of the active contacts, xi as seen from id_i."""
        n = C.c_int64(0)
        self._check(lib().cgdem_get_contact_springs(self.h, None, None, None, 0, C.byref(n), self._s()),
                    "get_contact_springs")
        cap = max(n.value, 1)
        i = np.zeros(cap, np.int32)
        j = np.zeros(cap, np.int32)
        xi = np.zeros((cap, 3))
        self._check(lib().cgdem_get_contact_springs(self.h, _ptr(i), _ptr(j), _ptr(xi), cap, C.byref(n),
                                                    self._s()), "get_contact_springs")
        k = n.value
        return i[:k], j[:k], xi[:k]

    def get_voidfrac(self, ncell):
        out = np.zeros(ncell, np.uint64)
        self._check(lib().cgdem_get_voidfrac(self.h, _ptr(out), ncell, self._s()), "get_voidfrac")
        return out

    def get_diagnostics(self):
        out = np.zeros((self.n_samples, 8))
        self._check(lib().cgdem_get_diagnostics(self.h, _ptr(out), out.size, self._s()),
                    "get_diagnostics")
        keys = ["ke", "ke_rot", "px", "py", "pz", "produced_mass", "n_active", "n_bonds"]
        return [dict(zip(keys, row)) for row in out]

    def get_removed_step(self):
        out = np.zeros(self.N, np.int32)
        self._check(lib().cgdem_get_removed_step(self.h, _ptr(out), self._s()), "get_removed_step")
        return out

    def get_fluid(self, ncell):
        """(pressure [Cf], superficial velocity [Cf,3], pressure gradient
        [Cf,3], drag reaction [Cf,3] in 2^-60 N quanta, iterations of the last
        solve) of the Darcy samples."""
        p, U, g = np.zeros(ncell), np.zeros((ncell, 3)), np.zeros((ncell, 3))
        r = np.zeros((ncell, 3), np.int64)
        it = C.c_int64(0)
        self._check(lib().cgdem_get_fluid(self.h, _ptr(p), _ptr(U), _ptr(g), _ptr(r), C.byref(it), self._s()),
                    "get_fluid")
        return p, U, g, r, it.value

    def bond_touching(self):
        """Bond every pair that touches now, keeping the other contacts and all springs."""
        self._check(lib().cgdem_bond_touching(self.h, self._s()), "bond_touching")

    def set_stage(self, sample, st: Stage):
        """Start a preparation stage on one cylinder sample (cgdem_set_stage)."""
        self._check(lib().cgdem_set_stage(self.h, int(sample), C.byref(st), self._s()), "set_stage")

    def boundaries(self):
        """Per sample: top-plate height, its velocity, the stress on it, the
        penetrometer tip's height and direction, the force along z on it."""
        out = np.zeros(6 * self.n_samples)
        self._check(lib().cgdem_get_boundaries(self.h, _ptr(out), out.size, self._s()), "get_boundaries")
        return [dict(H=o[0], v_plate=o[1], stress=o[2], pen_z=o[3], pen_dir=int(o[4]), pen_force=o[5])
                for o in out.reshape(-1, 6)]

    def set_psd_classes(self, edges):
        """Record produced sand by size class (fine-scale diameter edges [m])."""
        e = np.ascontiguousarray(edges, dtype=np.float64)
        self._check(lib().cgdem_set_psd_classes(self.h, _ptr(e), len(e) - 1, self._s()), "set_psd_classes")

    def produced_psd(self):
        """(mass [n_samples, 16] kg, count [n_samples, 16]) produced so far."""
        m = np.zeros((self.n_samples, PSD_MAX))
        c = np.zeros((self.n_samples, PSD_MAX), np.int64)
        self._check(lib().cgdem_get_produced_psd(self.h, _ptr(m), _ptr(c), m.size, self._s()),
                    "get_produced_psd")
        return m, c

    def counters(self):
        s, r, m, t = C.c_int64(0), C.c_int64(0), C.c_int32(0), C.c_int64(0)
        self._check(lib().cgdem_get_counters(self.h, C.byref(s), C.byref(r), C.byref(m), C.byref(t),
                                             self._s()), "get_counters")
        return dict(steps=s.value, rebuilds=r.value, max_candidates=m.value, total_candidates=t.value)

    def launch_counts(self):
        """(kernels cgdem_step launched unconditionally so far, kernels of one
        conditional rebuild sequence)."""
        k, b = C.c_int64(0), C.c_int32(0)
        self._check(lib().cgdem_get_launch_counts(self.h, C.byref(k), C.byref(b)), "get_launch_counts")
        return k.value, b.value

    # ---- learned closure ----
    def set_closure(self, theta=None, lo=None, hi=None, cd_log_max=3.0, cg_log_max=1.386,
                    enable=True):
        """Enable the closure with parameters theta (array or tensor of
        MLP_NPARAMS floats) and input range [lo, hi], or disable it."""
        t = self.torch
        if enable:
            th = t.as_tensor(np.asarray(theta, dtype=np.float32) if not isinstance(theta, t.Tensor)
                             else theta, dtype=t.float32, device=self.device).contiguous()
            if th.numel() != MLP_NPARAMS:
                raise ValueError("theta must hold %d floats" % MLP_NPARAMS)
            self._closure_theta = th  # kept alive until the copy on the stream has run
            cp = ClosureParams((C.c_float * 5)(*lo), (C.c_float * 5)(*hi), cd_log_max, cg_log_max)
            self._check(lib().cgdem_set_closure(self.h, C.c_void_p(th.data_ptr()), C.byref(cp), 1,
                                                self._s()), "set_closure")
        else:
            self._check(lib().cgdem_set_closure(self.h, None, None, 0, self._s()), "set_closure")

    def closure_record(self, enable=True):
        self._check(lib().cgdem_closure_record(self.h, int(bool(enable)), self._s()), "closure_record")

    def closure_data(self):
        """[N, 12] rows recorded by the last force evaluation (see include/cgdem.h)."""
        out = np.zeros((self.N, CL_COLS), np.float32)
        self._check(lib().cgdem_get_closure_data(self.h, _ptr(out), self.N, self._s()),
                    "get_closure_data")
        return out

    def profile_step(self, n):
        out = np.zeros(6)
        self._check(lib().cgdem_profile_step(self.h, int(n), _ptr(out), self._s()), "profile_step")
        return dict(force_ms=out[0], rebuild_ms_total=out[1], rebuilds=int(out[2]), total_ms=out[3],
                    steps=int(out[4]), rebuild_floor_ms=out[5])

    def status(self):
        return lib().cgdem_status_sync(self.h, self._s())
