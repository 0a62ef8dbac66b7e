"""ctypes binding of the FP64 C oracle (test infrastructure only).

Every function here restates the paper (arXiv 2211.06142) in plain C; see
``cgdem_oracle.c`` for the equation each part follows.  Nothing in the CUDA
package imports this module.
"""
import ctypes as C
import numpy as np

from .build import build

_lib = None


class OraParams(C.Structure):
    _fields_ = [
        ("rho", C.c_double), ("E", C.c_double), ("nu", C.c_double), ("e", C.c_double),
        ("mu", C.c_double), ("gamma", C.c_double),
        ("rho_f", C.c_double), ("mu_f", C.c_double),
        ("use_drag", C.c_int), ("use_buoyancy", C.c_int),
        ("kind", C.c_int),
        ("L", C.c_double * 3),
        ("Rc", C.c_double), ("H", C.c_double), ("r_out", C.c_double),
        ("g", C.c_double * 3),
        ("dt", C.c_double),
        ("coulomb_mode", C.c_int),
        ("nf", C.c_int * 3),
        ("f_lo", C.c_double * 3), ("hf", C.c_double * 3), ("inv_hf", C.c_double * 3),
        ("V_cell", C.c_double), ("n_min", C.c_double),
        ("vf_mode", C.c_int), ("couple_every", C.c_int),
        ("fluid_mode", C.c_int), ("p_inlet", C.c_double), ("perm_d", C.c_double), ("n_cap", C.c_double),
        ("jkr_mode", C.c_int),
    ]


class OraStage(C.Structure):
    _fields_ = [
        ("jkr_mode", C.c_int),
        ("plate_mode", C.c_int), ("plate_H", C.c_double), ("plate_stress", C.c_double),
        ("plate_gain", C.c_double), ("plate_vmax", C.c_double),
        ("pen_mode", C.c_int), ("pen_radius", C.c_double), ("pen_speed", C.c_double),
        ("pen_z_start", C.c_double), ("pen_z_stop", C.c_double), ("pen_force", C.c_double),
        ("outlet_closed", C.c_int),
    ]


def make_stage(**kw) -> OraStage:
    """A preparation stage from keyword arguments (missing ones are zero)."""
    st = OraStage()
    for k, v in kw.items():
        setattr(st, k, v)
    return st


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        d, i, i64, vp = C.c_double, C.c_int, C.c_int64, C.c_void_p
        pd = C.POINTER(C.c_double)
        for name, res, args in [
            ("ora_estar", d, [d, d]),
            ("ora_beta", d, [d]),
            ("ora_jkr_contact_radius", d, [d, d, d, d]),
            ("ora_jkr_force", d, [d, d, d, d]),
            ("ora_jkr_overlap", d, [d, d, d, d]),
            ("ora_delta_c", d, [d, d, d]),
            ("ora_bond_breaks", i, [d, d, d, d]),
            ("ora_delta_s", d, [d, d, d]),
            ("ora_contact_separates", i, [d, d, d, d]),
            ("ora_jkr_contact_radius_s", d, [d, d, d, d]),
            ("ora_set_stage", i, [vp, vp]),
            ("ora_tool_overlap", d, [pd, d, d, d, pd]),
            ("ora_get_boundaries", i, [vp, pd]),
            ("ora_rayleigh_dt", d, [d, d, d, d]),
            ("ora_pair_contact", i, [vp, pd, pd, pd, d, d, pd, pd, pd, d, d, pd, C.POINTER(C.c_int), pd]),
            ("ora_drag", None, [d, d, d, pd, pd, d, pd]),
            ("ora_create", vp, [vp, i64, pd, pd, pd, pd, pd]),
            ("ora_destroy", None, [vp]),
            ("ora_bond_touching", i, [vp]),
            ("ora_couple_fluid", i, [vp]),
            ("ora_compute_forces", i, [vp]),
            ("ora_step", i, [vp, i64]),
            ("ora_get_state", i, [vp, pd, pd, pd, pd, pd]),
            ("ora_set_forces", i, [vp, pd, pd]),
            ("ora_num_contacts", i64, [vp]),
            ("ora_get_contacts", i, [vp, vp, vp, vp, vp, i64]),
            ("ora_get_voidfrac", i, [vp, vp]),
            ("ora_get_diagnostics", i, [vp, pd]),
            ("ora_get_removed_step", i, [vp, vp]),
            ("ora_get_force_scale", i, [vp, vp]),
            ("ora_get_force_scale_net", i, [vp, vp]),
            ("ora_set_threads", i, [i]),
            ("ora_darcy_solve", i, [i, i, i, pd, d, vp, vp, vp, d, vp, d, i]),
            ("ora_darcy_velocity", i, [i, i, i, pd, d, vp, vp, vp, d, vp, vp]),
            ("ora_get_fluid", i, [vp, vp, vp, vp, vp]),
            ("ora_get_reaction", i, [vp, vp]),
            ("ora_pairs_bruteforce", i64, [vp, i64, pd, pd, d, vp, vp, i64]),
            ("ora_voidfrac", i, [vp, i64, pd, pd, vp]),
            ("ora_set_closure", i, [vp, i, d]),
            ("ora_set_corrections", i, [vp, pd, pd]),
            ("ora_get_closure_data", i, [vp, pd]),
        ]:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _pd(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def make_params(**kw) -> OraParams:
    """Build an OraParams from keyword arguments (missing ones are zero)."""
    p = OraParams()
    for k, v in kw.items():
        f = getattr(p, k)
        if isinstance(f, C.Array):
            for i, x in enumerate(v):
                f[i] = x
        else:
            setattr(p, k, v)
    if "couple_every" not in kw:
        p.couple_every = 1
    if "n_cap" not in kw:
        p.n_cap = 0.95
    return p


# ---- closed forms and single-contact laws ----

def estar(E, nu):
    return lib().ora_estar(E, nu)


def beta(e):
    return lib().ora_beta(e)


def jkr_contact_radius(delta, Rs, Es, gamma):
    return lib().ora_jkr_contact_radius(delta, Rs, Es, gamma)


def jkr_force(a, Rs, Es, gamma):
    return lib().ora_jkr_force(a, Rs, Es, gamma)


def jkr_overlap(a, Rs, Es, gamma):
    return lib().ora_jkr_overlap(a, Rs, Es, gamma)


def delta_c(Rs, Es, gamma):
    return lib().ora_delta_c(Rs, Es, gamma)


def delta_s(Rs, Es, gamma):
    return lib().ora_delta_s(Rs, Es, gamma)


def contact_separates(delta, Rs, Es, gamma):
    return bool(lib().ora_contact_separates(delta, Rs, Es, gamma))


def jkr_contact_radius_s(delta, Rs, Es, gamma):
    return lib().ora_jkr_contact_radius_s(delta, Rs, Es, gamma)


def tool_overlap(x, R, rp, zt):
    """Overlap with the penetrometer and the unit vector towards it."""
    x = _f64(x, (3,))
    n = np.zeros(3)
    return lib().ora_tool_overlap(_pd(x), R, rp, zt, _pd(n)), n


def bond_breaks(delta, Rs, Es, gamma):
    return bool(lib().ora_bond_breaks(delta, Rs, Es, gamma))


def rayleigh_dt(Rbar, rho, E, nu):
    return lib().ora_rayleigh_dt(Rbar, rho, E, nu)


def pair_contact(p, xi, vi, wi, Ri, mi, xj, vj, wj, Rj, mj, hist=None, bonded=False):
    """One contact in isolation. Returns (active, Fi, Ti, Tj, Fne, a, delta, hist, bonded)."""
    h = np.zeros(3) if hist is None else np.array(hist, dtype=np.float64)
    b = C.c_int(1 if bonded else 0)
    out = np.zeros(12)
    args = [_f64(t, 3) for t in (xi, vi, wi)]
    argj = [_f64(t, 3) for t in (xj, vj, wj)]
    act = lib().ora_pair_contact(C.byref(p), _pd(args[0]), _pd(args[1]), _pd(args[2]), Ri, mi,
                                 _pd(argj[0]), _pd(argj[1]), _pd(argj[2]), Rj, mj, _pd(h),
                                 C.byref(b), _pd(out))
    return bool(act), out[0:3].copy(), out[3:6].copy(), out[6:9].copy(), out[9], out[10], out[11], h, bool(b.value)


def drag(rho_f, mu_f, d, u, v, n):
    f = np.zeros(3)
    uu, vv = _f64(u, 3), _f64(v, 3)
    lib().ora_drag(rho_f, mu_f, d, _pd(uu), _pd(vv), n, _pd(f))
    return f


def darcy_solve(nf, h, mu, K, ctype, outlet, p_out, p0, tol=1e-13, max_iter=100000):
    """Pressures of a Darcy flow on a grid (see ora_darcy_solve); returns (p, iterations)."""
    nx, ny, nz = (int(v) for v in nf)
    hh = _f64(h, 3)
    K = np.ascontiguousarray(K, dtype=np.float64).reshape(-1)
    t = np.ascontiguousarray(ctype, dtype=np.int8).reshape(-1)
    o = np.ascontiguousarray(outlet, dtype=np.uint8).reshape(-1)
    p = np.array(p0, dtype=np.float64).reshape(-1)
    it = lib().ora_darcy_solve(nx, ny, nz, _pd(hh), mu, K.ctypes.data, t.ctypes.data, o.ctypes.data,
                               p_out, p.ctypes.data, tol, max_iter)
    return p, it


def darcy_velocity(nf, h, mu, K, ctype, outlet, p_out, p):
    nx, ny, nz = (int(v) for v in nf)
    hh = _f64(h, 3)
    K = np.ascontiguousarray(K, dtype=np.float64).reshape(-1)
    t = np.ascontiguousarray(ctype, dtype=np.int8).reshape(-1)
    o = np.ascontiguousarray(outlet, dtype=np.uint8).reshape(-1)
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(-1)
    U = np.zeros((len(p), 3))
    lib().ora_darcy_velocity(nx, ny, nz, _pd(hh), mu, K.ctypes.data, t.ctypes.data, o.ctypes.data,
                             p_out, p.ctypes.data, U.ctypes.data)
    return U


def set_threads(n):
    """Host threads the oracle's loops use (results do not depend on it);
    returns the number in use."""
    return lib().ora_set_threads(int(n))


def pairs_bruteforce(p, x, R, skin):
    x = _f64(x, (-1, 3))
    R = _f64(R)
    n = len(R)
    cnt = lib().ora_pairs_bruteforce(C.byref(p), n, _pd(x), _pd(R), skin, None, None, 0)
    pi = np.zeros(max(cnt, 1), np.int32)
    pj = np.zeros(max(cnt, 1), np.int32)
    lib().ora_pairs_bruteforce(C.byref(p), n, _pd(x), _pd(R), skin, pi.ctypes.data, pj.ctypes.data, cnt)
    return pi[:cnt], pj[:cnt]


def voidfrac(p, x, R):
    x = _f64(x, (-1, 3))
    R = _f64(R)
    nc = p.nf[0] * p.nf[1] * p.nf[2]
    out = np.zeros(nc, np.uint64)
    lib().ora_voidfrac(C.byref(p), len(R), _pd(x), _pd(R), out.ctypes.data)
    return out


class Sim:
    """One sample simulated by the oracle."""

    def __init__(self, p: OraParams, x, v, w, R, Us=None):
        self.p = p
        self.x = _f64(x, (-1, 3))
        self.n = self.x.shape[0]
        v = _f64(v, (-1, 3))
        w = _f64(w, (-1, 3))
        R = _f64(R)
        nc = p.nf[0] * p.nf[1] * p.nf[2]
        Us = np.zeros((max(nc, 1), 3)) if Us is None else _f64(Us, (-1, 3))
        self._keep = (self.x, v, w, R, Us)
        self.h = lib().ora_create(C.byref(p), self.n, _pd(self.x), _pd(v), _pd(w), _pd(R), _pd(Us))
        if not self.h:
            raise RuntimeError("ora_create failed")
        self.ncell = nc

    def __del__(self):
        if getattr(self, "h", None):
            lib().ora_destroy(self.h)
            self.h = None

    def bond_touching(self):
        lib().ora_bond_touching(self.h)

    def couple_fluid(self):
        lib().ora_couple_fluid(self.h)

    def compute_forces(self):
        lib().ora_compute_forces(self.h)

    def step(self, n=1):
        lib().ora_step(self.h, n)

    def set_forces(self, F, T):
        F = _f64(F, (-1, 3))
        T = _f64(T, (-1, 3))
        lib().ora_set_forces(self.h, _pd(F), _pd(T))

    def state(self):
        arrs = [np.zeros((self.n, 3)) for _ in range(5)]
        lib().ora_get_state(self.h, *[_pd(a) for a in arrs])
        return dict(zip(["x", "v", "w", "F", "T"], arrs))

    def contacts(self):
        nc = lib().ora_num_contacts(self.h)
        i = np.zeros(max(nc, 1), np.int32)
        j = np.zeros(max(nc, 1), np.int32)
        b = np.zeros(max(nc, 1), np.uint8)
        xi = np.zeros((max(nc, 1), 3))
        lib().ora_get_contacts(self.h, i.ctypes.data, j.ctypes.data, b.ctypes.data, xi.ctypes.data, max(nc, 1))
        return i[:nc], j[:nc], b[:nc], xi[:nc]

    def voidfrac(self):
        out = np.zeros(self.ncell, np.uint64)
        lib().ora_get_voidfrac(self.h, out.ctypes.data)
        return out

    def diagnostics(self):
        out = np.zeros(8)
        lib().ora_get_diagnostics(self.h, _pd(out))
        return dict(zip(["ke", "ke_rot", "px", "py", "pz", "produced_mass", "n_active", "n_bonds"], out))

    def force_scale(self):
        """Per particle: the sum of the magnitudes of every force term."""
        out = np.zeros(self.n)
        lib().ora_get_force_scale(self.h, out.ctypes.data)
        return out

    def force_scale_net(self):
        """Per particle: the sum of the magnitudes of its contact, wall and
        body force vectors."""
        out = np.zeros(self.n)
        lib().ora_get_force_scale_net(self.h, out.ctypes.data)
        return out

    # ---- learned-closure hooks ----
    def set_closure(self, enable, k_feat):
        lib().ora_set_closure(self.h, int(enable), float(k_feat))

    def set_corrections(self, cd, cg):
        cd = _f64(cd)
        cg = _f64(cg)
        assert cd.shape == (self.n,) and cg.shape == (self.n,)
        lib().ora_set_corrections(self.h, _pd(cd), _pd(cg))

    def closure_data(self):
        """[n, 12] per particle from the last force evaluation: features
        (solid fraction, slip speed, k, coordination, mean overlap / d), drag
        force (3), half the summed bond capacity, fluid cell, c_d, c_g."""
        out = np.zeros((self.n, CL_COLS))
        lib().ora_get_closure_data(self.h, _pd(out))
        return out

    def step_closure(self, theta, nsteps, lo, hi, cd_max, cg_max):
        """Steps with the learned closure: each step's force evaluation uses
        the corrections from the previous one; after it the network (in the
        kernels' bfloat16 rounding) maps the features it measured to the
        corrections of the next step.  A particle whose features leave the
        box [lo, hi] gets c_d = c_g = 1 (plain coarse-graining)."""
        for _ in range(nsteps):
            self.step(1)
            cd, cg = closure_corrections(theta, self.closure_data(), lo, hi, cd_max, cg_max)
            self.set_corrections(cd, cg)

    def set_stage(self, st: OraStage):
        if lib().ora_set_stage(self.h, C.byref(st)) != 0:
            raise ValueError("ora_set_stage: invalid stage")

    def boundaries(self):
        """Top-plate height, its velocity, the stress on it, the penetrometer
        tip's height and direction, the force along z on the penetrometer."""
        out = np.zeros(6)
        lib().ora_get_boundaries(self.h, _pd(out))
        return dict(H=out[0], v_plate=out[1], stress=out[2], pen_z=out[3], pen_dir=int(out[4]),
                    pen_force=out[5])

    def fluid(self):
        """(pressure [Cf], superficial velocity [Cf,3], dynamic pressure
        gradient [Cf,3], iterations of the last solve) of a Darcy sample."""
        nc = self.ncell
        p, U, g = np.zeros(nc), np.zeros((nc, 3)), np.zeros((nc, 3))
        it = C.c_int64(0)
        lib().ora_get_fluid(self.h, p.ctypes.data, U.ctypes.data, g.ctypes.data, C.byref(it))
        return p, U, g, it.value

    def reaction(self):
        """Drag reaction per cell (Eq. 7) in quanta of 2^-60 N [Cf,3]."""
        out = np.zeros((self.ncell, 3), np.int64)
        lib().ora_get_reaction(self.h, out.ctypes.data)
        return out

    def removed_step(self):
        out = np.zeros(self.n, np.int64)
        lib().ora_get_removed_step(self.h, out.ctypes.data)
        return out


CL_COLS = 12


def closure_corrections(theta, data, lo, hi, cd_max, cg_max):
    """(c_d, c_g) per particle from closure data rows (see Sim.closure_data)."""
    from . import mlp
    X = data[:, :5]
    o, _ = mlp.forward(theta, X, bf16_ops=True)
    cd, cg = mlp.corrections(o, cd_max, cg_max)
    inside = np.all((X >= np.asarray(lo)) & (X <= np.asarray(hi)), axis=1)
    cd = np.where(inside, cd, 1.0)
    cg = np.where(inside, cg, 1.0)
    return cd, cg


# ---- coarse-graining rules (Sec. 2.4, Eq. 14-35, Table 3) ----

def cg_scale(d_fine, k, scheme, gamma_fine):
    """Grain diameters and surface energy for a coarse-grained sample.

    SSW (Sec. 2.4, Fig. 3): every grain is one fine particle scaled by k
    (d_g = k d_p, Eq. 14) and N_g = N_p / k^3 (Eq. 16), so the PSD shape is
    kept; the grains are the first N_p / k^3 fine particles (a random
    subsample when the input is a random draw).  SSP: monodisperse grains of
    k times the volume-mean fine diameter, N_g = N_p / k^3 (mass kept,
    Eq. 17-20).  gamma_g = k gamma_p (Eq. 24); E, nu, e, mu and rho are
    unchanged (Eq. 19, 28, 34, 35; Table 3).
    """
    d_fine = np.asarray(d_fine, dtype=np.float64)
    ng = int(len(d_fine) // (k ** 3))
    if scheme == "none" or k == 1:
        return d_fine.copy(), gamma_fine
    if scheme == "ssw":
        return k * d_fine[:ng], k * gamma_fine
    if scheme == "ssp":
        dbar = float(np.mean(d_fine ** 3)) ** (1.0 / 3.0)
        return np.full(ng, k * dbar), k * gamma_fine
    raise ValueError(scheme)
