"""FP64 CPU oracle for the eco-driving DP (ctypes wrapper over ecodp_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use this package; the CUDA library and its
Python binding never import it.  The oracle shares no code with the CUDA
path; it reads problem instances through plain attributes (duck-typed), so it
does not import the product package either.

Entry points (see ecodp_oracle.c for the semantics and the paper passages):
  make(problem, grids=None)  -> OracleProblem
  stage(op, k, Vnext, mode, idx=None)
  solve(op, mode)            -> (list of J_k, list of pi_k, list of second_k)
  rollout(op, Vall, x0)
  model_step(op, k, v, soc, t, Te, Tm, b)
  sequence_cost(op, x0, useq)
  evaluate(op, k, Vnext, v, soc, t, ie, im, b, mode)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ecodp_oracle.c")
LIB = os.path.join(HERE, "libecodp_oracle.so")

NOMINAL, LENIENT, STRICT = 0, 1, 2
# FP32 resolution band in index units (2^-18 ~ 3.8e-6, times 1 + scale) and the
# phase band of the acceptance criteria (1e-4 s).
FP_BAND = 2.0 ** -18
PHASE_BAND = 1e-4

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", SRC, "-o", LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


class _Problem(C.Structure):
    _fields_ = [
        ("n_stages", C.c_int32), ("ds", C.c_double), ("grade", C.c_void_p),
        ("nv", C.c_void_p), ("v_nodes", C.c_void_p),
        ("nxi", C.c_void_p), ("xi_nodes", C.c_void_p),
        ("nt", C.c_void_p), ("t_nodes", C.c_void_p),
        ("n_te", C.c_int32), ("te", C.c_void_p),
        ("n_tm", C.c_int32), ("tm", C.c_void_p),
        ("n_b", C.c_int32), ("brake_decel", C.c_double),
        ("a_min", C.c_double), ("a_max", C.c_double),
        ("mass", C.c_double), ("cda", C.c_double), ("crr", C.c_double), ("rho", C.c_double),
        ("g", C.c_double), ("r_wheel", C.c_double), ("gear", C.c_double), ("eta_motor", C.c_double),
        ("voc", C.c_double), ("r0", C.c_double), ("cap_As", C.c_double),
        ("fuel_coef", C.c_double * 6), ("fuel_scale", C.c_double), ("gamma", C.c_double),
        ("soc_ref", C.c_double), ("w_soc", C.c_double), ("v_ref", C.c_double), ("w_v", C.c_double),
        ("n_lights", C.c_int32), ("light_node", C.c_void_p),
        ("cycle", C.c_void_p), ("red", C.c_void_p), ("offset", C.c_void_p),
        ("fp_band", C.c_double), ("phase_band", C.c_double),
        ("v_off", C.c_void_p), ("xi_off", C.c_void_p), ("t_off", C.c_void_p), ("V_off", C.c_void_p),
        ("light_model", C.c_int32), ("torque_limits", C.c_int32),
        ("te_max_coef", C.c_double * 3), ("bsg_power_max", C.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            P = C.POINTER(_Problem)
            vp = C.c_void_p
            L.orc_value_offset.argtypes = [P, C.c_int]
            L.orc_value_offset.restype = C.c_int64
            L.orc_is_red.argtypes = [P, C.c_int, C.c_double]
            L.orc_terminal_cost.argtypes = [P, C.c_double, C.c_double]
            L.orc_terminal_cost.restype = C.c_double
            L.orc_model_step.argtypes = [P, C.c_int, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_double, C.c_int, vp]
            L.orc_interp.argtypes = [P, C.c_int, vp, C.c_double, C.c_double, C.c_double]
            L.orc_interp.restype = C.c_double
            L.orc_terminal.argtypes = [P, vp]
            L.orc_stage.argtypes = [P, C.c_int, C.c_int, vp, C.c_int64, vp, vp, vp, vp, vp, C.c_int]
            L.orc_solve.argtypes = [P, C.c_int, vp, vp, vp, C.c_int]
            L.orc_rollout.argtypes = [P, vp, vp, vp, vp, vp, vp]
            L.orc_sequence_cost.argtypes = [P, vp, vp, vp]
            L.orc_sequence_cost.restype = C.c_double
            L.orc_adjoint.argtypes = [P, vp, vp, vp, vp, vp, vp, vp, vp]
            L.orc_eval.argtypes = [P, C.c_int, C.c_int, vp, C.c_double, C.c_double, C.c_double,
                                   C.c_int, C.c_int, C.c_int, vp]
            L.orc_eval.restype = C.c_double
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _uniform(lo, hi, n):
    if n == 1:
        return np.array([lo], np.float64)
    i = np.arange(n, dtype=np.float64)
    return lo + (hi - lo) * i / (n - 1)


class OracleProblem:
    """A problem marshalled for the C oracle; keeps its arrays alive."""

    def __init__(self, p, grids=None, fp_band: float = FP_BAND, phase_band: float = PHASE_BAND):
        N = int(p.n_stages)
        self.p = p
        self.N = N
        if grids is None:
            v = _uniform(p.v_lo, p.v_hi, p.n_v)
            x = _uniform(p.soc_lo, p.soc_hi, p.n_soc)
            t = _uniform(p.t_lo, p.t_hi, p.n_t)
            grids = [(v, x, t)] * (N + 1)
        assert len(grids) == N + 1
        self.grids = [tuple(np.ascontiguousarray(a, np.float64) for a in g) for g in grids]
        for g in self.grids:
            for a in g:
                assert a.ndim == 1 and a.size >= 1 and np.all(np.diff(a) > 0), "grid nodes must increase"
        self.shapes = [(g[0].size, g[1].size, g[2].size) for g in self.grids]
        self._keep = {}

        def keep(name, arr):
            self._keep[name] = arr
            return _ptr(arr)

        s = _Problem()
        s.n_stages = N
        s.ds = float(p.ds)
        s.grade = keep("grade", np.ascontiguousarray(p.grade, np.float64))
        s.nv = keep("nv", np.array([g[0].size for g in self.grids], np.int32))
        s.v_nodes = keep("vn", np.concatenate([g[0] for g in self.grids]))
        s.nxi = keep("nx", np.array([g[1].size for g in self.grids], np.int32))
        s.xi_nodes = keep("xn", np.concatenate([g[1] for g in self.grids]))
        s.nt = keep("nt", np.array([g[2].size for g in self.grids], np.int32))
        s.t_nodes = keep("tn", np.concatenate([g[2] for g in self.grids]))
        self.te = _uniform(p.te_lo, p.te_hi, p.n_te)
        self.tm = _uniform(p.tm_lo, p.tm_hi, p.n_tm)
        s.n_te = p.n_te
        s.te = keep("te", self.te)
        s.n_tm = p.n_tm
        s.tm = keep("tm", self.tm)
        s.n_b = p.n_brake
        s.brake_decel = p.brake_decel
        for f in ("a_min", "a_max", "mass", "cda", "crr", "rho", "g", "r_wheel", "gear", "eta_motor",
                  "voc", "r0", "fuel_scale", "gamma", "soc_ref", "w_soc", "v_ref", "w_v"):
            setattr(s, f, float(getattr(p, f)))
        s.cap_As = float(p.capacity_As)
        for i in range(6):
            s.fuel_coef[i] = float(p.fuel_coef[i])
        nl = len(p.light_stage)
        s.n_lights = nl
        s.light_node = keep("ln", np.ascontiguousarray(p.light_stage, np.int32))
        s.cycle = keep("cy", np.ascontiguousarray(p.cycle, np.float64))
        s.red = keep("rd", np.ascontiguousarray(p.red, np.float64))
        s.offset = keep("of", np.ascontiguousarray(p.offset, np.float64))
        s.fp_band = fp_band
        s.phase_band = phase_band
        cum = lambda n: np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
        s.v_off = keep("vo", cum([g[0].size for g in self.grids]))
        s.xi_off = keep("xo", cum([g[1].size for g in self.grids]))
        s.t_off = keep("to", cum([g[2].size for g in self.grids]))
        s.V_off = keep("Vo", cum([int(np.prod(sh)) for sh in self.shapes]))
        # paper variants (absent attributes: the default readings)
        s.light_model = int(getattr(p, "light_model", 0))
        s.torque_limits = int(getattr(p, "torque_limits", 0))
        coef = getattr(p, "te_max_coef", (0.0, 0.0, 0.0))
        for i in range(3):
            s.te_max_coef[i] = float(coef[i])
        s.bsg_power_max = float(getattr(p, "bsg_power_max", 0.0))
        self.s = s
        self.ref = C.byref(s)

    @property
    def n_controls(self):
        return self.p.n_te * self.p.n_tm * self.p.n_brake

    def decode(self, u: int):
        """Control index u = (ie * n_tm + im) * n_b + b -> (Te, Tm, b)."""
        nb, ntm = self.p.n_brake, self.p.n_tm
        b = u % nb
        im = (u // nb) % ntm
        ie = u // (nb * ntm)
        return self.te[ie], self.tm[im], b


def make(p, grids=None, **kw) -> OracleProblem:
    return OracleProblem(p, grids, **kw)


def terminal(op: OracleProblem) -> np.ndarray:
    out = np.empty(op.shapes[op.N], np.float64)
    lib().orc_terminal(op.ref, _ptr(out))
    return out


def stage(op: OracleProblem, k: int, Vnext: np.ndarray, mode: int = NOMINAL, idx=None, nthreads: int = 0):
    """One backward step at stage k.  Returns dict(V, pi, second, nfrag), each
    shaped like the stage-k grid (or like idx when sampling)."""
    Vn = np.ascontiguousarray(Vnext, np.float64)
    assert Vn.shape == op.shapes[k + 1], (Vn.shape, op.shapes[k + 1])
    if idx is None:
        shape = op.shapes[k]
        n = 0
        ip = None
    else:
        idx = np.ascontiguousarray(idx, np.int64)
        shape = idx.shape
        n = idx.size
        ip = _ptr(idx)
    V = np.empty(shape, np.float64)
    pi = np.empty(shape, np.int32)
    sec = np.empty(shape, np.float64)
    nf = np.empty(shape, np.int32)
    rc = lib().orc_stage(op.ref, k, mode, _ptr(Vn), n, ip, _ptr(V), _ptr(pi), _ptr(sec), _ptr(nf),
                         nthreads)
    if rc:
        raise RuntimeError(f"orc_stage failed: {rc}")
    return dict(V=V, pi=pi, second=sec, nfrag=nf)


def solve(op: OracleProblem, mode: int = NOMINAL, nthreads: int = 0):
    """Full backward sweep; returns (V[k] arrays for k=0..N, pi[k] for
    k=0..N-1, second[k] for k=0..N-1)."""
    N = op.N
    total = int(lib().orc_value_offset(op.ref, N + 1))
    Vall = np.empty(total, np.float64)
    piall = np.full(total, -1, np.int32)
    secall = np.empty(total, np.float64)
    rc = lib().orc_solve(op.ref, mode, _ptr(Vall), _ptr(piall), _ptr(secall), nthreads)
    if rc:
        raise RuntimeError(f"orc_solve failed: {rc}")
    Vs, pis, secs = [], [], []
    for k in range(N + 1):
        o = int(lib().orc_value_offset(op.ref, k))
        n = int(np.prod(op.shapes[k]))
        Vs.append(Vall[o:o + n].reshape(op.shapes[k]))
        if k < N:
            pis.append(piall[o:o + n].reshape(op.shapes[k]))
            secs.append(secall[o:o + n].reshape(op.shapes[k]))
    op._Vall, op._piall, op._secall = Vall, piall, secall
    return Vs, pis, secs


def rollout(op: OracleProblem, Vs, x0=None):
    """Forward rollout through J_1..J_N.  Returns a dict with traj [(N+1),3],
    u [N], dt, wait, fuel, cost, gap [N], fuel_g, time_s, J, status."""
    N = op.N
    Vall = np.concatenate([np.ascontiguousarray(V, np.float64).ravel() for V in Vs])
    x0 = np.array(op.p.x0 if x0 is None else x0, np.float64)
    traj = np.zeros((N + 1) * 3)
    u = np.full(N, -1, np.int32)
    step = np.zeros(N * 5)
    tot = np.zeros(4)
    rc = lib().orc_rollout(op.ref, _ptr(Vall), _ptr(x0), _ptr(traj), _ptr(u), _ptr(step), _ptr(tot))
    st = step.reshape(N, 5)
    return dict(traj=traj.reshape(N + 1, 3), u=u, dt=st[:, 0], wait=st[:, 1], fuel=st[:, 2],
                cost=st[:, 3], gap=st[:, 4], fuel_g=tot[0], time_s=tot[1], J=tot[2],
                status=int(rc), fail_stage=int(tot[3]))


THETA = ("mass", "cda", "crr", "r0", "fuel_scale")


def adjoint(op: OracleProblem, x0=None, want_lam: bool = False):
    """dJ_0(x0)/dtheta for theta = THETA by the forward lambda sweep, on the
    nominal solution of the last `solve(op)` call.  Returns (grad[5], diag
    dict, support flags over the states of stages 0..N-1, status); with
    want_lam the diag dict also holds "lam", the lambda of every state (same
    layout as the support flags)."""
    if getattr(op, "_piall", None) is None:
        raise RuntimeError("call solve(op) first")
    x0 = np.array(op.p.x0 if x0 is None else x0, np.float64)
    grad = np.zeros(5)
    diag = np.zeros(6)
    support = np.zeros(op._Vall.size, np.uint8)
    lam = np.zeros(op._Vall.size, np.float64) if want_lam else None
    rc = lib().orc_adjoint(op.ref, _ptr(op._Vall), _ptr(op._piall), _ptr(op._secall), _ptr(x0), _ptr(grad),
                           _ptr(diag), _ptr(support), _ptr(lam) if want_lam else None)
    d = dict(support_size=int(diag[0]), snapped=bool(diag[1]), infeasible_corner=bool(diag[2]),
             min_gap=float(diag[3]), near_tie_mass=float(diag[4]), snapped_mass=float(diag[5]))
    if want_lam:
        d["lam"] = lam
    return grad, d, support, int(rc)


def model_step(op: OracleProblem, k, v, soc, t, Te, Tm, b):
    """One model step: returns None if infeasible, else dict(v1, soc1, t1, dt,
    wait, fuel_rate, cost)."""
    out = np.zeros(7)
    ok = lib().orc_model_step(op.ref, int(k), float(v), float(soc), float(t), float(Te), float(Tm), int(b),
                              _ptr(out))
    if not ok:
        return None
    return dict(zip(("v1", "soc1", "t1", "dt", "wait", "fuel_rate", "cost"), out.tolist()))


def evaluate(op: OracleProblem, k, Vnext, v, soc, t, ie, im, b, mode: int = NOMINAL):
    """One transition's value c + J_{k+1}(f(x, u)) from the stage-k state
    (v, soc, t) under control (ie, im, b) in a mode; returns (value, number of
    fragile decisions met by the nominal evaluation)."""
    Vn = np.ascontiguousarray(Vnext, np.float64)
    assert Vn.shape == op.shapes[k + 1]
    nf = np.zeros(1, np.int32)
    F = lib().orc_eval(op.ref, int(k), int(mode), _ptr(Vn), float(v), float(soc), float(t), int(ie), int(im),
                       int(b), _ptr(nf))
    return float(F), int(nf[0])


def terminal_cost(op: OracleProblem, v, soc) -> float:
    return float(lib().orc_terminal_cost(op.ref, float(v), float(soc)))


def is_red(op: OracleProblem, j: int, t: float) -> bool:
    return bool(lib().orc_is_red(op.ref, int(j), float(t)))


def interp(op: OracleProblem, stage_idx: int, V: np.ndarray, v, soc, t) -> float:
    Va = np.ascontiguousarray(V, np.float64)
    assert Va.shape == op.shapes[stage_idx]
    return float(lib().orc_interp(op.ref, int(stage_idx), _ptr(Va), float(v), float(soc), float(t)))


def sequence_cost(op: OracleProblem, x0, useq):
    """Exact cost of a control sequence from x0 (no grid), +inf if infeasible
    or if a state leaves the grid box."""
    x0 = np.array(x0, np.float64)
    us = np.ascontiguousarray(useq, np.int32)
    xN = np.zeros(3)
    J = lib().orc_sequence_cost(op.ref, _ptr(x0), _ptr(us), _ptr(xN))
    return float(J), xN
