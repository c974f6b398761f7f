"""Python view of the FP64 CPU oracle (``glmb_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py``.  The library under
``paper_2512_06230_gb300`` never imports it, and it imports nothing from
there.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glmb_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ERRORS = {0: "ok", 1: "invalid argument", 3: "capacity", 5: "numeric", 6: "call order"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, OpenMP over parents)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "glmb_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
                               "-Wall", "-Wno-unknown-pragmas", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Config(C.Structure):
    _fields_ = [("dim_x", C.c_int32), ("dim_z", C.c_int32), ("dt", C.c_double),
                ("q", C.c_double), ("R", C.c_double * 9), ("p_s", C.c_double),
                ("p_d", C.c_double), ("lambda_d", C.c_double), ("clutter_rate", C.c_double),
                ("volume", C.c_double), ("gate", C.c_double), ("h_max", C.c_int32),
                ("h_up", C.c_int32), ("tau", C.c_double), ("seed", C.c_uint64),
                ("score_mode", C.c_int32), ("n_threads", C.c_int32), ("model", C.c_int32),
                ("n_particles", C.c_int32), ("sigma_a", C.c_double), ("sigma_w", C.c_double),
                ("ess_frac", C.c_double)]


class _Birth(C.Structure):
    _fields_ = [("r", C.c_double), ("mean", C.c_double * 6), ("cov", C.c_double * 36)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [C.POINTER(_Config)]
        lib.orc_destroy.argtypes = [P]
        lib.orc_reset.argtypes = [P]
        lib.orc_import.argtypes = [P, C.c_int, C.c_int, P, P, P, P, P, P, P]
        lib.orc_export_counts.argtypes = [P, P, P, P]
        lib.orc_export.argtypes = [P, P, P, P, P, P, P, P]
        lib.orc_predict.argtypes = [P, P, C.c_int]
        lib.orc_update.argtypes = [P, P, C.c_int]
        lib.orc_prune.argtypes = [P]
        lib.orc_num_parents.argtypes = [P]
        lib.orc_parent_slots.argtypes = [P, C.c_int]
        lib.orc_slot.argtypes = [P, C.c_int, C.c_int, P, P, P, P, P, P, P]
        lib.orc_pair.argtypes = [P, C.c_int, C.c_int, C.c_int, P, P, P, P]
        lib.orc_gate_margin.argtypes = [P, C.c_int]
        lib.orc_gate_margin.restype = C.c_double
        lib.orc_children.argtypes = [P, P, P, P, P, P]
        lib.orc_child.argtypes = [P, C.c_int, C.c_int, P, P]
        lib.orc_kept.argtypes = [P, P, P, P]
        lib.orc_kept_theta.argtypes = [P, P]
        lib.orc_estimates.argtypes = [P, C.c_int, P, P, P, P, P, P, P, C.c_int, P]
        lib.orc_meas_assoc.argtypes = [P, P]
        lib.orc_bruteforce.argtypes = [P, C.c_int, C.c_int, P, P, P]
        lib.orc_parent_pairs.argtypes = [P, C.c_int, P, P, P, P, P]
        lib.orc_set_gate.argtypes = [P, P, C.c_double]
        lib.orc_mlp_margin.argtypes = [P, C.c_int]
        lib.orc_mlp_margin.restype = C.c_double
        lib.orc_gate_eval.argtypes = [P, C.c_int, C.c_int, C.c_int, P, P]
        lib.orc_mlp_logit.argtypes = [P, P, C.c_int]
        lib.orc_mlp_logit.restype = C.c_double
        lib.orc_philox.argtypes = [P, P, P]
        lib.orc_mix64.argtypes = [C.c_uint64]
        lib.orc_mix64.restype = C.c_uint64
        lib.orc_import_particles.argtypes = [P, P, P]
        lib.orc_export_particles.argtypes = [P, P, P]
        lib.orc_slot_particles.argtypes = [P, C.c_int, C.c_int, P, P]
        lib.orc_resample_margin.argtypes = [P]
        lib.orc_resample_margin.restype = C.c_double
        lib.orc_ctrv.argtypes = [P, C.c_double, C.c_double, C.c_double, P]
        lib.orc_particle_normals.argtypes = [P, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                             C.c_uint32, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what}: {ERRORS.get(rc, rc)}")


GATE_NPARAM = 8779


def mlp_logit(params, feat, round_act: bool = True) -> float:
    """The C oracle's MLP forward pass on one raw feature row."""
    p = np.ascontiguousarray(params, np.float32).reshape(-1)
    f = np.ascontiguousarray(feat, np.float64).reshape(-1)
    assert p.size == GATE_NPARAM and f.size == 5
    return _load().orc_mlp_logit(_ptr(p), _ptr(f), int(round_act))


def philox(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def mix64(x: int) -> int:
    return int(_load().orc_mix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def make_config(cfg: dict, n_threads: int = 1) -> _Config:
    c = _Config()
    c.dim_x, c.dim_z = int(cfg["dim_x"]), int(cfg["dim_z"])
    c.dt, c.q = float(cfg["dt"]), float(cfg["q"])
    R = np.zeros(9)
    d = c.dim_z
    R[: d * d] = np.asarray(cfg["R"], dtype=np.float64).reshape(d, d).ravel()
    for i in range(9):
        c.R[i] = R[i]
    c.p_s, c.p_d, c.lambda_d = float(cfg["p_s"]), float(cfg["p_d"]), float(cfg["lambda_d"])
    c.clutter_rate, c.volume = float(cfg["clutter_rate"]), float(cfg["volume"])
    c.gate = float(cfg["gate"])
    c.h_max, c.h_up, c.tau = int(cfg["h_max"]), int(cfg["h_up"]), float(cfg["tau"])
    c.seed = int(cfg["seed"]) & 0xFFFFFFFFFFFFFFFF
    c.score_mode = int(cfg.get("score_mode", 0))
    c.n_threads = int(n_threads)
    c.model = int(cfg.get("model", 0))
    c.n_particles = int(cfg.get("n_particles", 0))
    c.sigma_a = float(cfg.get("sigma_a", 0.0))
    c.sigma_w = float(cfg.get("sigma_w", 0.0))
    c.ess_frac = float(cfg.get("ess_frac", 0.0))
    return c


def ctrv(x, dt, a=0.0, alpha=0.0) -> np.ndarray:
    """The oracle's CTRV step of one state (px, py, v, heading, turn rate)."""
    xi = np.ascontiguousarray(x, np.float64).reshape(5)
    out = np.zeros(5)
    _load().orc_ctrv(_ptr(xi), float(dt), float(a), float(alpha), _ptr(out))
    return out


def births_array(births, dim_x: int):
    arr = (_Birth * max(len(births), 1))()
    for j, (r, mean, cov) in enumerate(births):
        arr[j].r = float(r)
        m = np.asarray(mean, dtype=np.float64)
        P = np.asarray(cov, dtype=np.float64).reshape(dim_x, dim_x)
        for a in range(dim_x):
            arr[j].mean[a] = m[a]
        flat = P.ravel()
        for a in range(dim_x * dim_x):
            arr[j].cov[a] = flat[a]
    return arr


class Oracle:
    """The FP64 oracle filter.  Method names follow the library's C ABI."""

    def __init__(self, cfg: dict, n_threads: int = 1):
        self.lib = _load()
        self.cfg = dict(cfg)
        self._c = make_config(cfg, n_threads)
        self.dx, self.dz = self._c.dim_x, self._c.dim_z
        self.h = self.lib.orc_create(C.byref(self._c))
        if not self.h:
            raise OracleError("orc_create rejected the configuration")
        self.M = 0

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.orc_destroy(h)
            self.h = None

    # -- filter steps ---------------------------------------------------
    def reset(self):
        self.lib.orc_reset(self.h)

    def predict(self, births):
        arr = births_array(births, self.dx)
        _check(self.lib.orc_predict(self.h, C.cast(arr, C.c_void_p), len(births)), "predict")

    def update(self, Z):
        Z = np.ascontiguousarray(Z, dtype=np.float32).reshape(-1, self.dz)
        self.M = len(Z)
        _check(self.lib.orc_update(self.h, _ptr(Z), len(Z)), "update")

    def prune(self):
        _check(self.lib.orc_prune(self.h), "prune")

    def step(self, births, Z):
        self.predict(births)
        self.update(Z)
        self.prune()

    # -- state -------------------------------------------------------------
    @property
    def particles(self) -> int:
        return self._c.n_particles if self._c.model == 1 else 0

    def import_state(self, frame, logw, uid, tracks):
        """tracks: list (per hypothesis) of (lk, lb, mean, cov), or with the
        particle model (lk, lb, mean, cov, x[P][5], logw[P]) (the mean and
        covariance are then recomputed from the particles)."""
        H = len(logw)
        ntr = np.array([len(t) for t in tracks], dtype=np.int32)
        n = int(ntr.sum())
        lk = np.zeros(max(n, 1), np.uint32)
        lb = np.zeros(max(n, 1), np.uint32)
        mean = np.zeros((max(n, 1), self.dx))
        cov = np.zeros((max(n, 1), self.dx, self.dx))
        o = 0
        for tr in tracks:
            for rec in tr:
                lk[o], lb[o], mean[o], cov[o] = rec[:4]
                o += 1
        lw = np.ascontiguousarray(logw, dtype=np.float64)
        ud = np.ascontiguousarray(uid, dtype=np.uint64)
        _check(self.lib.orc_import(self.h, int(frame), H, _ptr(lw), _ptr(ud), _ptr(ntr),
                                   _ptr(lk), _ptr(lb), _ptr(mean), _ptr(cov)), "import")
        Np = self.particles
        if Np:
            x = np.zeros((max(n, 1), Np, 5))
            pw = np.zeros((max(n, 1), Np))
            o = 0
            for tr in tracks:
                for rec in tr:
                    x[o], pw[o] = rec[4], rec[5]
                    o += 1
            _check(self.lib.orc_import_particles(self.h, _ptr(x), _ptr(pw)), "import_particles")

    def export_state(self):
        H, n, fr = C.c_int(), C.c_int(), C.c_int()
        self.lib.orc_export_counts(self.h, C.byref(H), C.byref(n), C.byref(fr))
        H, n = H.value, n.value
        logw = np.zeros(H)
        uid = np.zeros(H, np.uint64)
        ntr = np.zeros(H, np.int32)
        lk = np.zeros(max(n, 1), np.uint32)
        lb = np.zeros(max(n, 1), np.uint32)
        mean = np.zeros((max(n, 1), self.dx))
        cov = np.zeros((max(n, 1), self.dx, self.dx))
        self.lib.orc_export(self.h, _ptr(logw), _ptr(uid), _ptr(ntr), _ptr(lk), _ptr(lb),
                            _ptr(mean), _ptr(cov))
        Np = self.particles
        if Np:
            x = np.zeros((max(n, 1), Np, 5))
            pw = np.zeros((max(n, 1), Np))
            _check(self.lib.orc_export_particles(self.h, _ptr(x), _ptr(pw)), "export_particles")
        tracks, o = [], 0
        for h in range(H):
            if Np:
                tracks.append([(int(lk[o + t]), int(lb[o + t]), mean[o + t].copy(), cov[o + t].copy(),
                                x[o + t].copy(), pw[o + t].copy()) for t in range(ntr[h])])
            else:
                tracks.append([(int(lk[o + t]), int(lb[o + t]), mean[o + t].copy(), cov[o + t].copy())
                               for t in range(ntr[h])])
            o += ntr[h]
        return fr.value, logw, uid, tracks

    def slot_particles(self, h, t):
        Np = self.particles
        x = np.zeros((Np, 5))
        pw = np.zeros(Np)
        _check(self.lib.orc_slot_particles(self.h, h, t, _ptr(x), _ptr(pw)), "slot_particles")
        return x, pw

    def resample_margin(self) -> float:
        return self.lib.orc_resample_margin(self.h)

    def particle_normals(self, lk, lb, p, stream, call) -> np.ndarray:
        out = np.zeros(2)
        self.lib.orc_particle_normals(self.h, lk, lb, p, stream, call, _ptr(out))
        return out

    # -- introspection -------------------------------------------------------
    def num_parents(self):
        return self.lib.orc_num_parents(self.h)

    def parent_slots(self, h):
        return self.lib.orc_parent_slots(self.h, h)

    def slot(self, h, t):
        lk, lb = C.c_uint32(), C.c_uint32()
        mean = np.zeros(self.dx)
        cov = np.zeros((self.dx, self.dx))
        p, dp, ld = C.c_double(), C.c_double(), C.c_double()
        _check(self.lib.orc_slot(self.h, h, t, C.byref(lk), C.byref(lb), _ptr(mean), _ptr(cov),
                                 C.byref(p), C.byref(dp), C.byref(ld)), "slot")
        return dict(label=(lk.value, lb.value), mean=mean, cov=cov, p=p.value, dprob=dp.value,
                    logdetS=ld.value)

    def pair(self, h, t, i):
        d2, lc, q = C.c_double(), C.c_double(), C.c_double()
        e = np.zeros(3)
        g = self.lib.orc_pair(self.h, h, t, i, C.byref(d2), C.byref(lc), _ptr(e), C.byref(q))
        if g < 0:
            raise OracleError("pair index")
        return dict(gated=bool(g), d2=d2.value, logC=lc.value, e=e[: self.dz].copy(), q=q.value)

    def gate_margin(self, h):
        return self.lib.orc_gate_margin(self.h, h)

    def parent_pairs(self, h):
        """Parent h's gated-pair table: dict(ptr, meas, logC, q, e)."""
        K = self.lib.orc_parent_pairs(self.h, h, None, None, None, None, None)
        if K < 0:
            raise OracleError("parent index")
        T = self.parent_slots(h)
        ptr = np.zeros(T + 1, np.int32)
        meas = np.zeros(max(K, 1), np.int32)
        lc = np.zeros(max(K, 1))
        q = np.zeros(max(K, 1))
        e = np.zeros((max(K, 1), self.dz))
        self.lib.orc_parent_pairs(self.h, h, _ptr(ptr), _ptr(meas), _ptr(lc), _ptr(q), _ptr(e))
        return dict(ptr=ptr, meas=meas[:K], logC=lc[:K], q=q[:K], e=e[:K])

    # -- learned gate ----------------------------------------------------------
    def set_gate(self, params, threshold: float = 0.0):
        """Switch the learned gate on (params: GATE_NPARAM float32 values) or
        off (None); applies from the next update."""
        if params is None:
            self._gate = None
            _check(self.lib.orc_set_gate(self.h, None, 0.0), "set_gate")
            return
        self._gate = np.ascontiguousarray(params, np.float32).reshape(-1)
        assert self._gate.size == GATE_NPARAM
        _check(self.lib.orc_set_gate(self.h, _ptr(self._gate), float(threshold)), "set_gate")

    def mlp_margin(self, h):
        return self.lib.orc_mlp_margin(self.h, h)

    def gate_eval(self, h, t, i):
        feat = np.zeros(5)
        lg = C.c_double()
        if self.lib.orc_gate_eval(self.h, h, t, i, _ptr(feat), C.byref(lg)) != 0:
            raise OracleError("gate_eval index")
        return feat, lg.value

    def children(self):
        n = self.num_parents() * self._c.h_up
        st = np.zeros(n, np.int8)
        lw = np.zeros(n)
        mg = np.zeros(n)
        na = np.zeros(n, np.int32)
        ud = np.zeros(n, np.uint64)
        _check(self.lib.orc_children(self.h, _ptr(st), _ptr(lw), _ptr(mg), _ptr(na), _ptr(ud)),
               "children")
        return dict(status=st, logw=lw, margin=mg, n_alive=na, uid=ud)

    def child(self, h, n):
        T = self.parent_slots(h)
        dead = np.zeros(max(T, 1), np.uint8)
        theta = np.zeros(max(self.M, 1), np.uint16)
        _check(self.lib.orc_child(self.h, h, n, _ptr(dead), _ptr(theta)), "child")
        return dead[:T].copy(), theta[: self.M].copy()

    def kept(self):
        nk = self.lib.orc_kept(self.h, None, None, None)
        if nk < 0:
            raise OracleError("kept: call order")
        idx = np.zeros(nk, np.int64)
        lw = np.zeros(nk)
        lse = C.c_double()
        self.lib.orc_kept(self.h, _ptr(idx), _ptr(lw), C.byref(lse))
        return idx, lw, lse.value

    def kept_theta(self):
        nk = self.lib.orc_kept(self.h, None, None, None)
        th = np.zeros((max(nk, 1), max(self.M, 1)), np.uint16)
        self.lib.orc_kept_theta(self.h, _ptr(th))
        return th[:nk, : self.M].copy()

    def estimates(self, cap: int = 4096, pmf_cap: int = 4096):
        n = C.c_int()
        lk = np.zeros(cap, np.uint32)
        lb = np.zeros(cap, np.uint32)
        mean = np.zeros((cap, self.dx))
        cov = np.zeros((cap, self.dx, self.dx))
        r = np.zeros(cap)
        pmf = np.zeros(pmf_cap)
        mi = C.c_int()
        _check(self.lib.orc_estimates(self.h, cap, C.byref(n), _ptr(lk), _ptr(lb), _ptr(mean),
                                      _ptr(cov), _ptr(r), _ptr(pmf), pmf_cap, C.byref(mi)),
               "estimates")
        k = n.value
        return dict(n=k, labels=list(zip(lk[:k].tolist(), lb[:k].tolist())), mean=mean[:k],
                    cov=cov[:k], r=r[:k], pmf=pmf, map_index=mi.value)

    def meas_assoc(self):
        r = np.zeros(max(self.M, 1))
        _check(self.lib.orc_meas_assoc(self.h, _ptr(r)), "meas_assoc")
        return r[: self.M]

    def bruteforce(self, h: int = 0, cap: int = 2_000_000):
        T = self.parent_slots(h)
        dead = np.zeros((cap, max(T, 1)), np.uint8)
        theta = np.zeros((cap, max(self.M, 1)), np.uint16)
        lw = np.zeros(cap)
        n = self.lib.orc_bruteforce(self.h, h, cap, _ptr(dead), _ptr(theta), _ptr(lw))
        if n < 0:
            raise OracleError("bruteforce: too large")
        return dead[:n, :T], theta[:n, : self.M], lw[:n]
