"""Seeded synthetic multi-object scenes: the one input source shared by the
FP64 oracle and the CUDA path.

This module draws ground truth, detections, clutter and the per-frame LMB
birth sets.  It holds none of the filter's arithmetic (no prediction, no
likelihood, no association): it only samples the *world* that the filter
observes, so both implementations can be fed identical inputs.

Model of the world (one reading per item, the paper is silent on these
details for the Gaussian form):

* Objects move with a constant-velocity model driven by continuous white
  acceleration noise of power spectral density ``q`` (per axis, per frame of
  length ``dt``).  State order is ``[positions..., velocities...]``.
* Each frame an existing object survives with probability ``p_s``.
* A live object is detected with probability ``p_d``; a detected object
  yields ``1 + Poisson(lambda_d)`` i.i.d. position detections with noise
  ``N(0, sigma^2 I)`` (the multi-detection model of Section 3 of the paper;
  the paper's convoy experiment fixes the count at ``D`` instead).
* Clutter is Poisson(``clutter_rate``) per frame, uniform over the region.
* Detections of a frame are shuffled (the paper notes the update does not
  depend on their order, Section 4.1).
* Births: the LMB birth set of a frame holds one component per object that
  appears in that frame (centred on its true position plus N(0, (2 sigma)^2)
  noise, zero velocity, existence ``r_birth``) and Poisson(``false_births``)
  spurious components uniform over the region (existence ``r_false``).

Seeds: ``scene_seed = 1000 * cfg + rep`` by convention, filter seed
``scene_seed ^ 0x5eed``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

__all__ = ["SceneParams", "Scene", "PRESETS", "preset", "make_scene", "batch_scenes", "convoy_scene",
           "CtrvParams", "ctrv_scene", "ctrv_filter_config",
           "gate_params", "GATE_NPARAM",
           "random_state", "chi2_gate"]


@dataclasses.dataclass(frozen=True)
class SceneParams:
    name: str
    dim: int                    # spatial dimension (2 or 3); state is 2*dim
    n_objects: int
    frames: int
    extent: float               # region is [0, extent]^dim
    dt: float = 1.0
    q: float = 1.0              # white-acceleration PSD [m^2/s^3]
    sigma: float = 5.0          # detection noise std [m]
    p_s: float = 0.99
    p_d: float = 0.9
    lambda_d: float = 1.0       # detected object yields 1+Poisson(lambda_d)
    clutter_rate: float = 5.0
    birth_window: Optional[Tuple[int, int]] = (0, 24)   # birth frame ~ U{lo..hi}
    births_per_frame: float = 0.0   # extra Poisson births per frame (sweep scenes)
    speed_max: float = 10.0
    r_birth: float = 0.5
    r_false: float = 0.05
    false_births: float = 1.0
    birth_vel_std: float = 10.0
    h_max: int = 100
    h_up: int = 100
    tau: float = 1e-5
    gate_tail: float = 1e-4     # chi-square tail outside the Mahalanobis gate
    filter_clutter_rate: Optional[float] = None   # the filter's clutter rate, if not the world's


# Scene presets.  "tiny" and "mid" are the 2-D constant-velocity scenes with
# 10 and 100 objects; "sweep_N<n>" are the 3-D scalability scenes.
PRESETS = {
    "tiny": SceneParams(name="tiny", dim=2, n_objects=10, frames=50, extent=1000.0,
                        lambda_d=1.0, clutter_rate=5.0, birth_window=(0, 24),
                        h_max=100),
    "mid": SceneParams(name="mid", dim=2, n_objects=100, frames=100, extent=1000.0,
                       lambda_d=1.5, clutter_rate=20.0, birth_window=(0, 49),
                       h_max=1000),
}
for _n in (50, 200, 500, 1000):
    PRESETS[f"sweep_N{_n}"] = SceneParams(
        name=f"sweep_N{_n}", dim=3, n_objects=_n, frames=50, extent=5000.0,
        p_d=0.85, lambda_d=2.0, clutter_rate=50.0, birth_window=None,
        births_per_frame=0.01 * _n, h_max=1000)


def batch_scenes(n_scenes: int, seed: int, frames: int = 100, h_range=(100, 5000),
                 n_range=(5, 300), clutter_range=(5.0, 40.0)):
    """The batched workload: n_scenes independent 2-D scenes shaped like the
    mid scene (P_D 0.9, 1 + Poisson(1.5) detections, births over frames
    0-49) with N ~ U{n_range}, clutter rate ~ U(clutter_range) and a
    hypothesis cap H ~ U{h_range} per scene.  Returns (params, seed) pairs;
    the cap is params.h_max."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_scenes):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        h = int(rng.integers(h_range[0], h_range[1] + 1))
        lam = float(rng.uniform(*clutter_range))
        p = SceneParams(name=f"batch_{k}", dim=2, n_objects=n, frames=frames, extent=1000.0,
                        lambda_d=1.5, clutter_rate=lam, birth_window=(0, min(49, frames - 1)),
                        h_max=h)
        out.append((p, seed * 1000 + k))
    return out


def preset(name: str, **overrides) -> SceneParams:
    return dataclasses.replace(PRESETS[name], **overrides)


def convoy_path(steps: int, seed: int, dt: float = 0.1, extent: float = 80.0, laps: int = 3) -> np.ndarray:
    """A smooth closed ground track inside [0, extent]^2 standing in for the
    paper's GPS track (which is not public): a random ellipse with small
    2nd and 3rd harmonics, scaled to 80 % of the area and walked `laps`
    times, at constant speed, in `steps` samples dt apart, so that sample
    `steps` would be sample 0 again (about 10 m/s for 548 samples and 3
    laps).  Returns (steps, 4) states [x, y, vx, vy]."""
    rng = np.random.default_rng(seed)
    u = 2 * np.pi * np.linspace(0.0, 1.0, 16 * steps, endpoint=False)
    # an ellipse plus 2nd and 3rd harmonics whose derivatives stay below half
    # the ellipse's: the tangent never vanishes, so the track has no cusp
    A, B = 1.0, rng.uniform(0.6, 1.0)
    xy = np.stack([A * np.cos(u), B * np.sin(u)], 1)
    for h, amp in ((2, 0.15), (3, 0.05)):
        for a in range(2):
            xy[:, a] += amp * rng.uniform(0.3, 1.0) * B / h * np.sin(h * u + rng.uniform(0, 2 * np.pi))
    xy -= xy.min(0)
    xy *= 0.8 * extent / xy.max()
    xy += 0.1 * extent
    seg = np.linalg.norm(np.roll(xy, -1, axis=0) - xy, axis=1)
    arc = np.concatenate([[0.0], np.cumsum(seg)[:-1]])
    total = arc[-1] + seg[-1]
    s_t = (laps * total * np.arange(steps) / steps) % total
    x = np.interp(s_t, arc, xy[:, 0], period=total)
    y = np.interp(s_t, arc, xy[:, 1], period=total)
    pos = np.stack([x, y], 1)
    vel = (np.roll(pos, -1, axis=0) - np.roll(pos, 1, axis=0)) / (2 * dt)
    return np.concatenate([pos, vel], 1)


def convoy_scene(n_objects: int, seed: int, steps: int = 548, detections: int = 5,
                 sigma: float = 0.25, delta: int = 2, dt: float = 0.1, h_max: int = 100,
                 extent: float = 80.0, track_len: int = 548, particles: int = 0) -> "Scene":
    """The paper's benchmark shape (Section 4.1): n_objects copies of one
    closed ground track of track_len samples, copy n at step k at sample
    (k + n * delta) mod track_len; the first `steps` steps.  Every object gives exactly `detections` detections per step,
    N(x, sigma^2 I), left in sorted order (object, then draw); no clutter.
    All objects exist from the first step: one birth component per object
    there (position + N(0, (2 sigma)^2), velocity + N(0, 1 m^2/s^2),
    r = 0.5), plus Poisson(1) spurious births anywhere (zero velocity,
    r = 0.05) every step.  The filter model
    reads D detections as 1 + Poisson(D - 1) and P_D = 0.999.  The world
    has no clutter, but the filter assumes a little (0.5 per step over the
    area): with none, one detection outside every gate would leave no
    hypothesis with a finite weight.

    particles > 0: the same world for the particle track model (the
    paper's own): births in the CTRV state (position, speed, heading, turn
    rate; the true objects' births at their true speed and heading plus
    noise, spurious ones with any heading), filter accelerations sigma_a =
    3 m/s^2 and sigma_w = 3 rad/s^2: five detections of sigma 0.25 m leave
    few particles with weight, and smaller accelerations let the cloud
    collapse after resampling (measured on the oracle, N = 10, H_max = 100:
    1 m/s^2 and 1 rad/s^2 gave 8 % cardinality error and 0.50 m tracking
    error, 3 and 3 give 3 % and 0.12 m)."""
    rng = np.random.default_rng(seed)
    track = convoy_path(track_len, seed ^ 0xC0, dt=dt, extent=extent)
    K = len(track)
    p = SceneParams(name=f"convoy_N{n_objects}", dim=2, n_objects=n_objects, frames=steps, extent=extent,
                    dt=dt, q=10.0, sigma=sigma, p_s=0.999, p_d=0.999, lambda_d=float(detections - 1),
                    clutter_rate=0.0, birth_window=None, h_max=h_max, r_birth=0.5, r_false=0.05,
                    false_births=1.0, birth_vel_std=6.0, h_up=100, tau=1e-5, gate_tail=1e-12,
                    filter_clutter_rate=0.5)
    sb = 2.0 * sigma
    birth_cov = np.diag([sb ** 2] * 2 + [p.birth_vel_std ** 2] * 2)
    sv = 1.0
    track_cov = np.diag([sb ** 2] * 2 + [sv ** 2] * 2)
    if particles:
        p = CtrvParams(name=f"convoy_N{n_objects}", n_objects=n_objects, frames=steps, extent=extent, offset=0.0,
                       dt=dt, sigma=sigma, sigma_a=3.0, filter_sigma_w=3.0, p_s=0.999, p_d=0.999,
                       lambda_d=float(detections - 1), clutter_rate=0.0, filter_clutter_rate=0.5,
                       h_max=h_max, h_up=100, tau=1e-5, n_particles=particles, gate_tail=1e-12)
        track_cov = np.diag([sb ** 2, sb ** 2, 1.0, 0.1 ** 2, 0.1 ** 2])
        birth_cov = np.diag([sb ** 2, sb ** 2, 6.0 ** 2, 1.8 ** 2, 0.3 ** 2])
    frames = []
    for k in range(steps):
        truth = np.stack([track[(k + n * delta) % K] for n in range(n_objects)])
        Z = np.concatenate([truth[n, :2] + sigma * rng.normal(size=(detections, 2))
                            for n in range(n_objects)]).astype(np.float32)
        births = []
        if k == 0:
            for n in range(n_objects):
                if particles:
                    x, y, vx, vy = truth[n]
                    mean = np.array([x, y, math.hypot(vx, vy), math.atan2(vy, vx), 0.0])
                    mean += rng.normal(size=5) * np.array([sb, sb, 1.0, 0.1, 0.1])
                else:
                    mean = truth[n] + rng.normal(size=4) * np.array([sb, sb, sv, sv])
                births.append((0.5, mean, track_cov.copy()))
        for _ in range(int(rng.poisson(1.0))):
            if particles:
                mean = np.array([*rng.uniform(0.0, extent, size=2), 10.0, rng.uniform(-math.pi, math.pi), 0.0])
            else:
                mean = np.concatenate([rng.uniform(0.0, extent, size=2), np.zeros(2)])
            births.append((0.05, mean, birth_cov.copy()))
        frames.append(Frame(Z=Z, births=births, truth=truth, truth_ids=np.arange(n_objects)))
    return Scene(params=p, seed=seed, frames=frames)


@dataclasses.dataclass(frozen=True)
class CtrvParams:
    """Vehicles with constant-turn-rate-and-velocity motion in the plane (the
    paper's track model, Section 3), seen by the multi-detection sensor of
    the constant-velocity scenes."""
    name: str = "ctrv"
    dim: int = 2                # the plane; positions are measured
    n_objects: int = 20
    frames: int = 40
    extent: float = 1000.0      # objects start in [offset, offset + extent]^2
    offset: float = 200.0       # keeps coordinates far from the origin
    dt: float = 1.0
    sigma: float = 3.0          # detection noise std [m]
    sigma_a: float = 0.5        # longitudinal acceleration std [m/s^2]
    sigma_w: float = 0.02       # yaw acceleration std [rad/s^2]
    filter_sigma_w: float = 0.05   # the filter's yaw acceleration std (a looser model)
    speed: Tuple[float, float] = (5.0, 15.0)
    turn: float = 0.05          # initial turn rate ~ U(-turn, turn) [rad/s]
    p_s: float = 0.99
    p_d: float = 0.9
    lambda_d: float = 1.0
    clutter_rate: float = 10.0
    birth_window: Tuple[int, int] = (0, 19)
    r_birth: float = 0.5
    r_false: float = 0.05
    false_births: float = 1.0
    h_max: int = 1000
    h_up: int = 100
    tau: float = 1e-5
    n_particles: int = 256
    ess_frac: float = 0.5
    gate_tail: float = 1e-4     # chi-square tail outside the Mahalanobis gate
    filter_clutter_rate: Optional[float] = None   # the filter's clutter rate, if not the world's


def _ctrv_truth_step(x, dt, a, alpha):
    """World motion (simulation only): one CTRV step with accelerations."""
    px, py, v, psi, om = x
    if abs(om) > 1e-12:
        px2 = px + v / om * (math.sin(psi + om * dt) - math.sin(psi))
        py2 = py + v / om * (math.cos(psi) - math.cos(psi + om * dt))
    else:
        px2 = px + v * math.cos(psi) * dt
        py2 = py + v * math.sin(psi) * dt
    return np.array([px2 + 0.5 * dt * dt * math.cos(psi) * a, py2 + 0.5 * dt * dt * math.sin(psi) * a,
                     v + dt * a, psi + om * dt + 0.5 * dt * dt * alpha, om + dt * alpha])


def ctrv_scene(params: CtrvParams, seed: int) -> Scene:
    """Draw a CTRV scene: truth, detections (as make_scene), clutter over the
    region and LMB births (one per appearing vehicle: its position plus
    N(0, (2 sigma)^2), speed 10 +- 5 m/s, its heading plus N(0, 0.3^2), turn
    rate 0 +- 0.05; and Poisson(false_births) uniform spurious ones).  Frame
    truth rows are (px, py, v, heading, turn rate)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = params
    lo, hi = p.birth_window
    t_birth = sorted(int(rng.integers(lo, hi + 1)) for _ in range(p.n_objects))
    sb = 2.0 * p.sigma
    cov = np.diag([sb ** 2, sb ** 2, 5.0 ** 2, 0.3 ** 2, 0.05 ** 2])
    cov_false = np.diag([sb ** 2, sb ** 2, 5.0 ** 2, 1.5 ** 2, 0.05 ** 2])
    alive, frames, nxt, ptr = {}, [], 0, 0
    for f in range(p.frames):
        for oid in sorted(alive):
            if rng.uniform() >= p.p_s:
                del alive[oid]
                continue
            alive[oid] = _ctrv_truth_step(alive[oid], p.dt, p.sigma_a * rng.normal(),
                                          p.sigma_w * rng.normal())
        births = []
        while ptr < len(t_birth) and t_birth[ptr] == f:
            x = np.array([*(p.offset + rng.uniform(0.0, p.extent, 2)), rng.uniform(*p.speed),
                          rng.uniform(-math.pi, math.pi), rng.uniform(-p.turn, p.turn)])
            alive[nxt] = x
            mean = np.array([x[0] + rng.normal(scale=sb), x[1] + rng.normal(scale=sb), 10.0,
                             x[3] + rng.normal(scale=0.3), 0.0])
            births.append((p.r_birth, mean, cov.copy()))
            nxt += 1
            ptr += 1
        for _ in range(int(rng.poisson(p.false_births))):
            mean = np.array([*(p.offset + rng.uniform(0.0, p.extent, 2)), 10.0,
                             rng.uniform(-math.pi, math.pi), 0.0])
            births.append((p.r_false, mean, cov_false.copy()))
        Z = []
        for oid in sorted(alive):
            if rng.uniform() < p.p_d:
                m = 1 + int(rng.poisson(p.lambda_d))
                Z.append(alive[oid][:2] + p.sigma * rng.normal(size=(m, 2)))
        nc = int(rng.poisson(p.clutter_rate))
        if nc:
            Z.append(p.offset + rng.uniform(0.0, p.extent, size=(nc, 2)))
        Z = np.concatenate(Z, axis=0) if Z else np.zeros((0, 2))
        Z = Z[rng.permutation(len(Z))].astype(np.float32)
        ids = np.array(sorted(alive), dtype=np.int64)
        truth = np.array([alive[i] for i in ids]) if len(ids) else np.zeros((0, 5))
        frames.append(Frame(Z=Z, births=births, truth=truth, truth_ids=ids))
    return Scene(params=p, seed=seed, frames=frames)


def ctrv_filter_config(params: CtrvParams, seed: int, **overrides) -> dict:
    """The particle filter's configuration for a CTRV scene (model 1)."""
    p = params
    cfg = dict(dim_x=5, dim_z=2, dt=float(np.float32(p.dt)), q=0.0,
               R=(p.sigma ** 2 * np.eye(2)).tolist(), p_s=p.p_s, p_d=p.p_d, lambda_d=p.lambda_d,
               clutter_rate=p.clutter_rate if p.filter_clutter_rate is None else p.filter_clutter_rate,
               volume=p.extent ** 2, gate=chi2_gate(2, p.gate_tail),
               h_max=p.h_max, h_up=p.h_up, tau=p.tau, seed=(seed ^ 0x5EED) & ((1 << 64) - 1),
               score_mode=1, model=1, n_particles=p.n_particles, sigma_a=p.sigma_a,
               sigma_w=p.filter_sigma_w, ess_frac=p.ess_frac)
    cfg.update(overrides)
    return cfg


def chi2_gate(dim_z: int, tail: float = 1e-4) -> float:
    """Mahalanobis gate G: the chi-square(dim_z) quantile at 1 - tail."""
    from scipy.stats import chi2
    return float(chi2.isf(tail, dim_z))


@dataclasses.dataclass
class Frame:
    Z: np.ndarray                 # (M, dim) float32, shuffled
    births: List[Tuple[float, np.ndarray, np.ndarray]]   # (r, mean (2dim,), cov (2dim,2dim)) float64
    truth: np.ndarray             # (n_alive, 2dim) float64
    truth_ids: np.ndarray         # (n_alive,) int


@dataclasses.dataclass
class Scene:
    params: SceneParams
    seed: int
    frames: List[Frame]

    @property
    def dim_x(self) -> int:
        return 5 if isinstance(self.params, CtrvParams) else 2 * self.params.dim

    @property
    def dim_z(self) -> int:
        return self.params.dim

    def filter_config(self, **overrides) -> dict:
        """Model parameters of the world, as the filter's configuration."""
        p = self.params
        if isinstance(p, CtrvParams):
            return ctrv_filter_config(p, self.seed, **overrides)
        cfg = dict(dim_x=2 * p.dim, dim_z=p.dim, dt=float(np.float32(p.dt)), q=p.q,
                   R=(p.sigma ** 2 * np.eye(p.dim)).tolist(), p_s=p.p_s, p_d=p.p_d,
                   lambda_d=p.lambda_d,
                   clutter_rate=p.clutter_rate if p.filter_clutter_rate is None else p.filter_clutter_rate,
                   volume=p.extent ** p.dim, gate=chi2_gate(p.dim, p.gate_tail),
                   h_max=p.h_max, h_up=p.h_up, tau=p.tau,
                   seed=(self.seed ^ 0x5EED) & ((1 << 64) - 1), score_mode=0)
        cfg.update(overrides)
        return cfg


def _cv_matrices(dim: int, dt: float, q: float):
    """Transition and process-noise covariance used only to *simulate* truth."""
    I = np.eye(dim)
    F = np.block([[I, dt * I], [np.zeros((dim, dim)), I]])
    Q = q * np.block([[dt ** 3 / 3 * I, dt ** 2 / 2 * I], [dt ** 2 / 2 * I, dt * I]])
    return F, Q


def _random_velocity(rng, dim, speed_max):
    speed = rng.uniform(0.0, speed_max)
    d = rng.normal(size=dim)
    d /= np.linalg.norm(d)
    return speed * d


def make_scene(params: SceneParams, seed: int) -> Scene:
    """Draw a full scene (truth, detections, clutter, births) from ``seed``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = params
    dim = p.dim
    F, Q = _cv_matrices(dim, p.dt, p.q)
    Lq = np.linalg.cholesky(Q + 1e-12 * np.eye(2 * dim))

    # birth frames
    if p.birth_window is not None:
        lo, hi = p.birth_window
        t_birth = [int(rng.integers(lo, hi + 1)) for _ in range(p.n_objects)]
    else:
        t_birth = [0] * p.n_objects
        for f in range(1, p.frames):
            t_birth += [f] * int(rng.poisson(p.births_per_frame))
    n_total = len(t_birth)

    alive = {}          # id -> state
    dead = set()
    next_id = 0
    order = sorted(range(n_total), key=lambda j: t_birth[j])
    born_ptr = 0
    frames: List[Frame] = []
    sb = 2.0 * p.sigma
    birth_cov = np.diag([sb ** 2] * dim + [p.birth_vel_std ** 2] * dim)
    for f in range(p.frames):
        # survival + motion of existing objects
        for oid in sorted(alive):
            if rng.uniform() >= p.p_s:
                dead.add(oid)
                del alive[oid]
                continue
            alive[oid] = F @ alive[oid] + Lq @ rng.normal(size=2 * dim)
        # appearances
        births = []
        while born_ptr < n_total and t_birth[order[born_ptr]] == f:
            pos = rng.uniform(0.0, p.extent, size=dim)
            vel = _random_velocity(rng, dim, p.speed_max)
            x = np.concatenate([pos, vel])
            alive[next_id] = x
            mean = np.concatenate([pos + rng.normal(scale=sb, size=dim), np.zeros(dim)])
            births.append((p.r_birth, mean, birth_cov.copy()))
            next_id += 1
            born_ptr += 1
        for _ in range(int(rng.poisson(p.false_births))):
            mean = np.concatenate([rng.uniform(0.0, p.extent, size=dim), np.zeros(dim)])
            births.append((p.r_false, mean, birth_cov.copy()))
        # detections
        Z = []
        for oid in sorted(alive):
            if rng.uniform() < p.p_d:
                m = 1 + int(rng.poisson(p.lambda_d))
                Z.append(alive[oid][:dim] + p.sigma * rng.normal(size=(m, dim)))
        nc = int(rng.poisson(p.clutter_rate))
        if nc:
            Z.append(rng.uniform(0.0, p.extent, size=(nc, dim)))
        Z = np.concatenate(Z, axis=0) if Z else np.zeros((0, dim))
        Z = Z[rng.permutation(len(Z))].astype(np.float32)
        ids = np.array(sorted(alive), dtype=np.int64)
        truth = np.array([alive[i] for i in ids]) if len(ids) else np.zeros((0, 2 * dim))
        frames.append(Frame(Z=Z, births=births, truth=truth, truth_ids=ids))
    return Scene(params=p, seed=seed, frames=frames)


def random_state(rng: np.random.Generator, dim: int, H: int, n_labels: int,
                 extent: float, frame: int, keep: float = 0.8, spread: float = 5.0):
    """A synthetic GLMB state: ``H`` hypotheses over ``n_labels`` labelled
    tracks.  Each hypothesis keeps each label with probability ``keep`` and
    carries its own jittered copy of the track density, so hypotheses share
    labels but not means.  Returns plain arrays (log-weights normalised,
    hypothesis uids, per-hypothesis track lists).
    """
    dx = 2 * dim
    base = np.concatenate([rng.uniform(0, extent, size=(n_labels, dim)),
                           rng.uniform(-8, 8, size=(n_labels, dim))], axis=1)
    labels = [(int(rng.integers(0, max(frame, 1))), j) for j in range(n_labels)]
    labels = sorted(set(labels))
    n_labels = len(labels)
    logw = rng.normal(scale=2.0, size=H)
    logw -= np.log(np.sum(np.exp(logw - logw.max()))) + logw.max()
    uids = rng.integers(0, 2 ** 63, size=H, dtype=np.int64).astype(np.uint64)
    hyps = []
    for h in range(H):
        keep_mask = rng.uniform(size=n_labels) < keep
        tr = []
        for j in np.nonzero(keep_mask)[0]:
            A = rng.normal(size=(dx, dx))
            P = np.diag([spread ** 2] * dim + [2.0 ** 2] * dim) + 0.3 * A @ A.T
            mean = base[j % len(base)] + rng.normal(scale=spread, size=dx) * 0.2
            tr.append((labels[j][0], labels[j][1], mean, P))
        hyps.append(tr)
    return logw, uids, hyps


GATE_NPARAM = 8779


def gate_params(seed: int, mu=None, sd=None, scale: float = 1.0, bias: float = 0.0) -> np.ndarray:
    """Seeded parameters of the gate's 5-64-64-64-1 MLP (float32, layout
    W1[64][5] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] w4[64] b4 mu[5]
    sd[5]): each matrix N(0, scale^2 / fan_in), biases N(0, 0.1^2), the
    output bias `bias`, standardisation mu (default 0) and sd (default 1)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, n_out in ((5, 64), (64, 64), (64, 64)):
        parts.append(rng.normal(scale=scale / np.sqrt(fan_in), size=(n_out, fan_in)).ravel())
        parts.append(rng.normal(scale=0.1, size=n_out))
    parts.append(rng.normal(scale=scale / 8.0, size=64))
    parts.append(np.array([bias]))
    parts.append(np.zeros(5) if mu is None else np.asarray(mu, np.float64))
    parts.append(np.ones(5) if sd is None else np.asarray(sd, np.float64))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == GATE_NPARAM
    return p
