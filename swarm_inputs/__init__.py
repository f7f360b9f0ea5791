"""Seeded synthetic swarm workloads shared by the oracle tests, the GPU tests
and the benchmark.

This module holds none of the safety filter's arithmetic: it only draws
random numbers and lays them out. Both the FP64 oracle and the CUDA path take
its arrays as inputs; neither is imported here.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: output i of stream ``seed`` is mix(seed + (i + 1) * golden_gamma).
Uniforms take the top 53 bits; normals use the Box-Muller transform
(cosine branch) on two uniforms.

Scene recipe (stands in for the paper's generator outputs, which need its
trained CVAE / VQ-VAE and dataset, Sec. V-A):
  * starts and goals: either on a circle with goals at the antipodes, or
    uniform in a box centred at the origin with a minimum pairwise
    separation (rejection sampling, starts first, then goals);
  * sampled coefficients xi_bar: the straight line from start to goal in
    Bernstein form, c_k = s + (k / order) (g - s), plus i.i.d. N(0, sigma^2)
    noise on every coefficient of every robot and axis;
  * draw order: scene-major; within a scene: starts, goals, then samples in
    the order sample -> axis -> robot -> k.
"""
from __future__ import annotations

from dataclasses import dataclass, asdict

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream ``seed``."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def uniform(self, n: int) -> np.ndarray:
        z = splitmix64(self.seed, self.pos, n)
        self.pos += n
        return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        u = self.uniform(2 * n).reshape(n, 2)
        r = np.sqrt(-2.0 * np.log(1.0 - u[:, 0]))
        return r * np.cos(2.0 * np.pi * u[:, 1])


@dataclass
class SceneSpec:
    dim: int = 3
    n_robots: int = 16
    n_samples: int = 1024
    T: int = 100
    order: int = 10
    t_final: float = 5.0
    radius: float = 0.25          # robot radius; collision semi-axes a = b = 2 r
    v_max: float = 2.0
    a_max: float = 3.0
    layout: str = "box"           # "box" or "circle"
    box: tuple = (8.0, 8.0, 4.0)  # full edge lengths
    min_sep: float = 1.0
    circle_radius: float = 3.0
    sigma: float = 0.8
    K: int = 200
    init: str = "sample"          # "sample" (xi0 = xi_bar, lambda0 = 0) or "zero"
    rho: float = 1.0

    @property
    def coll(self) -> float:
        return 2.0 * self.radius

    @property
    def nvar(self) -> int:
        return self.order + 1


@dataclass
class Scene:
    spec: SceneSpec
    start: np.ndarray     # [N][dim]
    goal: np.ndarray      # [N][dim]
    xi_bar: np.ndarray    # [S][dim][N][nvar]

    @property
    def xi0(self):
        if self.spec.init == "zero":
            return np.zeros_like(self.xi_bar)
        return None


def _points_box(st: Stream, n: int, dim: int, box, min_sep: float, max_tries: int = 200000):
    half = np.asarray(box[:dim], dtype=np.float64) / 2.0
    pts = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place robots with the requested separation")
        c = (st.uniform(dim) * 2.0 - 1.0) * half
        if all(np.linalg.norm(c - p) >= min_sep for p in pts):
            pts.append(c)
    return np.array(pts)


def make_scene(spec: SceneSpec, st: Stream) -> Scene:
    N, dim = spec.n_robots, spec.dim
    if spec.layout == "circle":
        ang = 2.0 * np.pi * np.arange(N) / N
        start = np.zeros((N, dim))
        start[:, 0] = spec.circle_radius * np.cos(ang)
        start[:, 1] = spec.circle_radius * np.sin(ang)
        goal = -start
    else:
        start = _points_box(st, N, dim, spec.box, spec.min_sep)
        goal = _points_box(st, N, dim, spec.box, spec.min_sep)
    k = np.arange(spec.nvar) / spec.order
    line = start.T[:, :, None] + k[None, None, :] * (goal - start).T[:, :, None]  # [dim][N][nvar]
    noise = st.normal(spec.n_samples * dim * N * spec.nvar).reshape(spec.n_samples, dim, N, spec.nvar)
    xi_bar = line[None] + spec.sigma * noise
    return Scene(spec, start, goal, xi_bar)


def scene(spec: SceneSpec, seed: int) -> Scene:
    return make_scene(spec, Stream(seed))


# --- the workloads -------------------------------------------------------------

def config_small_2d(**kw) -> SceneSpec:
    """1 scene, 2D, N=4 on a circle of radius 3 m, goals at the antipodes,
    robot radius 0.3 m, S=16, sigma 0.5, T=100 over 5 s, K=100, zero init."""
    base = dict(dim=2, n_robots=4, n_samples=16, T=100, radius=0.3, layout="circle",
                circle_radius=3.0, sigma=0.5, K=100, init="zero")
    base.update(kw)
    return SceneSpec(**base)


def config_n16_3d(**kw) -> SceneSpec:
    """1 scene, 3D, N=16 uniform in an 8x8x4 m box, >= 1 m separation, robot
    radius 0.25 m, S=1024, sigma 0.8, T=100, K=200, sample init."""
    base = dict(dim=3, n_robots=16, n_samples=1024, T=100, radius=0.25, layout="box",
                box=(8.0, 8.0, 4.0), min_sep=1.0, sigma=0.8, K=200, init="sample")
    base.update(kw)
    return SceneSpec(**base)


def config_n32_3d(**kw) -> SceneSpec:
    """1 scene, 3D, N=32 (496 pairs), S=2048, T=120, K=200, else as the N=16 case."""
    base = dict(dim=3, n_robots=32, n_samples=2048, T=120, radius=0.25, layout="box",
                box=(8.0, 8.0, 4.0), min_sep=1.0, sigma=0.8, K=200, init="sample")
    base.update(kw)
    return SceneSpec(**base)


def config_diff(**kw) -> SceneSpec:
    """N=16, 3D, S=512, T=100, K=50 (differentiation workload)."""
    base = dict(dim=3, n_robots=16, n_samples=512, T=100, radius=0.25, layout="box",
                box=(8.0, 8.0, 4.0), min_sep=1.0, sigma=0.8, K=50, init="sample")
    base.update(kw)
    return SceneSpec(**base)


def ragged_batch(seed: int, n_scenes: int = 64, n_lo: int = 8, n_hi: int = 32, s_lo: int = 128,
                 s_hi: int = 512, K: int = 150, **kw):
    """Many scenes with uneven swarm sizes and sample counts: N ~ U{n_lo..n_hi},
    S ~ U{s_lo..s_hi}, 3D, T=100, otherwise as the N=16 case. The sizes are
    drawn first (2 uniforms per scene), then the scenes in order."""
    st = Stream(seed)
    u = st.uniform(2 * n_scenes).reshape(n_scenes, 2)
    Ns = (n_lo + np.floor(u[:, 0] * (n_hi - n_lo + 1))).astype(int)
    Ss = (s_lo + np.floor(u[:, 1] * (s_hi - s_lo + 1))).astype(int)
    scenes = []
    for N, S in zip(Ns, Ss):
        spec = config_n16_3d(n_robots=int(N), n_samples=int(S), K=K, **kw)
        scenes.append(make_scene(spec, st))
    return scenes


def spec_dict(spec: SceneSpec) -> dict:
    return asdict(spec)
