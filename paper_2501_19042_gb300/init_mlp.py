"""Learned initialisation of the safety filter (Sec. III-C, "Learned
Initialization for SF"; Eq. NN_loss), reduced to a 3-layer MLP.

The network maps (starts, goals, xi_bar) of one sample to the SF's initial
iterate (xi^0, lambda^0) and is trained self-supervised through the unrolled
solver, whose gradient comes from the hand-written adjoint kernel
(``sf_project_backward``). Loss per sample (Eq. NN_loss as read here):

    L = w * sum_{k<K} ||z^{k+1} - z^k||^2 + ||xi^K - xi_bar||^2,  z = (xi, lambda).

The output layer is residual and starts at zero, so the untrained network is
exactly the sample initialisation (xi^0 = xi_bar, lambda^0 = 0), which stays
the fallback: ``project_with_fallback`` keeps, per sample, whichever start
gives the smaller final primal residual.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import torch
from torch import nn

import swarm_inputs as si

from .autograd import sf_unroll


class InitMLP(nn.Module):
    """[start, goal, xi_bar] -> (xi^0, lambda^0); width 256, float32."""

    def __init__(self, n_robots: int, dim: int = 3, nvar: int = 11, width: int = 256, scale: float = 4.0):
        super().__init__()
        self.N, self.dim, self.nvar, self.scale = n_robots, dim, nvar, scale
        self.n = dim * n_robots * nvar
        n_in = 2 * n_robots * dim + self.n
        self.net = nn.Sequential(nn.Linear(n_in, width), nn.LeakyReLU(0.1), nn.Linear(width, width),
                                 nn.LeakyReLU(0.1), nn.Linear(width, 2 * self.n))
        nn.init.zeros_(self.net[-1].weight)
        nn.init.zeros_(self.net[-1].bias)

    def forward(self, start_s, goal_s, xi_bar):
        """start_s, goal_s: [S, N, dim] (each sample's scene); xi_bar: [S, dim, N, nvar]."""
        S = xi_bar.shape[0]
        x = torch.cat([start_s.reshape(S, -1), goal_s.reshape(S, -1), xi_bar.reshape(S, -1)], 1) / self.scale
        y = self.net(x) * self.scale
        xi0 = xi_bar + y[:, : self.n].reshape(xi_bar.shape)
        lam0 = y[:, self.n:].reshape(xi_bar.shape)
        return xi0.contiguous(), lam0.contiguous()


class InitPointNet(nn.Module):
    """The paper's initialisation network (Sec. IV, "Initialization Network
    Details"): a PointNet-like CNN over the agents, whose 18 input channels
    are the start and goal position, velocity and acceleration of an agent in
    3D, max-pooled over the agents into a feature vector c; c concatenated
    with the sample xi_bar goes through a 4-layer MLP (linear, batch
    normalisation, LeakyReLU). Same residual output as ``InitMLP`` (zero last
    layer: untrained, it is the sample initialisation). Velocities and
    accelerations at the boundary are zero in these workloads."""

    def __init__(self, n_robots: int, dim: int = 3, nvar: int = 11, width: int = 512, feat: int = 256,
                 scale: float = 4.0):
        super().__init__()
        self.N, self.dim, self.nvar, self.scale = n_robots, dim, nvar, scale
        self.n = dim * n_robots * nvar
        ch = 6 * dim
        self.point = nn.Sequential(nn.Conv1d(ch, 64, 1), nn.BatchNorm1d(64), nn.ReLU(),
                                   nn.Conv1d(64, 128, 1), nn.BatchNorm1d(128), nn.ReLU(),
                                   nn.Conv1d(128, feat, 1))
        self.mlp = nn.Sequential(nn.Linear(feat + self.n, width), nn.BatchNorm1d(width), nn.LeakyReLU(0.1),
                                 nn.Linear(width, width), nn.BatchNorm1d(width), nn.LeakyReLU(0.1),
                                 nn.Linear(width, width), nn.BatchNorm1d(width), nn.LeakyReLU(0.1),
                                 nn.Linear(width, 2 * self.n))
        nn.init.zeros_(self.mlp[-1].weight)
        nn.init.zeros_(self.mlp[-1].bias)

    def forward(self, start_s, goal_s, xi_bar):
        """start_s, goal_s: [S, N, dim]; xi_bar: [S, dim, N, nvar]."""
        S = xi_bar.shape[0]
        z = torch.zeros_like(start_s)
        states = torch.cat([start_s, z, z, goal_s, z, z], 2) / self.scale      # [S, N, 6 dim]
        c = self.point(states.transpose(1, 2)).amax(2)                         # [S, feat]
        y = self.mlp(torch.cat([c, xi_bar.reshape(S, -1) / self.scale], 1)) * self.scale
        xi0 = xi_bar + y[:, : self.n].reshape(xi_bar.shape)
        lam0 = y[:, self.n:].reshape(xi_bar.shape)
        return xi0.contiguous(), lam0.contiguous()


def make_init_net(arch: str, n_robots: int, dim: int = 3):
    """``mlp``: the 3-layer MLP; ``pointnet``: the paper's network."""
    if arch == "mlp":
        return InitMLP(n_robots, dim)
    if arch == "pointnet":
        return InitPointNet(n_robots, dim)
    raise ValueError(f"unknown init network {arch!r}")


@dataclass
class SceneBatch:
    xi_bar: torch.Tensor     # [S_total, dim, N, nvar]
    start: torch.Tensor      # [n_scenes * N, dim]
    goal: torch.Tensor
    start_s: torch.Tensor    # [S_total, N, dim] per sample
    goal_s: torch.Tensor
    n_robots: list
    n_samples: list


def make_batch(spec: si.SceneSpec, seed: int, n_scenes: int, device) -> SceneBatch:
    """n_scenes seeded scenes of `spec` (each with spec.n_samples samples)."""
    st = si.Stream(seed)
    scenes = [si.make_scene(spec, st) for _ in range(n_scenes)]
    S = spec.n_samples
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
    xb = t(np.concatenate([s.xi_bar for s in scenes]))
    start = np.concatenate([s.start for s in scenes])
    goal = np.concatenate([s.goal for s in scenes])
    ss = np.repeat(np.stack([s.start for s in scenes]), S, axis=0)
    gs = np.repeat(np.stack([s.goal for s in scenes]), S, axis=0)
    return SceneBatch(xb, t(start), t(goal), t(ss), t(gs), [spec.n_robots] * n_scenes, [S] * n_scenes)


def nn_loss(sf, mlp, b: SceneBatch, K: int, fp_weight: float):
    xi0, lam0 = mlp(b.start_s, b.goal_s, b.xi_bar)
    xi, lam, fp, res = sf_unroll(sf, b.xi_bar, b.start, b.goal, K, xi0=xi0, lam0=lam0,
                                 n_robots=b.n_robots, n_samples=b.n_samples)
    dev = ((xi - b.xi_bar) ** 2).flatten(1).sum(1)
    per = fp_weight * fp + dev
    return per.mean(), res


def train(sf, mlp, spec: si.SceneSpec, K: int = 50, n_train_scenes: int = 20000, scenes_per_step: int = 64,
          epochs: int = 1, lr: float = 1e-3, fp_weight: float = 1.0, seed: int = 4, max_steps: int | None = None,
          log_every: int = 50, verbose: bool = False):
    """Trains over n_train_scenes seeded scenes (stream `seed`, split into
    consecutive batches of scenes_per_step scenes). Returns the loss history."""
    dev = sf.device
    opt = torch.optim.Adam(mlp.parameters(), lr=lr)
    steps_per_epoch = max(1, n_train_scenes // scenes_per_step)
    hist = []
    step = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        for q in range(steps_per_epoch):
            if max_steps is not None and step >= max_steps:
                return hist
            b = make_batch(spec, seed * 1_000_003 + q, scenes_per_step, dev)
            loss, res = nn_loss(sf, mlp, b, K, fp_weight)
            opt.zero_grad(set_to_none=True)
            loss.backward()
            opt.step()
            hist.append(float(loss.detach()))
            if verbose and step % log_every == 0:
                print(f"step {step} loss {hist[-1]:.4f} median residual {float(res.median()):.2e} "
                      f"({time.perf_counter() - t0:.1f} s)", flush=True)
            step += 1
    return hist


@torch.no_grad()
def evaluate(sf, mlp, spec: si.SceneSpec, K: int, seed: int = 5, n_scenes: int = 64):
    """Final ||r_p|| after K iterations on held-out scenes for the sample,
    zero and learned initialisations, and the per-sample fallback choice."""
    b = make_batch(spec, seed * 1_000_003, n_scenes, sf.device)
    kw = dict(n_robots=b.n_robots, n_samples=b.n_samples)
    r_sample = sf.project(b.xi_bar, b.start, b.goal, K, **kw).residual
    r_zero = sf.project(b.xi_bar, b.start, b.goal, K, xi0=torch.zeros_like(b.xi_bar),
                        lam0=torch.zeros_like(b.xi_bar), **kw).residual
    was = mlp.training
    mlp.eval()
    xi0, lam0 = mlp(b.start_s, b.goal_s, b.xi_bar)
    mlp.train(was)
    r_learn = sf.project(b.xi_bar, b.start, b.goal, K, xi0=xi0, lam0=lam0, **kw).residual
    r_fb = torch.minimum(r_learn, r_sample)
    q = lambda r: {"median": float(r.median()), "p90": float(r.quantile(0.9)), "mean": float(r.mean())}
    return {"sample_init": q(r_sample), "zero_init": q(r_zero), "learned_init": q(r_learn),
            "learned_with_fallback": q(r_fb), "learned_better_frac": float((r_learn < r_sample).float().mean()),
            "n_samples": int(r_sample.numel()), "K": K}


@torch.no_grad()
def residual_curves(sf, nets: dict, spec: si.SceneSpec, K: int, seed: int = 5, n_scenes: int = 64,
                    at=(1, 2, 5, 10, 20, 50, 100, 200)):
    """Median projection residual ||F xi^k - e^{k+1}|| across held-out samples
    at iterations `at` (the per-iteration history of sf_project) for the zero
    and sample initialisations and each trained network in `nets` (name ->
    module, evaluated in eval mode), as in the paper's residual figure."""
    b = make_batch(spec, seed * 1_000_003, n_scenes, sf.device)
    kw = dict(n_robots=b.n_robots, n_samples=b.n_samples, hist=True)
    inits = {"zero": (torch.zeros_like(b.xi_bar), torch.zeros_like(b.xi_bar)), "sample": (None, None)}
    for name, net in nets.items():
        was = net.training
        net.eval()
        inits[name] = net(b.start_s, b.goal_s, b.xi_bar)
        net.train(was)
    out = {}
    for name, (x0, l0) in inits.items():
        r = sf.project(b.xi_bar, b.start, b.goal, K, xi0=x0, lam0=l0, **kw)
        med = r.hist.median(dim=1).values.cpu()
        out[name] = {str(k): float(med[k - 1]) for k in at if k <= K}
        out[name]["final_rp_median"] = float(r.residual.median())
    return out


@torch.no_grad()
def project_with_fallback(sf, mlp, xi_bar, start, goal, start_s, goal_s, K, n_robots=None, n_samples=None):
    """Runs the SF from the learned and from the sample initialisation and
    keeps, per sample, the result with the smaller final primal residual."""
    kw = dict(n_robots=n_robots, n_samples=n_samples)
    a = sf.project(xi_bar, start, goal, K, **kw)
    was = mlp.training
    mlp.eval()
    xi0, lam0 = mlp(start_s, goal_s, xi_bar)
    mlp.train(was)
    b = sf.project(xi_bar, start, goal, K, xi0=xi0, lam0=lam0, **kw)
    pick = (b.residual < a.residual)
    shape = (-1,) + (1,) * (xi_bar.dim() - 1)
    xi = torch.where(pick.view(shape), b.xi, a.xi)
    lam = torch.where(pick.view(shape), b.lam, a.lam)
    return xi, lam, torch.where(pick, b.residual, a.residual), pick


def main():
    import argparse
    import json

    from .safety_filter import SafetyFilter
    ap = argparse.ArgumentParser(description="train the learned SF initialisation and report residuals")
    ap.add_argument("--K", type=int, default=50)
    ap.add_argument("--epochs", type=int, default=1)
    ap.add_argument("--scenes", type=int, default=20000)
    ap.add_argument("--scenes-per-step", type=int, default=64)
    ap.add_argument("--samples-per-scene", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--fp-weight", type=float, default=1.0)
    ap.add_argument("--rho", type=float, default=0.1)
    ap.add_argument("--eval-scenes", type=int, default=64)
    ap.add_argument("--arch", default="mlp", choices=["mlp", "pointnet", "both"])
    ap.add_argument("--curves-K", type=int, default=0,
                    help="after training, median residual vs iteration over K iterations for every init")
    args = ap.parse_args()
    spec = si.config_diff(n_samples=args.samples_per_scene, K=args.K)
    sf = SafetyFilter(dim=3, T=spec.T, rho=args.rho, coll_a=spec.coll, v_max=spec.v_max, a_max=spec.a_max,
                      max_robots=spec.n_robots, checkpoint_every=10)
    result, nets = {}, {}
    for arch in (["mlp", "pointnet"] if args.arch == "both" else [args.arch]):
        torch.manual_seed(0)
        net = make_init_net(arch, spec.n_robots).to(sf.device)
        before = evaluate(sf, net, spec, args.K, n_scenes=args.eval_scenes)
        t0 = time.perf_counter()
        hist = train(sf, net, spec, K=args.K, n_train_scenes=args.scenes, scenes_per_step=args.scenes_per_step,
                     epochs=args.epochs, lr=args.lr, fp_weight=args.fp_weight)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        after = evaluate(sf, net, spec, args.K, n_scenes=args.eval_scenes)
        result[arch] = {"train_scenes": args.scenes, "epochs": args.epochs, "steps": len(hist),
                        "train_seconds": dt, "loss_first": hist[0], "loss_last": hist[-1],
                        "heldout_before": before, "heldout_after": after}
        nets[arch] = net
    if args.curves_K > 0:
        cspec = si.config_diff(n_samples=args.samples_per_scene, K=args.curves_K)
        result["residual_curves"] = residual_curves(sf, nets, cspec, args.curves_K, n_scenes=args.eval_scenes)
    print(json.dumps(result))


if __name__ == "__main__":
    main()
