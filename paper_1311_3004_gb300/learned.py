"""Learned sub-grid correction for coarse focused-source runs (not in the paper).

A coarse grid (dx) runs the same scheme as a fine grid (dx/2, dt/2); the
network learns the one-step residual between the coarse step and the fine
solution restricted to the coarse grid, and is then applied after every
coarse step (fvna_set_correction).  Everything the method computes runs in
the library's kernels: the solver steps, the network's forward and backward
passes and its optimiser.  PyTorch only holds device buffers and does the
data plumbing of the training set (restriction to the coarse grid, random
crops).

    X, T = generate(spec, amplitudes)        # solver-made training data
    net, info = train_net(X, T, steps)       # on the GPU, our kernels
    X2, T2 = generate_rollout(spec, amplitudes, net, info)   # on its own trajectory
    result = evaluate(spec, amp, net, info)  # coarse+net vs coarse vs fine
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import fvna
from . import workloads as wl


@dataclass
class Spec:
    """Coarse/fine pair of focused axisymmetric grids (fine = 2x finer)."""
    nz: int            # coarse cells along z
    nr: int            # coarse cells along r
    cpw: float         # coarse cells per wavelength
    aperture_m: float
    focal_m: float
    t_train: float     # training runs end here
    t_end: float       # evaluation runs end here
    sample_every: int  # coarse steps between training samples
    every: int = 1     # the network corrects every `every` coarse steps
    band: int = 0      # cells next to the domain edges left uncorrected
    nu: float = 0.4
    freq: float = 1.0e6

    def workload(self, fine: bool, p_surface: float):
        k = 2 if fine else 1
        return wl.focused_axisym(nz=k * self.nz, nr=k * self.nr, cells_per_wavelength=k * self.cpw,
                                 p_surface=p_surface, aperture_m=self.aperture_m,
                                 focal_m=self.focal_m, freq=self.freq)

    def dt(self, fine: bool) -> float:
        return self.nu / self.cpw / (2 if fine else 1)


SMALL = Spec(nz=256, nr=64, cpw=8.0, aperture_m=9e-3, focal_m=18e-3, t_train=30.0, t_end=40.0,
             sample_every=10)
FULL = Spec(nz=2048, nr=512, cpw=15.0, aperture_m=30e-3, focal_m=60e-3, t_train=320.0,
            t_end=320.0, sample_every=200, every=10, band=4)


def _solver(spec: Spec, fine: bool, p_surface: float, q0=None, t0: float = 0.0,
            precision=fvna.FP32_PERT, dt_fixed=True, steps_per_graph=2):
    w = spec.workload(fine, p_surface)
    e = w.extra
    cfg = fvna.make_config(precision=precision, geometry=fvna.AXISYMMETRIC, beta=w.beta,
                           delta=w.delta, dx=w.dx, nu_w=spec.nu,
                           dt_fixed=spec.dt(fine) if dt_fixed else 0.0,
                           steps_per_graph=steps_per_graph)
    dom = fvna.make_domain(w.nx, w.ny, bc=w.bc, envelope=e["envelope"], amp=e["amp"],
                           focal=e["focal"], aperture=e["aperture"], t0=t0)
    return fvna.Solver(cfg, [dom], [w.q0 if q0 is None else q0]), w


def _pert(torch, q):
    """(3, ny, nx) total variables (float64) -> perturbation (float32)."""
    p = q.clone()
    p[0] -= 1.0
    return p.to(torch.float32)


def restrict(torch, pf, dx_fine):
    """r-weighted 2x2 average of fine perturbation fields onto the coarse grid
    (cell volumes grow like r in the axisymmetric form)."""
    import torch.nn.functional as F
    nr = pf.shape[-2]
    r = (torch.arange(nr, device=pf.device, dtype=torch.float64) + 0.5) * dx_fine
    num = F.avg_pool2d((pf.double() * r[:, None]).unsqueeze(0), 2).squeeze(0)
    den = F.avg_pool2d(r[:, None].expand(nr, pf.shape[-1]).unsqueeze(0).unsqueeze(0), 2)[0, 0]
    return (num / den).to(torch.float32)


def generate(spec: Spec, amplitudes, log=print):
    """Training samples (X, T): X = `every` coarse steps from the restricted
    fine state, T = the restricted fine state at the same time minus X."""
    import torch
    xs, ts = [], []
    dxf = spec.workload(True, 1.0).dx
    for a in amplitudes:
        t0 = time.perf_counter()
        sf, wf = _solver(spec, True, a, steps_per_graph=2 * spec.sample_every)
        qf = torch.empty((3, wf.ny, wf.nx), dtype=torch.float64, device="cuda")
        t_now, k = 0.0, 0
        k_ = spec.every
        while t_now < spec.t_train:
            sf.run(max_steps=2 * max(spec.sample_every - k_, 0))
            st = sf.stats(0)
            A = restrict(torch, _pert(torch, sf.q(0, out=qf)), dxf)
            ta = st["t"]
            sf.run(max_steps=2 * k_)
            B = restrict(torch, _pert(torch, sf.q(0, out=qf)), dxf)
            t_now = sf.stats(0)["t"]
            qa = A.double()
            qa[0] += 1.0
            sc, _ = _solver(spec, False, a, q0=qa, t0=ta)
            sc.run(max_steps=k_)
            X = _pert(torch, sc.q(0, out=torch.empty_like(qa)))
            sc.close()
            xs.append(X)
            ts.append(B - X)
            k += 1
        sf.close()
        if log:
            log(f"  amplitude {a / 1e6:.2f} MPa: {k} samples, {time.perf_counter() - t0:.1f} s")
    return torch.stack(xs), torch.stack(ts)


def generate_rollout(spec: Spec, amplitudes, net, info, gain=0.5, log=print):
    """Training samples on the corrected coarse run's own trajectory (data
    aggregation): at each sample time t_a the corrected coarse state Y is
    advanced `every` plain coarse steps to X', and the target is the
    restricted fine state at t_a + every coarse steps minus X'.  The network
    so learns to steer the states its own corrections lead to back towards
    the fine solution.  A run whose correction makes it fail stops adding
    samples."""
    import torch
    xs, ts = [], []
    dxf = spec.workload(True, 1.0).dx
    k_ = spec.every
    for a in amplitudes:
        t0 = time.perf_counter()
        sf, wf = _solver(spec, True, a, steps_per_graph=2 * spec.sample_every)
        sc, wc = _solver(spec, False, a, steps_per_graph=spec.sample_every)
        sc.set_correction(net, info["in_scale"], gain * info["out_scale"], spec.every,
                          edge_band=spec.band)
        qf = torch.empty((3, wf.ny, wf.nx), dtype=torch.float64, device="cuda")
        qc = torch.empty((3, wc.ny, wc.nx), dtype=torch.float64, device="cuda")
        t_now, k = 0.0, 0
        while t_now < spec.t_train:
            sf.run(max_steps=2 * max(spec.sample_every - k_, 0))
            st = sc.run(max_steps=max(spec.sample_every - k_, 0), check=False)
            if st["rc"] != 0:
                break
            ta = sc.stats(0)["t"]
            Y = sc.q(0, out=qc).clone()
            sf.run(max_steps=2 * k_)
            B = restrict(torch, _pert(torch, sf.q(0, out=qf)), dxf)
            sx, _ = _solver(spec, False, a, q0=Y, t0=ta)
            sx.run(max_steps=k_)
            X = _pert(torch, sx.q(0, out=torch.empty_like(Y)))
            sx.close()
            st = sc.run(max_steps=k_, check=False)
            t_now = sf.stats(0)["t"]
            xs.append(X)
            ts.append(B - X)
            k += 1
            if st["rc"] != 0:
                break
        sf.close()
        sc.close()
        if log:
            log(f"  rollout at {a / 1e6:.2f} MPa: {k} samples, {time.perf_counter() - t0:.1f} s")
    return torch.stack(xs), torch.stack(ts)


def _init_params(seed: int):
    """He-style seeded initial weights, the last layer scaled down."""
    rng = np.random.default_rng(seed)
    flat = []
    for (o, c) in [(32, 3), (32, 32), (3, 32)]:
        std = np.sqrt(2.0 / (9 * c)) * (0.1 if o == 3 else 1.0)
        flat.append(rng.normal(0.0, std, size=(o, c, 3, 3)).reshape(-1))
        flat.append(np.zeros(o))
    return np.concatenate(flat).astype(np.float32)


def _bias_slices():
    """Index ranges of b1, b2, b3 in the flat parameter layout
    (w1 b1 w2 b2 w3 b3, [out][in][row][col])."""
    out, o = [], 0
    for (co, ci) in [(32, 3), (32, 32), (3, 32)]:
        o += co * ci * 9
        out.append(slice(o, o + co))
        o += co
    return out


def train_net(X, T, steps=1500, batch=8, crop=96, lr=1e-3, margin=4, seed=0, noise=0.0,
              importance=False, bias=True, log=print):
    """Train a fresh network on random crops of (X, T); returns (net, info).
    in_scale normalises the state, out_scale the residual.  Crops are drawn
    with probability proportional to the residual energy they contain (plus
    a floor) if importance, since the residual is concentrated where the
    wave is; otherwise uniformly.  With
    noise > 0 the inputs get Gaussian noise of that many standard deviations
    of X, so the network tolerates the drift of a corrected run.  With bias
    False the biases stay zero (they are reset after every step): the ReLU
    network then maps a field at rest to no correction, so a corrected run
    cannot drift where there is no wave."""
    import torch
    import torch.nn.functional as F
    g = torch.Generator(device="cpu").manual_seed(seed)
    in_scale = float(1.0 / X.std())
    out_scale = float(T.std())
    net = fvna.Net(_init_params(seed))
    n, _, H, W = X.shape
    ch, cw = min(crop, H), min(crop, W)
    # residual energy of every crop position (stride 8), as sampling weights
    e = F.avg_pool2d((T * T).sum(dim=1, keepdim=True), (ch, cw), stride=8)[:, 0]
    wts = (e + 0.05 * e.mean()).reshape(-1).double().cpu()
    gh, gw = e.shape[1], e.shape[2]
    last_i, last_j = H - ch, W - cw
    losses = []
    t0 = time.perf_counter()
    for it in range(steps):
        if importance:
            pick = torch.multinomial(wts, batch, replacement=True, generator=g)
            idx = pick // (gh * gw)
            i0 = torch.clamp((pick // gw) % gh * 8 + torch.randint(0, 8, (batch,), generator=g),
                             0, last_i)
            j0 = torch.clamp(pick % gw * 8 + torch.randint(0, 8, (batch,), generator=g),
                             0, last_j)
        else:
            idx = torch.randint(0, n, (batch,), generator=g)
            i0 = torch.randint(0, H - ch + 1, (batch,), generator=g)
            j0 = torch.randint(0, W - cw + 1, (batch,), generator=g)
        xb = torch.stack([X[idx[b], :, i0[b]:i0[b] + ch, j0[b]:j0[b] + cw] for b in range(batch)])
        tb = torch.stack([T[idx[b], :, i0[b]:i0[b] + ch, j0[b]:j0[b] + cw] for b in range(batch)])
        if noise > 0:
            xb = xb + (noise / in_scale) * torch.randn(xb.shape, generator=g).to(xb.device)
        # the loss covers the cells at least `margin` from every crop edge;
        # the correction is applied on the same band of the full field
        # (at least `margin` from every domain edge)
        edges = None
        lr_t = lr * (0.1 ** (it / steps))
        losses.append(net.train_step(xb.contiguous(), (tb / out_scale).contiguous(), lr_t,
                                     in_scale=in_scale, margin=margin, edges=edges))
        if not bias:
            p = net.params()
            for sl in _bias_slices():
                p[sl] = 0.0
            net.set_params(p)
        if log and (it % max(1, steps // 5) == 0 or it == steps - 1):
            log(f"  step {it}: loss {np.mean(losses[-50:]):.4e}")
    info = {"in_scale": in_scale, "out_scale": out_scale, "margin": margin, "bias": bias,
            "loss_first": float(np.mean(losses[:50])),
            "loss_last": float(np.mean(losses[-50:])), "seconds": time.perf_counter() - t0,
            "steps": steps}
    return net, info


def reference(spec: Spec, p_surface: float, t_end=None, fine_precision=fvna.FP64):
    """The fine-grid run restricted to the coarse grid: (restricted pressure
    perturbation on the CPU, binary64; its maximum; run seconds)."""
    import torch
    t_end = spec.t_end if t_end is None else t_end
    dxf = spec.workload(True, 1.0).dx
    s, w = _solver(spec, True, p_surface, precision=fine_precision, steps_per_graph=64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.run(t_end=t_end)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    pf = torch.from_numpy(s.q(0))
    s.close()
    pfr = restrict(torch, _pert(torch, pf.cuda()), dxf)[0].cpu().double()
    return pfr, float(pfr.max()), sec


def evaluate(spec: Spec, p_surface: float, net=None, info=None, fine_precision=fvna.FP64,
             t_end=None, gains=(1.0,), fine32=False, ref=None):
    """Run coarse (with and without the network) and fine to t_end; return the
    focal peak pressures, errors against the fine run and the run times;
    with fine32 also the fine grid in binary32 (the fastest plain solver of
    the same accuracy) against the same reference."""
    import torch
    t_end = spec.t_end if t_end is None else t_end
    out = {}
    dxf = spec.workload(True, 1.0).dx
    runs = [("coarse", 0.0)] + ([(f"coarse_net" if g == 1.0 else f"coarse_net_gain{g}", g)
                                 for g in gains] if net is not None else [])
    for name, gain in runs:
        use_net = gain > 0
        s, w = _solver(spec, False, p_surface, steps_per_graph=64)
        if use_net:
            s.set_correction(net, info["in_scale"], gain * info["out_scale"], spec.every,
                             edge_band=spec.band)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = s.run(t_end=t_end, check=False)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "p": torch.from_numpy(s.pressure(0)),
                     "status": st["rc"]}
        s.close()
    pfr, peak_f, fine_s = ref if ref is not None else reference(spec, p_surface, t_end,
                                                                 fine_precision)
    out["fine"] = {"seconds": fine_s}
    res = {"t_end": t_end, "p_surface": p_surface, "focal_peak_fine": peak_f,
           "fine_seconds": out["fine"]["seconds"]}
    if fine32:
        s, w = _solver(spec, True, p_surface, precision=fvna.FP32_PERT, steps_per_graph=64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = s.run(t_end=t_end, check=False)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        p32 = restrict(torch, _pert(torch, torch.from_numpy(s.q(0)).cuda()), dxf)[0].cpu().double()
        s.close()
        res["fine_fp32"] = {"seconds": sec, "status": st["rc"],
                            "focal_peak_rel_err": abs(float(p32.max()) - peak_f) / peak_f,
                            "l2_rel_err": float(torch.linalg.norm(p32 - pfr) /
                                                torch.linalg.norm(pfr))}
    for name in out:
        if name == "fine":
            continue
        p = out[name]["p"].double()
        if out[name]["status"] != 0:
            res[name] = {"seconds": out[name]["seconds"], "status": out[name]["status"],
                         "focal_peak_rel_err": float("inf"), "l2_rel_err": float("inf")}
            continue
        res[name] = {"seconds": out[name]["seconds"], "status": 0,
                     "focal_peak": float(p.max()),
                     "focal_peak_rel_err": abs(float(p.max()) - peak_f) / peak_f,
                     "l2_rel_err": float(torch.linalg.norm(p - pfr) / torch.linalg.norm(pfr))}
    return res
