"""Training recipe of the learned shock sensor (orchestration only; every numerical step runs in
libosbli.so kernels through the C ABI).

collect(): runs a TENO5 problem with the GPU solver and, at snapshot times, gathers the
per-cell features (osbli_sensor_features) and TENO cut-off labels (osbli_sensor_labels) into
device tensors.  train(): Adam on the GPU (osbli_mlp_train).
"""
import numpy as np

from . import inputs as I
from . import osbli


def collect(cfg, U, nsnap, steps_between, precision=osbli.OSBLI_MIXED):
    import torch
    s = osbli.Solver(dict(cfg, sensor=0), precision=precision)
    s.set_state(U)
    N = int(np.prod(cfg["n"]))
    feats, labels = [], []
    for k in range(nsnap):
        if k:
            s.step(steps_between)
        f = torch.empty((N, osbli.SENSOR_NFEAT), dtype=torch.bfloat16, device="cuda")
        osbli.osbli_sensor_features(s.h, f)
        lab = torch.empty(N, dtype=torch.uint8, device="cuda")
        osbli.osbli_sensor_labels(s.h, lab)
        feats.append(f)
        labels.append(lab)
    state = s.get_state()
    s.close()
    return torch.cat(feats), torch.cat(labels), state


def default_weights(seed=0):
    rng = np.random.default_rng(seed)
    nf, nh = 135, 32
    W1 = rng.normal(0, np.sqrt(2.0 / nf), (nh, nf))
    W2 = rng.normal(0, np.sqrt(2.0 / nh), (nh, nh))
    w3 = rng.normal(0, np.sqrt(1.0 / nh), nh)
    return np.concatenate([W1.ravel(), np.zeros(nh), W2.ravel(), np.zeros(nh), w3,
                           [0.0]]).astype(np.float32)


def train(feats, labels, steps=1500, batch=4096, lr=3e-3, seed=1, pos_weight=None, w0=None):
    n = int(labels.numel())
    if pos_weight is None:
        pos = float(labels.float().mean().item())
        pos_weight = float(np.clip((1.0 - pos) / max(pos, 1e-3), 1.0, 10.0))
    w = default_weights(seed) if w0 is None else w0
    return osbli.osbli_mlp_train(feats, labels, n, steps, batch, lr, pos_weight, seed, w)


def collect_at(cfg, U, steps, precision=osbli.OSBLI_MIXED):
    """As collect(), with snapshots after each cumulative step count in `steps` (ascending)."""
    import torch
    s = osbli.Solver(dict(cfg, sensor=0), precision=precision)
    s.set_state(U)
    N = int(np.prod(cfg["n"]))
    feats, labels, done = [], [], 0
    for k in steps:
        s.step(int(k) - done)
        done = int(k)
        f = torch.empty((N, osbli.SENSOR_NFEAT), dtype=torch.bfloat16, device="cuda")
        osbli.osbli_sensor_features(s.h, f)
        lab = torch.empty(N, dtype=torch.uint8, device="cuda")
        osbli.osbli_sensor_labels(s.h, lab)
        feats.append(f)
        labels.append(lab)
    s.close()
    return torch.cat(feats), torch.cat(labels)


def tgv_training_set(N=48, Ma=1.25, nsnap=6, steps_between=12):
    """TENO5 TGV snapshots from the analytic field on (the smooth early phase)."""
    cfg, U = I.tgv(N, Ma=Ma, scheme=I.TENO5)
    return collect(cfg, U, nsnap, steps_between)


def tgv_shocklet_training_set(N=128, Ma=1.25, times=(1.5, 2.0, 2.5, 3.0, 3.5)):
    """TENO5 TGV snapshots in the shocklet phase (Ma 1.25 forms shocklets from t ~ 1.5 on), the
    state advanced by the mixed form between snapshots."""
    cfg, U = I.tgv(N, Ma=Ma, scheme=I.TENO5)
    steps = [int(round(t / cfg["dt"])) for t in times]
    f, lab = collect_at(cfg, U, steps)
    return f, lab, "TGV %d^3 Ma %.2f at t = %s" % (N, Ma, ", ".join("%.1f" % t for t in times))


SBLI_TRAIN_DESC = ("shock / boundary-layer box 96x48x8 on 60x20x4 (Mach 2, Re 1e4, 10 deg shock from "
                   "x=10), 5 snapshots every 1200 steps")


def sbli_training_set(nsnap=5, steps_between=1200):
    """TENO5 snapshots of a reduced shock / boundary-layer box while the imposed oblique shock
    enters the domain and reflects off the boundary layer."""
    cfg, U = I.sbli(n=(96, 48, 8), L=(60.0, 20.0, 4.0), x_shock=10.0, scheme=I.TENO5)
    return collect(cfg, U, nsnap, steps_between)


def calibrate_threshold(w, feats, labels, recall=0.95):
    """Largest threshold whose recall of the positive labels on (feats, labels) is >= recall."""
    import torch
    n = int(labels.numel())
    probs = torch.empty(n, dtype=torch.float32, device="cuda")
    osbli.osbli_mlp_forward(feats, n, w, probs)
    pos = probs[labels.bool()]
    if pos.numel() == 0:
        return 0.5
    if pos.numel() > 1000000:   # an even sample over the whole set (torch.quantile's size limit)
        idx = torch.linspace(0, pos.numel() - 1, 1000000, device=pos.device).long()
        pos = pos[idx]
    q = torch.quantile(pos.float().cpu(), 1.0 - recall).item()
    return float(min(max(q, 1e-4), 0.9999))
