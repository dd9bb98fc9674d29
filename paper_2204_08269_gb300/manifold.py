"""Similarity study on the paper's synthetic AM/FM chirps (Sec. 3.2-3.4): JTFS features of the
16^3 = 4096 Eq. 5 signals, K-nearest-neighbour regression of the synthesizer parameters
(f_c, f_m, gamma) and an Isomap embedding, for the transform of this library only (the paper's
comparison representations are not built).

Features: the transform without frequential averaging (Eq. 4, as the study does) with J = 14,
Q = 8, J_fr = 4, Q_fr = 1 on N = 2^16 samples at 22050 Hz (2.97 s) and T = 2^14 (0.74 s, the
power of two nearest the study's 1000 ms); S1 and S2 averaged over the four frames (global
time invariance), then mu-log compressed path by path (Sec. 4.3, Eq. 6-7, eps = 0.1; S1
counts as one path).  The frequential filterbank (J_fr, Q_fr) and the signal length are not
given for the study; these are readings.  The transform, the averaging and the compression run on the GPU through the
library; the neighbour search and the embedding are PyTorch linear algebra on the device.

K-NN regression (Sec. 3.4): each example's estimate is the mean parameter of its K = 40
nearest neighbours in feature space (Euclidean, itself excluded); the error ratio is estimate /
truth.  Isomap (Sec. 3.3): the symmetric 40-nearest-neighbour graph with Euclidean edge
lengths, geodesic distances by Floyd-Warshall, classical scaling to three coordinates; each
parameter's alignment is the largest |Spearman rank correlation| of its logarithm with one
coordinate.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import jtfs

STUDY = dict(N=2 ** 16, J=14, Q=8, J_fr=4, Q_fr=1, T=2 ** 14, F=1, average_fr=False)


def features(x, plan, batch=64):
    """mu-log compressed, time-averaged [S1, S2] of every signal of x (host [M, N] float32):
    returns a device tensor [M, D] and the seconds spent in the transform."""
    M = x.shape[0]
    sh = plan.shapes
    feats, secs = [], 0.0
    for i in range(0, M, batch):
        xb = torch.from_numpy(np.ascontiguousarray(x[i:i + batch])).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s0, s1, s2, _ = plan.forward(xb, keep_checkpoint=False)
        torch.cuda.synchronize()
        secs += time.perf_counter() - t0
        B = xb.shape[0]
        a1 = s1.mean(dim=-1).reshape(B, 1, sh.n1)                       # one path of n1
        a2 = s2.mean(dim=-1).reshape(B, -1, sh.n_lam_out)               # (alpha, c) paths
        feats.append(torch.cat([a1, a2], dim=1))
    f = torch.cat(feats, dim=0).contiguous()
    mu = jtfs.mulog_mean(f)
    return jtfs.mulog(f, mu, eps=0.1).reshape(M, -1), secs


def knn(f, K=40):
    """Indices [M, K] of every example's K nearest neighbours (Euclidean, itself excluded) and
    the full distance matrix."""
    d = torch.cdist(f.double(), f.double())
    d.fill_diagonal_(float("inf"))
    idx = torch.topk(d, K, dim=1, largest=False).indices
    d.fill_diagonal_(0.0)
    return idx, d


def knn_regression(idx, theta):
    """Error ratios estimate / truth [M, 3] of the K-NN mean of each parameter."""
    th = torch.as_tensor(theta, dtype=torch.float64, device=idx.device)
    return th[idx].mean(dim=1) / th


def isomap(idx, d, dims=3):
    """Geodesic distances on the symmetric K-NN graph (Floyd-Warshall), then classical scaling
    to ``dims`` coordinates [M, dims]."""
    M = d.shape[0]
    g = torch.full_like(d, float("inf"))
    rows = torch.arange(M, device=d.device)[:, None].expand_as(idx)
    g[rows, idx] = d[rows, idx]
    g = torch.minimum(g, g.T)
    g.fill_diagonal_(0.0)
    for k in range(M):
        torch.minimum(g, g[:, k:k + 1] + g[k:k + 1, :], out=g)
    finite = torch.isfinite(g)
    if not bool(finite.all()):
        g = torch.where(finite, g, g[finite].max())
    d2 = g * g
    J = torch.eye(M, dtype=d2.dtype, device=d2.device) - 1.0 / M
    Bm = -0.5 * J @ d2 @ J
    w, v = torch.linalg.eigh(Bm)
    top = torch.argsort(w, descending=True)[:dims]
    return v[:, top] * torch.sqrt(torch.clamp(w[top], min=0.0))


def _spearman(a, b):
    ra = torch.argsort(torch.argsort(a)).double()
    rb = torch.argsort(torch.argsort(b)).double()
    ra = ra - ra.mean()
    rb = rb - rb.mean()
    return float((ra * rb).sum() / torch.sqrt((ra * ra).sum() * (rb * rb).sum()))


def alignment(emb, theta):
    """For each parameter, the largest |Spearman rho| between its logarithm and one embedding
    coordinate, and that coordinate."""
    out = {}
    th = torch.as_tensor(np.log(theta), dtype=torch.float64, device=emb.device)
    for j, name in enumerate(("f_c", "f_m", "gamma")):
        rho = [abs(_spearman(emb[:, c], th[:, j])) for c in range(emb.shape[1])]
        out[name] = {"rho": max(rho), "coordinate": int(np.argmax(rho))}
    return out


def run(count=16, K=40, precision="fp32", seed_batch=64):
    """The study on the count^3 grid; returns a dict of the results."""
    import synth_signals as SS
    theta = SS.eq5_grid(count)
    cfg = dict(STUDY)
    N = cfg.pop("N")
    t0 = time.perf_counter()
    x = SS.chirp_eq5_batch(N, theta)
    gen_s = time.perf_counter() - t0
    plan = jtfs.JTFSPlan(N, precision=precision, **cfg)
    f, tf = features(x, plan, batch=seed_batch)
    idx, d = knn(f, K)
    ratios = knn_regression(idx, theta).cpu().numpy()
    emb = isomap(idx, d)
    res = {"signals": len(theta), "N": N, "feature_dim": int(f.shape[1]),
           "transform_s": tf, "signals_per_s": len(theta) / tf, "generate_s": gen_s,
           "knn_error_ratio": {}, "isomap_alignment": alignment(emb, theta)}
    for j, name in enumerate(("f_c", "f_m", "gamma")):
        r = ratios[:, j]
        res["knn_error_ratio"][name] = {
            "median": float(np.median(r)), "p10": float(np.percentile(r, 10)),
            "p90": float(np.percentile(r, 90)),
            "within_0.75_1.5": float(np.mean((r >= 0.75) & (r <= 1.5)))}
    return res


if __name__ == "__main__":
    import json
    torch.cuda.set_device(0)
    print(json.dumps(run()))
