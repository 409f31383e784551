"""Connectivity estimation on the GPU, end to end: simulate networks with a
known topology (batched form), export their observed traces, compute the lagged
correlation features of every candidate pair, train or apply the learned
estimator, and score both estimators against the ground truth.

Orchestration only: every step is one call of libgeonet.so; torch provides the
device buffers.
"""
from __future__ import annotations

import numpy as np

from . import geonet, netgen


def candidate_table(specs, cands=None):
    """Candidate pairs of several networks with global node ids (networks
    concatenated in order), their labels, the candidate radius of each pair, the
    network index of each pair and the concatenated positions.  `cands`: the
    networks' netgen.candidates results if already computed."""
    src, dst, lab, rad, net = [], [], [], [], []
    off = 0
    for i, sp in enumerate(specs):
        s, d, lb = netgen.candidates(sp) if cands is None else cands[i]
        src.append(s.astype(np.int64) + off)
        dst.append(d.astype(np.int64) + off)
        lab.append(lb)
        rad.append(np.full(s.shape[0], sp.radius))
        net.append(np.full(s.shape[0], i, np.int32))
        off += sp.n_nodes
    return dict(src=np.concatenate(src).astype(np.int32), dst=np.concatenate(dst).astype(np.int32),
                label=np.concatenate(lab), radius=np.concatenate(rad), net=np.concatenate(net),
                pos=np.ascontiguousarray(np.concatenate([sp.pos for sp in specs]), np.float64), n_nodes=off)


def simulate_features(specs, n_samples: int = 500, device: int = 0, stream=None, cands=None):
    """Simulate `specs` for n_samples observation intervals from rest (one batched
    run) and return the features [P, 33] and plain scores [P] of their candidate
    pairs (CUDA tensors) with the labels and network index of each pair (numpy).
    `cands`: the networks' netgen.candidates results if already computed."""
    import torch
    dev = torch.device("cuda", device)
    every = specs[0].obs["sample_every"]
    batch = geonet.Batch(specs, device=device, stream=stream, obs_capacity=n_samples)
    batch.gn_batch_step(n_samples * every)
    tab = candidate_table(specs, cands)
    traces = torch.empty((tab["n_nodes"], n_samples), dtype=torch.float32, device=dev)
    geonet.gn_batch_export_traces(batch, 0, n_samples, traces)
    batch.gn_batch_destroy()
    P = tab["src"].shape[0]
    feats = torch.empty((P, 33), dtype=torch.float32, device=dev)
    score = torch.empty(P, dtype=torch.float32, device=dev)
    geonet.gn_xcorr_features(traces, torch.from_numpy(tab["pos"]).to(dev), torch.from_numpy(tab["src"]).to(dev),
                             torch.from_numpy(tab["dst"]).to(dev), torch.from_numpy(tab["radius"]).to(dev),
                             feats, score, stream=stream)
    return dict(features=feats, score=score, label=tab["label"], net=tab["net"], traces=traces)


def train(mlp: geonet.Mlp, feats, labels, epochs: int, batch: int, seed: int, lr: float = 1e-3,
          weight_decay: float = 0.0, orders=None):
    """Minibatch AdamW over resident features: each epoch visits the samples in the
    order netgen.shuffles(seed, ...) draws (full batches only), as one
    gn_mlp_train_epoch call (`orders`: the same orders already on the device, to
    keep drawing them out of a timed region).  Returns the mean loss of each epoch."""
    import torch
    P = feats.shape[0]
    y = labels if hasattr(labels, "data_ptr") else torch.from_numpy(np.asarray(labels, np.float32)).to(feats.device)
    losses = []
    n_batches = P // batch
    if orders is None:
        orders = (torch.from_numpy(o).to(feats.device) for o in netgen.shuffles(seed, P, epochs))
    for idx in orders:
        if n_batches == 0:
            losses.append(0.0)
            continue
        step_losses = mlp.gn_mlp_train_epoch(feats, y, idx, n_batches, batch, lr=lr, weight_decay=weight_decay)
        losses.append(float(np.mean(step_losses.astype(np.float64))))
    return losses


def scores(pred, labels, threshold=None):
    """AUROC, and F1 at `threshold` (or at the best threshold if None)."""
    p = pred.detach().cpu().numpy() if hasattr(pred, "detach") else np.asarray(pred)
    auc = geonet.gn_score_auroc(p, labels)
    if threshold is None:
        threshold, f1 = geonet.gn_score_best_f1(p, labels)
    else:
        f1 = geonet.gn_score_f1(p, labels, threshold)
    return dict(auroc=auc, f1=f1, threshold=threshold)
