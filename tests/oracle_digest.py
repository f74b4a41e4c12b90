"""Compact per-frame oracle results for parity runs too large to keep whole
(test helper; imports no GPU code, so it can run in spawned worker processes).

The per-site arrays (labels, owners) are reduced to SHA-256 digests of their
int32 bytes; everything per bubble or per link is kept as is."""
from __future__ import annotations

import hashlib

import numpy as np

import oracle as O
from paper_1607_00908_gb300 import inputs as I


def array_digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.int32).tobytes()).hexdigest()


def site_digests(labels, owners):
    return array_digest(labels), array_digest(owners)


def batched_frames(spec, n_frames: int = 8):
    """Frames of one instance of the batched workload (smoothed noise, shear 0.02)."""
    L, sigma, seed = spec
    return I.noise_frames(L, sigma, n_frames, 0.02, seed)


def oracle_digests(spec, n_frames: int = 8):
    L = spec[0]
    det = O.Detector(L, L)
    out = []
    for F in batched_frames(spec, n_frames):
        r = det.push(F)
        lab, own = site_digests(r["labels"], r["owners"])
        out.append(dict(K=r["K"], labels=lab, owners=own, centroids=r["centroids"], edges=r["edges"],
                        K_prev=r["K_prev"], n_matched=r["n_matched"], breaking=r["breaking"],
                        breaking_prev=r["breaking_prev"], arising=r["arising"], active=r["active"]))
    return out


def oracle_sequence(task):
    """Oracle over one simulation's frame sequence: `task` = (L, pool frames,
    indices into the pool). Returns per frame its bubble and link counts,
    breaking (and their past keys), arising and active flags, and the final
    frame's label digest."""
    L, pool, seq = task
    det = O.Detector(L, L)
    frames = []
    r = None
    for j in seq:
        r = det.push(pool[j])
        frames.append(dict(K=r["K"], E=len(r["edges"]), breaking=r["breaking"], breaking_prev=r["breaking_prev"],
                           arising=r["arising"], active=r["active"]))
    lab = array_digest(r["labels"]) if r is not None else None
    return frames, lab
