"""Checkpoint and resume for long scoring jobs.

A job of many rotations (the 256^3 workload scores 5000) is scored in chunks
of a fixed number of rotations through ``Fixed.score_rotations``.  After each
chunk the per-rotation results so far are written to a checkpoint file
(replaced atomically), so a job that stops part way resumes after its last
saved chunk instead of starting over.  Rotations are independent (each
rotation's map and maximum, Section 3.2), so chunking changes nothing but the
grouping of launches; chunk boundaries are fixed by the chunk size, so a
resumed job returns exactly what the same job run without interruption with
the same chunk size returns.

Host orchestration only: the scoring itself runs in the CUDA library.  The
checkpoint records a fingerprint of the rotation set, the chunk size and the
volume shape, and a checkpoint that does not match the job is refused rather
than mixed in.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np


def job_fingerprint(quats: np.ndarray, chunk: int, dims) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(quats, dtype=np.float64).tobytes())
    h.update(np.asarray([chunk, *dims], dtype=np.int64).tobytes())
    return h.hexdigest()


def _load(path: str, fingerprint: str, R: int):
    with np.load(path) as d:
        if str(d["fingerprint"]) != fingerprint:
            raise ValueError(f"{path} belongs to another job (rotations, chunk size or shape "
                             "differ); remove it or pass overwrite=True")
        done = int(d["done"])
        scores, shifts = d["scores"].copy(), d["shifts"].copy()
    if not (0 <= done <= R) or scores.shape != (R,) or shifts.shape != (R, 3):
        raise ValueError(f"{path} is not a checkpoint of this job")
    return done, scores, shifts


def _save(path: str, fingerprint: str, done: int, scores: np.ndarray, shifts: np.ndarray):
    tmp = path + ".tmp.npz"               # np.savez keeps a name that ends in .npz
    np.savez(tmp, fingerprint=np.array(fingerprint), done=np.array(done), scores=scores,
             shifts=shifts)
    os.replace(tmp, path)


def score_rotations_resumable(f, B, MB, quats, path: str, chunk: int = 1000,
                              overwrite: bool = False, on_chunk=None):
    """Per-rotation best score [R] (float32) and shift [R, 3] (int32, z y x)
    as numpy arrays, scoring ``chunk`` rotations per call of
    ``f.score_rotations`` and saving progress to ``path`` after each chunk.

    If ``path`` holds a checkpoint of the same job (same rotations, chunk
    size and volume shape), the saved chunks are not scored again.
    ``on_chunk(done, R)`` is called after each saved chunk.  The checkpoint is
    left in place when the job completes (``done == R``)."""
    q = np.ascontiguousarray(np.asarray(quats, dtype=np.float64).reshape(-1, 4))
    R = q.shape[0]
    if chunk <= 0:
        raise ValueError("chunk must be positive")
    fp = job_fingerprint(q, chunk, f.dims)
    if os.path.exists(path) and not overwrite:
        done, scores, shifts = _load(path, fp, R)
    else:
        done = 0
        scores = np.full(R, -np.inf, dtype=np.float32)
        shifts = np.zeros((R, 3), dtype=np.int32)
    while done < R:
        end = min(R, done + chunk)
        s, c = f.score_rotations(B, MB, q[done:end])
        scores[done:end] = _to_numpy(s)
        shifts[done:end] = _to_numpy(c)
        done = end
        _save(path, fp, done, scores, shifts)
        if on_chunk is not None:
            on_chunk(done, R)
    return scores, shifts


def _to_numpy(t) -> np.ndarray:
    if isinstance(t, np.ndarray):
        return t
    return t.detach().cpu().numpy()
