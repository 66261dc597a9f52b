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
checkpoint records a fingerprint of the job: the rotation set, the chunk
size, the volume shape, the contents of B and its mask, the fixed handle's
A and mask and its scoring settings (eps, gamma, lengths, measure, precision,
padding mode).  A checkpoint that does not match the job is refused rather
than mixed in.  Each checkpoint is flushed to disk before it replaces the
previous one, so a crash leaves the old or the new checkpoint, not a torn one.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np


def _update_with(h, x):
    """Hash the contents of a host or device array (None hashes as a marker)."""
    if x is None:
        h.update(b"none")
        return
    a = _to_numpy(x)
    h.update(str(a.dtype).encode() + str(a.shape).encode())
    h.update(np.ascontiguousarray(a).tobytes())


def job_fingerprint(quats: np.ndarray, chunk: int, dims, B=None, MB=None, fixed=None) -> str:
    """SHA-256 over everything that decides the job's results: rotations,
    chunk size, shape, B and its mask, and (when ``fixed`` is a handle) the
    fixed volume, its mask and the handle's scoring settings."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(quats, dtype=np.float64).tobytes())
    h.update(np.asarray([chunk, *dims], dtype=np.int64).tobytes())
    _update_with(h, B)
    _update_with(h, MB)
    keep = getattr(fixed, "_keep", None) if fixed is not None else None
    _update_with(h, keep[0] if keep else None)
    _update_with(h, keep[1] if keep else None)
    settings = getattr(fixed, "settings", None) if fixed is not None else None
    h.update(repr(sorted(settings.items()) if settings else None).encode())
    return h.hexdigest()


def _load(path: str, fingerprint: str, R: int):
    try:
        d = np.load(path)
        fp, done = str(d["fingerprint"]), int(d["done"])
        scores, shifts = d["scores"].copy(), d["shifts"].copy()
        d.close()
    except Exception as e:          # truncated or foreign file
        raise ValueError(f"{path} is not a readable checkpoint ({e}); remove it or pass "
                         "overwrite=True") from e
    if fp != fingerprint:
        raise ValueError(f"{path} belongs to another job (rotations, chunk size, shape, "
                         "volumes or settings differ); remove it or pass overwrite=True")
    if not (0 <= done <= R) or scores.shape != (R,) or shifts.shape != (R, 3):
        raise ValueError(f"{path} is not a checkpoint of this job")
    return done, scores, shifts


def _save(path: str, fingerprint: str, done: int, scores: np.ndarray, shifts: np.ndarray):
    tmp = path + ".tmp"
    with open(tmp, "wb") as fh:
        np.savez(fh, fingerprint=np.array(fingerprint), done=np.array(done), scores=scores,
                 shifts=shifts)
        fh.flush()
        os.fsync(fh.fileno())
    os.replace(tmp, path)
    dirfd = os.open(os.path.dirname(os.path.abspath(path)), os.O_RDONLY)
    try:
        os.fsync(dirfd)
    finally:
        os.close(dirfd)


def score_rotations_resumable(f, B, MB, quats, path: str, chunk: int = 1000,
                              overwrite: bool = False, on_chunk=None):
    """Per-rotation best score [R] (float32) and shift [R, 3] (int32, z y x)
    as numpy arrays, scoring ``chunk`` rotations per call of
    ``f.score_rotations`` and saving progress to ``path`` after each chunk.

    If ``path`` holds a checkpoint of the same job (same rotations, chunk
    size, volumes, masks and handle settings), the saved chunks are not
    scored again.
    ``on_chunk(done, R)`` is called after each saved chunk.  The checkpoint is
    left in place when the job completes (``done == R``)."""
    q = np.ascontiguousarray(np.asarray(quats, dtype=np.float64).reshape(-1, 4))
    R = q.shape[0]
    if chunk <= 0:
        raise ValueError("chunk must be positive")
    fp = job_fingerprint(q, chunk, f.dims, B, MB, f)
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
