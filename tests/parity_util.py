"""Shared helpers for GPU-vs-oracle parity checks (no method arithmetic here)."""
import numpy as np

TAU_FP32 = 1e-4   # score-map error bound relative to max |s| (FP32 path)


def neighbourhood_mask(shape, idx, radius=1):
    m = np.zeros(shape, dtype=bool)
    sl = tuple(slice(max(0, i - radius), i + radius + 1) for i in idx)
    m[sl] = True
    return m


def check_best_against_map(oracle_map, gpu_score, gpu_shift, tau=TAU_FP32):
    """Gap rule: if the oracle's best beats every shift outside its 3x3x3
    neighbourhood by more than 2 tau s1, the GPU must return that exact shift;
    otherwise the GPU's shift must score within tau s1 of the best in the
    oracle's map.  The GPU's score must match the oracle's value at the GPU's
    shift within tau * max|s|."""
    fin = np.isfinite(oracle_map)
    if not fin.any():
        assert not np.isfinite(gpu_score), "oracle has no valid shift but GPU returned one"
        return "none"
    dims = tuple((s + 1) // 2 for s in oracle_map.shape)
    flat = int(np.argmax(np.where(fin, oracle_map, -np.inf)))
    idx1 = np.unravel_index(flat, oracle_map.shape)
    s1 = float(oracle_map[idx1])
    chi1 = tuple(int(i) - (n - 1) for i, n in zip(idx1, dims))
    rest = np.where(neighbourhood_mask(oracle_map.shape, idx1) | ~fin, -np.inf, oracle_map)
    s2 = float(rest.max()) if np.isfinite(rest).any() else -np.inf
    gidx = tuple(int(c) + n - 1 for c, n in zip(gpu_shift, dims))
    assert all(0 <= i < s for i, s in zip(gidx, oracle_map.shape)), gpu_shift
    o_at_gpu = float(oracle_map[gidx])
    assert np.isfinite(o_at_gpu), f"GPU shift {gpu_shift} is not valid for the oracle"
    scale = float(np.max(np.abs(oracle_map[fin])))
    assert abs(float(gpu_score) - o_at_gpu) <= tau * scale, (gpu_score, o_at_gpu)
    if s1 - s2 > 2 * tau * s1:
        assert tuple(int(v) for v in gpu_shift) == chi1, (gpu_shift, chi1, s1, s2)
        return "exact"
    assert o_at_gpu >= s1 - tau * s1, (o_at_gpu, s1)
    return "near-tie"


def check_maps(oracle_map, gpu_map, tau=TAU_FP32):
    fo = np.isfinite(oracle_map)
    fg = np.isfinite(gpu_map)
    assert np.array_equal(fo, fg), f"valid sets differ at {np.argwhere(fo != fg)[:5]}"
    if fo.any():
        scale = float(np.max(np.abs(oracle_map[fo])))
        err = float(np.max(np.abs(gpu_map[fo].astype(np.float64) - oracle_map[fo])))
        assert err <= tau * scale, (err, scale)
        return err / scale
    return 0.0


def face_neighbours(chi):
    """chi and its six face neighbours (the shifts a sampled check evaluates)."""
    out = [tuple(int(c) for c in chi)]
    for a in range(3):
        for d in (-1, 1):
            c = list(out[0])
            c[a] += d
            out.append(tuple(c))
    return out


def check_best_at_sampled_shifts(oracle_map, gpu_score, gpu_shift, tau=TAU_FP32):
    """Sampled form of the gap rule for volumes whose full oracle map is too
    large: the oracle's direct sum at the GPU's shift must be valid and within
    tau of the GPU's score (scores lie in [0, 1]), and no valid face
    neighbour may beat it by more than tau (the GPU's shift is a local
    maximum of the oracle's map)."""
    dims = tuple((s + 1) // 2 for s in oracle_map.shape)
    at = lambda chi: float(oracle_map[tuple(int(c) + n - 1 for c, n in zip(chi, dims))])
    chis = face_neighbours(gpu_shift)
    o_at_gpu = at(chis[0])
    assert np.isfinite(o_at_gpu), f"GPU shift {gpu_shift} is not valid for the oracle"
    assert abs(float(gpu_score) - o_at_gpu) <= tau, (gpu_score, o_at_gpu)
    for chi in chis[1:]:
        if all(abs(c) <= n - 1 for c, n in zip(chi, dims)):
            v = at(chi)
            if np.isfinite(v):
                assert v <= o_at_gpu + tau, (chi, v, gpu_shift, o_at_gpu)
