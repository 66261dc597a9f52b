"""Checkpoint and resume of long scoring jobs (paper_2110_10156_gb300.resume),
driven on the CPU by a stand-in scorer: the interruption is made on the host
(the scorer raises part way), never on a GPU."""
import numpy as np
import pytest

from paper_2110_10156_gb300 import resume
from paper_2110_10156_gb300.synth import random_quaternions


class FakeScorer:
    """Deterministic per-rotation results from the quaternion alone; counts
    the rotations it scored and can fail on a given call."""

    def __init__(self, dims=(16, 16, 16), fail_on_call=None):
        self.dims = dims
        self.calls = 0
        self.scored = 0
        self.fail_on_call = fail_on_call

    def score_rotations(self, B, MB, q):
        self.calls += 1
        if self.fail_on_call is not None and self.calls == self.fail_on_call:
            raise RuntimeError("stopped part way")
        q = np.asarray(q)
        self.scored += len(q)
        s = (q[:, 0] * 0.5 + 0.25).astype(np.float32)
        c = np.stack([np.rint(q[:, k] * 10) for k in (1, 2, 3)], axis=1).astype(np.int32)
        return s, c


@pytest.fixture()
def quats():
    return random_quaternions(np.random.default_rng(11), 23)


def test_uninterrupted_job_matches_one_call(tmp_path, quats):
    f = FakeScorer()
    s, c = resume.score_rotations_resumable(f, None, None, quats, str(tmp_path / "ck.npz"), chunk=5)
    s1, c1 = FakeScorer().score_rotations(None, None, quats)
    np.testing.assert_array_equal(s, s1)
    np.testing.assert_array_equal(c, c1)
    assert f.calls == 5 and f.scored == 23            # 5 + 5 + 5 + 5 + 3


def test_resume_scores_only_the_rest(tmp_path, quats):
    path = str(tmp_path / "ck.npz")
    first = FakeScorer(fail_on_call=3)                # two chunks saved, the third fails
    with pytest.raises(RuntimeError):
        resume.score_rotations_resumable(first, None, None, quats, path, chunk=5)
    assert first.scored == 10
    second = FakeScorer()
    progress = []
    s, c = resume.score_rotations_resumable(second, None, None, quats, path, chunk=5,
                                            on_chunk=lambda d, R: progress.append(d))
    assert second.scored == 13 and progress == [15, 20, 23]
    ref_s, ref_c = resume.score_rotations_resumable(FakeScorer(), None, None, quats,
                                                    str(tmp_path / "ref.npz"), chunk=5)
    np.testing.assert_array_equal(s, ref_s)
    np.testing.assert_array_equal(c, ref_c)
    # a finished checkpoint is reused as it stands
    third = FakeScorer()
    s3, _ = resume.score_rotations_resumable(third, None, None, quats, path, chunk=5)
    assert third.scored == 0
    np.testing.assert_array_equal(s3, s)


@pytest.mark.parametrize("change", ["rotations", "chunk", "shape"])
def test_a_checkpoint_of_another_job_is_refused(tmp_path, quats, change):
    path = str(tmp_path / "ck.npz")
    resume.score_rotations_resumable(FakeScorer(fail_on_call=2), None, None, quats[:5], path,
                                     chunk=5)
    q, chunk, dims = quats[:5], 5, (16, 16, 16)
    if change == "rotations":
        q = quats[5:10]
    elif change == "chunk":
        chunk = 4
    else:
        dims = (16, 16, 15)
    with pytest.raises(ValueError, match="another job"):
        resume.score_rotations_resumable(FakeScorer(dims=dims), None, None, q, path, chunk=chunk)
    s, _ = resume.score_rotations_resumable(FakeScorer(dims=dims), None, None, q, path,
                                            chunk=chunk, overwrite=True)
    assert np.all(np.isfinite(s))


def test_bad_chunk(tmp_path, quats):
    with pytest.raises(ValueError):
        resume.score_rotations_resumable(FakeScorer(), None, None, quats, str(tmp_path / "c.npz"),
                                         chunk=0)


def test_a_checkpoint_for_other_volumes_or_settings_is_refused(tmp_path, quats):
    """Same rotations, chunk and shape, but a different B, mask, fixed volume
    or scoring setting: the saved chunks must not be merged in."""
    path = str(tmp_path / "ck.npz")
    rng = np.random.default_rng(3)
    B = rng.random((16, 16, 16)).astype(np.float32)
    MB = np.ones((16, 16, 16), np.uint8)
    f = FakeScorer()
    f._keep = (rng.random((16, 16, 16)).astype(np.float32), MB)
    f.settings = dict(eps=1e-5, gamma=0.5)
    resume.score_rotations_resumable(f, B, MB, quats[:5], path, chunk=5)
    B2 = B.copy()
    B2[3, 4, 5] += 1.0
    with pytest.raises(ValueError, match="another job"):
        resume.score_rotations_resumable(f, B2, MB, quats[:5], path, chunk=5)
    MB2 = MB.copy()
    MB2[0, 0, 0] = 0
    with pytest.raises(ValueError, match="another job"):
        resume.score_rotations_resumable(f, B, MB2, quats[:5], path, chunk=5)
    g = FakeScorer()
    g._keep = (f._keep[0] + 1.0, MB)
    g.settings = f.settings
    with pytest.raises(ValueError, match="another job"):
        resume.score_rotations_resumable(g, B, MB, quats[:5], path, chunk=5)
    h = FakeScorer()
    h._keep = f._keep
    h.settings = dict(eps=1e-5, gamma=0.6)
    with pytest.raises(ValueError, match="another job"):
        resume.score_rotations_resumable(h, B, MB, quats[:5], path, chunk=5)
    # the same job again reuses the finished checkpoint as it stands
    again = FakeScorer()
    again._keep, again.settings = f._keep, f.settings
    resume.score_rotations_resumable(again, B, MB, quats[:5], path, chunk=5)
    assert again.scored == 0


def test_a_truncated_checkpoint_is_refused_with_a_message(tmp_path, quats):
    path = tmp_path / "ck.npz"
    resume.score_rotations_resumable(FakeScorer(), None, None, quats, str(path), chunk=5)
    data = path.read_bytes()
    path.write_bytes(data[: len(data) // 2])
    with pytest.raises(ValueError, match="not a readable checkpoint"):
        resume.score_rotations_resumable(FakeScorer(), None, None, quats, str(path), chunk=5)
