"""GPU tests of the output stage: statistics, slices, snapshots, checkpoints.

Snapshots must hold exactly the state gs_read returns at their step, and
writing them while stepping must not change the run; a checkpoint resumes
the run bit for bit (the step counter selects the noise draws).
"""
import numpy as np
import pytest

from paper_2309_10292_gb300 import gs, snapshot
from tests.gpu_util import PAPER, need_cuda

pytestmark = pytest.mark.gpu


def make(L, dtype="f32", **kw):
    need_cuda()
    prm = dict(PAPER, noise=0.1, seed=11)
    prm.update(kw)
    return gs.GrayScott(L, dtype=dtype, **prm)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_stats_match_numpy(dtype):
    sim = make(48, dtype)
    sim.step(30)
    u, v = sim.read()
    for field, a in ((gs.GS_U, u), (gs.GS_V, v)):
        st = sim.stats(field)
        a64 = a.astype(np.float64)
        assert st["min"] == a64.min() and st["max"] == a64.max() and st["nan"] == 0
        assert abs(st["mean"] - a64.mean()) <= 1e-12 * max(1.0, abs(a64.mean()))
        assert abs(st["rms"] - np.sqrt((a64 ** 2).mean())) <= 1e-12
    sim.close()


def test_stats_count_nans():
    sim = make(16)
    u, v = sim.read()
    u[3, 4, 5] = np.nan
    u[0, 0, 0] = np.nan
    sim.write(u, v)
    st = sim.stats(gs.GS_U)
    assert st["nan"] == 2
    good = u[~np.isnan(u)].astype(np.float64)
    assert st["min"] == good.min() and st["max"] == good.max()
    sim.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_slices_match_numpy(dtype):
    L = 40
    sim = make(L, dtype)
    sim.step(12)
    u, v = sim.read()
    for field, a in ((gs.GS_U, u), (gs.GS_V, v)):
        for idx in (0, 17, L - 1):
            np.testing.assert_array_equal(sim.slice(field, 2, idx), a[idx, :, :])
            np.testing.assert_array_equal(sim.slice(field, 1, idx), a[:, idx, :])
            np.testing.assert_array_equal(sim.slice(field, 0, idx), a[:, :, idx])
    with pytest.raises(gs.GsError):
        sim.slice(gs.GS_U, 3, 0)
    with pytest.raises(gs.GsError):
        sim.slice(gs.GS_U, 2, L)
    sim.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_snapshots_hold_the_state_and_leave_the_run_unchanged(tmp_path, dtype):
    L, every, n = 64, 5, 25
    path = str(tmp_path / "run.gs")
    sim = make(L, dtype)
    with sim.snapshots(path) as w:
        w.write()  # step 0
        for _ in range(n // every):
            sim.step(every)
            w.write()
        info_before = w.info()
    assert info_before["records"] <= n // every + 1
    ref = make(L, dtype)
    hdr, recs = snapshot.read(path)
    assert hdr["kind"] == "snapshot" and hdr["L"] == L and hdr["dtype"] == dtype
    assert (hdr["Du"], hdr["Dv"], hdr["F"], hdr["k"], hdr["dt"], hdr["noise"], hdr["seed"]) == (
        PAPER["Du"], PAPER["Dv"], PAPER["F"], PAPER["k"], PAPER["dt"], 0.1, 11)
    assert [r["step"] for r in recs] == list(range(0, n + 1, every))
    for r in recs:
        if r["step"]:
            ref.step(every)
        ur, vr = ref.read()
        np.testing.assert_array_equal(r["u"], ur)
        np.testing.assert_array_equal(r["v"], vr)
        assert r["u_min"] == ur.astype(np.float64).min() and r["v_max"] == vr.astype(np.float64).max()
    # the snapshotted run ends in the same state as the plain one
    us, vs = sim.read()
    np.testing.assert_array_equal(us, ref.read()[0])
    np.testing.assert_array_equal(vs, ref.read()[1])
    sim.close()
    ref.close()


def test_snapshot_back_to_back_writes(tmp_path):
    # more writes than host slots without stepping in between: all land, in order
    path = str(tmp_path / "b.gs")
    sim = make(32)
    w = sim.snapshots(path)
    for i in range(5):
        w.write()
        sim.step(1)
    w.close()
    _, recs = snapshot.read(path)
    assert [r["step"] for r in recs] == [0, 1, 2, 3, 4]
    sim.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_checkpoint_resume_is_bitwise(tmp_path, dtype):
    path = str(tmp_path / "c.ckpt")
    a = make(48, dtype)
    a.step(7)
    a.checkpoint(path)
    a.step(13)
    ua, va = a.read()
    b = make(48, dtype)
    b.restore(path)
    assert b.t == 7
    b.step(13)
    ub, vb = b.read()
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(va, vb)
    hdr, recs = snapshot.read(path)
    assert hdr["kind"] == "checkpoint" and recs[0]["step"] == 7
    a.close()
    b.close()


def test_checkpoint_rejects_other_runs_and_bad_files(tmp_path):
    path = str(tmp_path / "c.ckpt")
    a = make(32)
    a.step(3)
    a.checkpoint(path)
    for other in (make(32, F=0.03), make(32, seed=12), make(40), make(32, "f64")):
        with pytest.raises(gs.GsError) as e:
            other.restore(path)
        assert e.value.status == gs.GS_EINVAL
        assert other.t == 0  # untouched
        other.close()
    with pytest.raises(gs.GsError) as e:
        a.restore(str(tmp_path / "missing.ckpt"))
    assert e.value.status == gs.GS_EIO
    with open(path, "rb") as f:
        data = f.read()
    with open(path, "wb") as f:
        f.write(data[:-100])
    with pytest.raises(gs.GsError) as e:
        a.restore(path)
    assert e.value.status == gs.GS_EIO
    with pytest.raises(gs.GsError) as e:
        a.snapshots(str(tmp_path / "no" / "such" / "dir" / "x.gs"))
    assert e.value.status == gs.GS_EIO
    a.close()
