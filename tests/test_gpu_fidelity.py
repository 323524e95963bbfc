"""GPU: simulation fidelity of drop scenes whose contacts come from the
detector (the |signed distance| statistic of Table 2).

512 environments of two objects from the 16-shape library fall onto a plane
for 480 steps at 240 Hz; the contact-resolution step (``locc_sim_step``)
takes its object-object contacts from the trained network (BF16 path), or,
as a proxy-geometry baseline, from bounding spheres.  Whenever a contact is
reported, the true signed distance of the two posed meshes is its
penetration depth or gap (oracle (a)); over 600 sampled contacts the test
reports the average, top-10 % average and maximum of |sd| and checks that the
network's contacts are tighter than the proxy's.
"""

import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_ENV, N_STEPS, N_SAMPLE = 512, 480, 600


def _abs_sd(lib, rec, rng):
    """|signed distance| of N_SAMPLE sampled reported contacts (oracle (a))."""
    ev = [(t, i) for t in range(len(rec["n_pairs"])) for i in range(int(rec["n_pairs"][t]))
          if rec["contacts"][t, i, 0] > 0]
    assert len(ev) >= N_SAMPLE, f"only {len(ev)} contacts reported"
    pick = rng.choice(len(ev), N_SAMPLE, replace=False)
    poses = np.zeros((2 * N_SAMPLE, 7), np.float32)
    osh = np.zeros(2 * N_SAMPLE, np.int32)
    for k, e in enumerate(pick):
        t, i = ev[e]
        a, b = rec["pairs"][t, i]
        poses[2 * k], poses[2 * k + 1] = rec["poses"][t, a], rec["poses"][t, b]
        osh[2 * k], osh[2 * k + 1] = rec["shape"][a], rec["shape"][b]
    pairs = np.stack([np.arange(0, 2 * N_SAMPLE, 2), np.arange(1, 2 * N_SAMPLE, 2)], 1)
    out = oracle.contact(lib.meshes, lib.points, poses, osh, pairs.astype(np.int32), culled=True,
                         n_threads=os.cpu_count() or 1)
    return np.abs(out[:, 7]), len(ev)


def _stats(v):
    top = np.sort(v)[-max(1, len(v) // 10):]
    return {"average": float(v.mean()), "top10_average": float(top.mean()),
            "maximum": float(v.max())}


def test_drop_scene_min_sd_network_vs_sphere_proxy():
    from paper_2304_09439_b300 import Detector, simulate
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    lib = synth.make_library(16, 3)
    with open(os.path.join(ROOT, "paper_2304_09439_b300", "weights", "locc_trained.bin"),
              "rb") as f:
        blob = f.read()
    poses0, vel0, osh, env = synth.drop_initial_state(lib, N_ENV, seed=21)
    radius = np.linalg.norm(lib.points, axis=2).max(axis=1).astype(np.float32)
    recs = {}
    with Detector(lib.points, lib.aabb, blob, 0.25, "bf16") as det:
        det.reserve(N_ENV, N_ENV)
        for source in ("locc", "sphere"):
            p, v, s, e = (torch.from_numpy(a.copy()).to(dev) for a in (poses0, vel0, osh, env))
            rec = simulate.run_drop(det, p, v, s, e, N_STEPS, source=source,
                                    radius=torch.from_numpy(radius).to(dev))
            fin = p.cpu().numpy()
            assert np.isfinite(fin).all()
            assert fin[:, 6].min() > -0.5, "an object fell through the plane"
            rec["shape"] = osh
            recs[source] = rec
    rng = np.random.default_rng(0)
    res = {}
    for source, rec in recs.items():
        v, n_ev = _abs_sd(lib, rec, rng)
        res[source] = dict(_stats(v), contacts_reported=n_ev)
    print("min-|sd| (m):", res)
    assert res["locc"]["average"] < res["sphere"]["average"]
    assert res["locc"]["top10_average"] < res["sphere"]["top10_average"]
    assert res["locc"]["average"] < 0.1
