"""Serving loop on the GPU: requests of mixed sizes, channel counts and N (4
and 6) that arrive while others run are admitted as slots and memory free up,
overlap on the device, and each result equals the same request filtered alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1003_2022_gb300 import api, synth  # noqa: E402
from paper_1003_2022_gb300.serve import Request, Server  # noqa: E402

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(5)
    reqs = []
    t = 0.0
    for i in range(24):
        side = int(np.exp(rng.uniform(np.log(48), np.log(320))))
        C = 1 if rng.random() < 0.5 else 3
        dtype = "u8" if i % 3 == 0 else "f32"
        img = np.stack([synth.image(side, side, seed=100 + i, dtype=dtype, sub=c) for c in range(C)])
        prm = synth.srt_field(side, side, seed=100 + i, sigma=(1.0, 12.0), rho=(1.0, 8.0))
        N = 6 if i % 4 == 1 else (5 if i == 7 else 4)
        reqs.append(Request(i, img, prm, N=N, arrival=t, max_scale=12.0))
        # a burst of six at t = 0 fills the slots together; the rest arrive over time
        if i >= 5:
            t += float(rng.exponential(0.002))
    srv = Server(slots=3, budget_bytes=1 << 30, device=0)
    try:
        results, stats = srv.run(reqs)
    finally:
        srv.close()
    assert stats["completed"] == 23 and stats["rejected"] == 1
    assert results[7].status.startswith("unsupported N")
    assert stats["peak_bytes"] <= 1 << 30
    overlapped = sum(1 for a in results for b in results
                     if a.rid < b.rid and a.status == b.status == "ok"
                     and a.t_admit < b.t_done and b.t_admit < a.t_done)
    assert overlapped > 0
    for r, q in zip(results, reqs):
        if r.status != "ok":
            continue
        alone = api.filter(torch.from_numpy(q.image).to(dev), torch.from_numpy(q.params).to(dev), kind="srt",
                           N=q.N, max_scale=12.0).cpu().numpy()
        err = np.abs(r.out - alone).max() / np.abs(alone).max()
        assert err <= 1e-5, (r.rid, err)
    assert stats["p50_ms"] is not None and stats["p99_ms"] >= stats["p50_ms"]


def test_malformed_and_cancelled_requests():
    """A request whose field holds NaN is served with its pixels flagged (the
    device status names the condition), a request withdrawn before admission
    never runs, and the others are unaffected."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(8)
    reqs = []
    for i in range(6):
        img = synth.image(64, 72, seed=200 + i, dtype="f32")[None]
        prm = synth.srt_field(64, 72, seed=200 + i, sigma=(1.0, 4.0), rho=(1.0, 3.0))
        if i == 2:
            prm[0, 10:20, 10:20] = np.nan
        reqs.append(Request(i, img, prm, N=4, arrival=0.0, max_scale=4.0))
    reqs[5].cancel_at = 0.0   # withdrawn at once: one slot, so it cannot have been admitted
    srv = Server(slots=1, budget_bytes=64 << 20, device=0)
    try:
        results, stats = srv.run(reqs)
    finally:
        srv.close()
    assert results[2].status.startswith("invalid pixels"), results[2].status
    out = results[2].out
    nan = np.isnan(out)
    assert nan[0, 10:20, 10:20].all() and nan.sum() == 100
    assert np.isfinite(out[~nan]).all()
    assert results[5].status == "cancelled" and results[5].out is None
    assert all(results[i].status == "ok" for i in (0, 1, 3, 4))
    assert stats["cancelled"] == 1 and stats["invalid"] == 1 and stats["completed"] == 4
