"""The serving loop on the GPU: every sensor's frames, coded in the mix of
continuous batches, are the bytes the oracle writes for that sensor alone,
and every decode request returns the oracle's decoded scan."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2209_08196_gb300 import build as jbuild  # noqa: E402
from paper_2209_08196_gb300.serve import GpuBackend, Sensor, Server, poisson_arrivals  # noqa: E402
from tests.gpu_util import NP_DT, to_dev  # noqa: E402
from tests.test_gpu_batch import make_scans  # noqa: E402

jbuild.build()

CLASSES = [(16, 1024, [(4, 10)]), (32, 512, [(4, 10), (2, 1)]), (8, 2048, [(4, 10), (4, 10), (2, 1), (1, 1), (2, 1)])]


@pytest.mark.parametrize("realtime,graphs", [(False, False), (True, True)])
def test_each_result_is_the_same_alone_and_in_the_mix(realtime, graphs):
    rng = np.random.default_rng(21)
    pools_np = [make_scans(rng, H, W, a, 6) for H, W, a in CLASSES]
    pools = [[[to_dev(p) for p in sc] for sc in pool] for pool in pools_np]
    sensors = []
    for i in range(9):
        c = i % len(CLASSES)
        H, W, a = CLASSES[c]
        sensors.append(Sensor(i, H, W, a, float(rng.uniform(10, 20)) * (20 if realtime else 1), pool=c,
                              pool_offset=int(rng.integers(6))))
    reqs = poisson_arrivals(sensors, 0.6 if realtime else 1.0, 0.3, seed=22)
    be = GpuBackend(pools, graphs=graphs, keep=True)
    st = Server(be, sensors, budget_bytes=8 << 30).run(reqs, realtime=realtime)
    assert st.failed == 0 and st.encoded == len(reqs)
    assert st.decoded == sum(r.decode for r in reqs) > 0
    assert max(st.batch_sizes) > 1  # the scans really were batched
    for s in sensors:
        ref = oracle.Codec(s.H, s.W, s.attrs)
        refd = oracle.Codec(s.H, s.W, s.attrs)
        mine = sorted(r.seq for r in reqs if r.sensor == s.sid)
        assert mine == list(range(len(mine)))
        for seq in mine:
            scan = pools_np[s.pool][(s.pool_offset + seq) % 6]
            want = ref.encode(scan)
            assert be.frames[(s.sid, seq)] == want, (s.sid, seq)
            planes, _ = refd.decode(want)
            if (s.sid, seq) in be.decoded:
                for k, (b, _) in enumerate(s.attrs):
                    got = be.decoded[(s.sid, seq)][k].numpy().view(NP_DT[b])
                    assert np.array_equal(got, planes[k]), (s.sid, seq, k)


def test_results_hold_when_sensors_wait_for_budget_and_reuse_handles():
    # a budget of about three sensors: sensors wait to be admitted, released
    # sensors' handles are kept, reused by sensors of the same shape (reset
    # first) and freed when the budget needs the memory; every frame and
    # decode must still be the oracle's for that sensor alone
    rng = np.random.default_rng(23)
    pools_np = [make_scans(rng, H, W, a, 6) for H, W, a in CLASSES]
    pools = [[[to_dev(p) for p in sc] for sc in pool] for pool in pools_np]
    sensors = []
    for i in range(9):
        c = i % len(CLASSES)
        H, W, a = CLASSES[c]
        sensors.append(Sensor(i, H, W, a, float(rng.uniform(10, 20)), pool=c, pool_offset=int(rng.integers(6))))
    reqs = poisson_arrivals(sensors, 0.5, 0.3, seed=24)
    be = GpuBackend(pools, keep=True)
    budget = 3 * max(be.footprint(s) for s in sensors)
    st = Server(be, sensors, budget_bytes=budget).run(reqs, realtime=False)
    assert st.failed == 0 and st.encoded == len(reqs)
    assert st.deferred > 0 and st.admitted == len(sensors)
    assert be.cached_bytes + sum(be.footprint(be.s[sid]["sensor"]) for sid in be.s) <= budget
    for s in sensors:
        ref = oracle.Codec(s.H, s.W, s.attrs)
        refd = oracle.Codec(s.H, s.W, s.attrs)
        mine = sorted(r.seq for r in reqs if r.sensor == s.sid)
        for seq in mine:
            want = ref.encode(pools_np[s.pool][(s.pool_offset + seq) % 6])
            assert be.frames[(s.sid, seq)] == want, (s.sid, seq)
            planes, _ = refd.decode(want)
            if (s.sid, seq) in be.decoded:
                for k, (b, _) in enumerate(s.attrs):
                    got = be.decoded[(s.sid, seq)][k].numpy().view(NP_DT[b])
                    assert np.array_equal(got, planes[k]), (s.sid, seq, k)
