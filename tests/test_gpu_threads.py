"""Launch attributes are kept per device and shared between host threads:
decodes issued from several host threads at once (each on its own stream,
the first launches of kernels that need more than 48 KB of shared memory
among them) give the results of the same decodes issued one by one."""
import threading

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_decodes_from_several_host_threads():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0605069_gb300 import gfbp, workload as W
    jobs = []
    for k, (name, N, frames, sched, layout) in enumerate([
            ("gf16_n1000_awgn", None, 40, "sus", "resident"), ("gf16_n1000_awgn", None, 40, "pus", "auto"),
            ("gf8_n2000_markov_bsc", 600, 16, "sus", "l2resident"), ("gf4_n96_bsc005", None, 200, "pus", "lanes"),
            ("gf16_n1000_awgn", 400, 60, "sus", "thread")]):
        b = W.make_batch(name, frames=frames, N=N)
        jobs.append(dict(b=b, cd=gfbp.Code.from_coo(b.code), sched=sched, layout=layout))

    def run(j, stream=None):
        b = j["b"]
        obs = torch.from_numpy(b.obs).cuda()
        fp = torch.from_numpy(b.param.astype(np.float32)).cuda()
        out = gfbp.decode(j["cd"], obs, b.channel, 0.0, schedule=j["sched"], max_iter=30, T=b.T, K=b.K,
                          frame_param=fp, layout=j["layout"], stream=stream)
        (stream or torch.cuda.current_stream()).synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}

    results = [None] * len(jobs)
    errors = []

    def worker(i):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                results[i] = run(jobs[i], s)
        except Exception as e:   # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(jobs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for j, r in zip(jobs, results):
        ref = run(j)
        for k in ref:
            np.testing.assert_array_equal(r[k], ref[k], err_msg=f"{j['layout']} {j['sched']} {k}")
