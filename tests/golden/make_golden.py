"""Write the oracle's optimum of the single-QP workloads to tests/golden/*.json.

Calls only ``oracle`` and ``qpgen``.  The GPU tests compare against these
files instead of re-running the slow CPU oracle on the large workloads.

    python tests/golden/make_golden.py 0 1 2
    python tests/golden/make_golden.py many      # batched and served QPs (oracle_batch_serving.json)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import qpgen                      # noqa: E402
from oracle import ipm            # noqa: E402


def main(configs):
    for k in configs:
        qp = qpgen.config_qp(k)
        variant = "kkt4" if qp.n + qp.m1 + 2 * qp.m2 <= 3000 else "kkt3"
        t0 = time.time()
        r = ipm.solve_qp(qp, variant=variant)
        dt = time.time() - t0
        rep = ipm.kkt_report(qp.H, qp.c, qp.A, qp.b, qp.C, qp.d, r.x, r.lam, r.nu, r.s)
        out = dict(
            workload=qp.name, n=qp.n, m1=qp.m1, m2=qp.m2, oracle_variant=variant,
            status=r.status, ipm_iters=r.iters, f=r.f,
            x_norm2=float(np.linalg.norm(r.x)), x_head=[float(v) for v in r.x[:16]],
            nu_norm2=float(np.linalg.norm(r.nu)), lam_norm2=float(np.linalg.norm(r.lam)),
            res_p=rep["res_p"], res_d=rep["res_d"], mu=rep["mu"],
            mu_history=[h["mu"] for h in r.history],
            oracle_seconds=dt,
            source="oracle.ipm.solve_qp on qpgen.config_qp(%d)" % k,
        )
        path = os.path.join(HERE, f"oracle_config{k}.json")
        with open(path, "w") as fh:
            json.dump(out, fh, indent=1)
        np.save(os.path.join(HERE, f"oracle_config{k}_x.npy"), r.x) if qp.n <= 200 else None
        print(k, r.status, r.iters, r.f, f"{dt:.1f}s", flush=True)


def many(batch_n=160, serve_n=256, serve_idx=400):
    """Oracle optima of the batched workload's QPs with n <= batch_n (all 512) and of
    the served stream's requests 0..serve_idx-1 with n <= serve_n, keyed by QP name:
    the batch and serving measurements check their results against these."""
    out = {"objective": {}, "ipm_iters": {}, "source": "oracle.ipm.solve_qp (kkt3) on qpgen.batch_qp(i), "
           f"i < 512 with n <= {batch_n}, and qpgen.serving_qp(i), i < {serve_idx} with n <= {serve_n}"}
    qps = [qpgen.batch_qp(i) for i in range(512) if qpgen.batch_dims(i)[0] <= batch_n]
    qps += [qpgen.serving_qp(i) for i in range(serve_idx) if qpgen.serving_dims(i)[0] <= serve_n]
    t0 = time.time()
    for q in qps:
        r = ipm.solve_qp(q, variant="kkt3")
        out["objective"][q.name] = r.f
        out["ipm_iters"][q.name] = r.iters
    with open(os.path.join(HERE, "oracle_batch_serving.json"), "w") as fh:
        json.dump(out, fh, indent=0)
    print(len(qps), "QPs", f"{time.time() - t0:.1f}s", flush=True)


if __name__ == "__main__":
    if sys.argv[1:] == ["many"]:
        many()
    else:
        main([int(a) for a in sys.argv[1:]] or [0])
