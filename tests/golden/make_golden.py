"""Writes the stored expected values under tests/golden/ by running the FP64 oracle only.

    python tests/golden/make_golden.py parity50          # 50 x 50 x 50, 100 steps (seconds)
    python tests/golden/make_golden.py plain2000x1000    # 2000 x 1000, K = 10, 500 steps (~25 min, 8 cores)

Each file records the workload, the hyper-parameters, F before the first step (F_0) and after
every step, the gradient norms, the final impacts and the certificate. Inputs come from
paper_2406_10262_gb300.synth (seed 0); nothing here touches the CUDA library.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2406_10262_gb300 import synth  # noqa: E402

HYPER = dict(epsilon=1.0, lr=0.1, beta1=0.9, beta2=0.999, adam_eps=1e-8, warm_start=True)


def run(name: str) -> dict:
    w = synth.WORKLOADS[name]
    U, I, K = w["n_users"], w["n_items"], w["n_slots"]
    r = synth.workload_relevance(name, seed=0)
    o = oracle.Oracle(U, I, K, iters=w["iters"], **HYPER)
    o.set_relevance(r)
    o.set_exposure(synth.dcg_exposure(K))
    t0 = time.time()
    _, _, F0 = o.impacts()
    F, gn = o.step(w["steps"])
    imp, util, Fl = o.impacts()
    gap, res = o.certificate()
    out = dict(workload=name, n_users=U, n_items=I, n_slots=K, iters=w["iters"], steps=w["steps"],
               seed=0, param="full_cost", grad_mode="implicit", optimizer="adam", **HYPER,
               F0=F0, F=list(map(float, F)), grad_norm=list(map(float, gn)),
               imp_final=list(map(float, imp)), utility_final=util, certificate_gap=gap,
               col_residual=res, oracle_seconds=time.time() - t0, oracle_threads=os.cpu_count())
    return out


if __name__ == "__main__":
    for name in sys.argv[1:]:
        res = run(name)
        path = os.path.join(HERE, f"{name}.json")
        with open(path + ".tmp", "w") as f:
            json.dump(res, f, indent=0)
        os.replace(path + ".tmp", path)
        print(name, "F0", res["F0"], "F_final", res["F"][-1], "s", round(res["oracle_seconds"], 1))
