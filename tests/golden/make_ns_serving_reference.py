"""Writes ns_serving_reference.json: the log-evidence of the serving-size
nested-sampling run (tests/cases.py NS_SERVING) with every likelihood taken
from the FP64 oracle, for the GPU test that runs the same sampler fed by the
serving loop.  Calls only the oracle for likelihoods (about 12 million of
them; several minutes on a multi-core host).

    python tests/golden/make_ns_serving_reference.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import cases  # noqa: E402
import oracle as O  # noqa: E402
from paper_2603_13196_gb300 import ns  # noqa: E402

SEED = 1001


def main():
    sky, obs, m, data, truth, prior = cases.ns_serving_problem()
    c = cases.NS_SERVING
    t = time.time()
    r = ns.NestedSlice(prior, lambda th: O.loglike(m.A, m.B, data, obs, th), n_live=c["n_live"],
                       num_delete=c["num_delete"], num_inner_steps=5 * prior.dim, seed=SEED).run()
    out = {"what": "oracle-driven nested slice sampling of tests/cases.py NS_SERVING",
           "seed": SEED, "logZ": r.logZ, "logZ_err": r.logZ_err, "H": r.H, "n_like": r.n_like,
           "iterations": r.iterations, "logL_max": r.logL_max,
           "logL_truth": float(O.loglike(m.A, m.B, data, obs, truth[None])[0]),
           "seconds": round(time.time() - t, 1), "settings": {k: list(v) if isinstance(v, tuple) else v
                                                                for k, v in c.items()}}
    with open(os.path.join(HERE, "ns_serving_reference.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
