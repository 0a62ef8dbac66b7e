"""Short runs of the library's kernels for a profiler (ncu) to capture.

    python -m paper_2211_06142_gb300.profile_run step [mixed|fp64] [steps] [eager]
        the fused step on the 200,000-sphere sand-production cylinder (or
        the --workload one); "eager": the same kernels launched from the
        host (the library's profiling entry point), since a profiler does
        not see the kernel nodes of graphs that hold conditional nodes
    python -m paper_2211_06142_gb300.profile_run rebuild [mixed|fp64] [count]
        the candidate-list rebuild sequence, forced before each of `count`
        steps on the same cylinder (kernels launched from the host)
    python -m paper_2211_06142_gb300.profile_run closure [steps]
        the step with the learned closure on the same cylinder at SSW k = 2
        (kernels launched from the host)
    python -m paper_2211_06142_gb300.profile_run mlp [n] [iters]
        full-batch training steps of the closure network on n samples

Options (before or after the mode's arguments): --cell S (search-cell
scale), --skin F (skin / largest grain diameter), --block B (threads per
block of the force kernel), --ppw P (spheres per warp of that kernel), for
capturing the launch configuration the autotuner chose; --workload
cylinder200k | tiled500k | tiled2m (the benchmark's 2.0M-sphere cylinder).

Each prints its counters and "ok" when it ends without an error.
"""
from __future__ import annotations

import sys

import numpy as np


KNOBS = {"cell": 0.0, "skin": None, "block": 128, "ppw": 32, "workload": "cylinder200k"}

# --workload: the 200k-sphere cylinder, or the tiled cylinders of about
# 500k spheres (radius and height x1.357) and 2.0M spheres (x2.15, the
# benchmark's headline sample)
WORKLOADS = {
    "cylinder200k": lambda I: I.cached(I.fine_cylinder),
    "tiled500k": lambda I: I.cached(I.tiled_cylinder, 500_000, 1.357, 5, nf=(54, 54, 27)),
    "tiled2m": lambda I: I.cached(I.tiled_cylinder, 2_000_000, 2.15, 4),
}


def _cylinder_ctx(precision, closure=False, k=1, steps_per_graph=32):
    from . import cgdem
    from . import inputs as I
    from . import workloads as W
    s = WORKLOADS[KNOBS["workload"]](I) if k == 1 else W.coarse_cylinder(k=k)
    m = s.material
    Rbar = float(np.mean(s.R ** 3)) ** (1 / 3)
    dt = 0.2 * cgdem.cgdem_rayleigh_dt(Rbar, m["rho"], m["E"], m["nu"])
    skin_frac = KNOBS["skin"] if KNOBS["skin"] is not None else (0.06 if closure else 0.02)
    skin = skin_frac * 2 * float(s.R.max())
    p = cgdem.sample_params(s, dt, skin, k=k, scheme=cgdem.CG_SSW if k > 1 else cgdem.CG_NONE)
    ctx = cgdem.Context([p], [len(s.R)], precision=precision, max_neighbors=64 if closure else 48,
                        closure=closure, steps_per_graph=steps_per_graph, cell_scale=KNOBS["cell"],
                        block_size=128 if closure else KNOBS["block"], particles_per_warp=KNOBS["ppw"])
    ctx.set_fluid_velocity(s.Us)
    ctx.init_particles(s.x, s.v, s.w, s.R, bond_touching=True)
    ctx.compute_forces()
    return ctx


def main(argv):
    import torch

    from . import build as B
    from . import cgdem
    B.build()
    argv = list(argv)
    for flag, key, conv in (("--cell", "cell", float), ("--skin", "skin", float),
                            ("--block", "block", int), ("--ppw", "ppw", int), ("--workload", "workload", str)):
        if flag in argv:
            i = argv.index(flag)
            KNOBS[key] = conv(argv[i + 1])
            del argv[i:i + 2]
    what = argv[0] if argv else "step"
    if what == "step":
        prec = cgdem.FP64 if len(argv) > 1 and argv[1] == "fp64" else cgdem.MIXED
        steps = int(argv[2]) if len(argv) > 2 else 12
        ctx = _cylinder_ctx(prec)
        if "eager" in argv[3:]:
            print("force ms", ctx.profile_step(max(steps, 2))["force_ms"])
        else:
            ctx.step(steps)
        torch.cuda.synchronize()
        print("counters", ctx.counters())
        ctx.status()
    elif what == "rebuild":
        prec = cgdem.FP64 if len(argv) > 1 and argv[1] == "fp64" else cgdem.MIXED
        count = int(argv[2]) if len(argv) > 2 else 4
        ctx = _cylinder_ctx(prec, steps_per_graph=1)
        for _ in range(count):
            ctx.build_contacts()
            ctx.step(1)
        torch.cuda.synchronize()
        print("counters", ctx.counters())
        ctx.status()
    elif what == "closure":
        steps = int(argv[1]) if len(argv) > 1 else 12
        ctx = _cylinder_ctx(cgdem.MIXED, closure=True, k=2)
        rng = np.random.default_rng(0)
        theta = np.zeros(cgdem.MLP_NPARAMS, np.float32)
        theta[5:10] = 1.0
        theta[10:] = rng.normal(0, 0.1, cgdem.MLP_NPARAMS - 10)
        ctx.set_closure(theta, [-1e9] * 5, [1e9] * 5, 3.0, 0.5)
        # launched from the host, as "step ... eager"
        print("force ms", ctx.profile_step(max(steps, 2))["force_ms"])
        torch.cuda.synchronize()
        print("counters", ctx.counters())
        ctx.status()
    elif what == "mlp":
        n = int(argv[1]) if len(argv) > 1 else 65536
        iters = int(argv[2]) if len(argv) > 2 else 3
        rng = np.random.default_rng(0)
        theta = np.zeros(cgdem.MLP_NPARAMS, np.float32)
        theta[5:10] = 1.0
        theta[10:] = rng.normal(0, 0.1, cgdem.MLP_NPARAMS - 10)
        net = cgdem.Closure(theta)
        X = rng.normal(size=(n, 5)).astype(np.float32)
        Y = rng.normal(size=(n, 2)).astype(np.float32)
        hist = net.train(X, Y, np.ones_like(Y), iters, 1e-3)
        print("loss", hist.tolist())
    else:
        raise SystemExit(__doc__)
    print("ok")


if __name__ == "__main__":
    main(sys.argv[1:])
