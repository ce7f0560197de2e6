"""Small and degenerate grids for the bounds-checked build of the library.

run_all(rhd) steps every case through the library that `rhd` has loaded and
returns {name: (final state, status)}.  tests/test_gpu_bounds.py runs it
once in a child process on librhd_bounds.so (built with -DRHD_BOUNDS_CHECK,
whose stage kernels report an index outside its array as RHD_ERR_BOUNDS)
and once on librhd.so, and compares the two.

Usage in the child process: python bounds_cases.py <library> <output.npz>
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2404_08247_gb300 import inputs as I  # noqa: E402


def grid_cases():
    """(name, problem, state, steps, precision) of single grids: one cell,
    a few cells, tiles with ragged edges and a z-chunk tail of one plane,
    PPM at its smallest reflecting axis (3 cells), inflow faces, RK2-SSP
    with a temperature-dependent opacity, both precisions."""
    out = []

    def add(name, ndim, n, precision="fp64", steps=2, seed=0, **kw):
        prob = I.base_problem(ndim, n, [1.0 / v for v in n], c=30.0, chat=10.0, **kw)
        U = I.random_state(prob, 500 + seed, tau_range=(1e-2, 10.0), T_range=(1.0, 1.3))
        out.append((name, prob, U, steps, precision))

    add("1d_n1", 1, (1,))
    add("1d_n2_mixed", 1, (2,), "mixed", seed=1)
    add("1d_n3_ppm_reflect", 1, (3,), bc="reflect", reconstruction="ppm", cfl=0.3, seed=2)
    add("1d_n257_inflow", 1, (257,), seed=3, hll_mode="none",
        bc=[["inflow", "reflect"], ["periodic"] * 2, ["periodic"] * 2],
        bc_state={(0, 0): (2.0, 10.0, 0.0, 0.0)})
    add("2d_1x1", 2, (1, 1), seed=4)
    add("2d_33x1", 2, (33, 1), seed=5)
    add("2d_5x3_reflect_mixed", 2, (5, 3), "mixed", bc="reflect", seed=6)
    add("2d_17x9_ppm_inflow", 2, (17, 9), reconstruction="ppm", cfl=0.3, seed=7,
        hll_mode="none", bc=[["inflow", "reflect"], ["reflect", "reflect"], ["periodic"] * 2],
        bc_state={(0, 0): (2.0, 10.0, 3.0, 0.0)})
    add("3d_1x1x1", 3, (1, 1, 1), seed=8)
    add("3d_2x3x5_mixed", 3, (2, 3, 5), "mixed", seed=9)
    add("3d_33x9x17_reflect_tau", 3, (33, 9, 17), bc="reflect", seed=10)
    add("3d_7x5x11_ppm_mixed", 3, (7, 5, 11), "mixed", reconstruction="ppm", cfl=0.3,
        bc="reflect", seed=11)
    add("3d_4x4x3_rk2ssp_chiT", 3, (4, 4, 3), scheme="rk2ssp", hll_mode="none",
        kappa_T_exp=-3.0, kappa_T_ref=1.0, newton_max_iter=400, seed=12)
    return out


def run_all(rhd):
    res = {}
    for name, prob, U, steps, precision in grid_cases():
        with rhd.RHDContext(prob, precision) as ctx:
            ctx.set_state(U)
            info = ctx.step(steps, raise_on_error=False)
            res[name] = (ctx.get_state(), info["status"])
            if name == "3d_2x3x5_mixed":
                ctx.set_state(U)
                res["3d_2x3x5_rates"] = (ctx.transport(), rhd.RHD_OK)
    # the batched kernel on tiny problems of both dimensions
    probs = []
    for k, n in enumerate([(1,), (3,), (1, 1), (6, 2), (33, 17)]):
        p = I.base_problem(len(n), n, [1.0 / v for v in n], c=30.0, chat=10.0)
        probs.append((p, I.random_state(p, 600 + k, tau_range=(1e-2, 10.0),
                                        T_range=(1.0, 1.3))))
    with rhd.RHDBatch([p for p, _ in probs], "fp64") as b:
        for i, (_, U) in enumerate(probs):
            b.set_state(i, U)
        info = b.step(2, raise_on_error=False)
        for i in range(len(probs)):
            res["batch_%d" % i] = (b.get_state(i), info["status"])
    # z-slabs of 3 planes exchanging ghost planes (PPM: the full halo depth)
    prob = I.base_problem(3, (5, 4, 9), [0.2, 0.25, 1 / 9], c=30.0, chat=10.0,
                          reconstruction="ppm", cfl=0.3)
    U = I.random_state(prob, 700, tau_range=(1e-2, 10.0), T_range=(1.0, 1.3))
    cuts = [0, 3, 6, 9]
    import torch
    stream = torch.cuda.current_stream()  # slabs share one stream
    slabs = [rhd.RHDContext(q, stream=stream) for q in rhd.slab_problems(prob, cuts)]
    try:
        for c, z0, z1 in zip(slabs, cuts, cuts[1:]):
            c.set_state(np.ascontiguousarray(U[:, z0:z1]))
        info = rhd.step_slabs(slabs, 2, raise_on_error=False)
        res["slabs_ppm"] = (np.concatenate([c.get_state() for c in slabs], axis=1),
                            info["status"])
    finally:
        for c in slabs:
            c.close()
    return res


def main(lib, out):
    from paper_2404_08247_gb300 import rhd
    rhd.load(lib)
    res = run_all(rhd)
    np.savez(out, **{k: v[0] for k, v in res.items()},
             **{"status_" + k: np.array(v[1]) for k, v in res.items()})


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])
