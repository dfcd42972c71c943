"""Run the explicit right-hand side F_E (or its adjoint) of one truncation for
a batch of members, for profiling one stage kernel in a chosen configuration.

    python -m paper_1805_07923_gb300.profile_rhs --R 170 --nlon 512 --nlat 256 \\
        --precision bf16x3 --members 16 --reps 3

The plan is created (and, for the tensor-core precisions, autotuned) first;
the `reps` evaluations that follow run inside the NVTX range
"mlsdc_profile", so a profiler can select exactly them, e.g.
ncu --nvtx --nvtx-include "mlsdc_profile/" -k regex:k_tc_anal ...
Prints the mean stage times measured with CUDA events.

With --node, the node updates of one SDC level instead (update, implicit
solve, F_I; --coriolis-implicit for the coupled per-wavenumber solve): one
SDC step fills the level's arrays, then `reps` rounds of the node updates
run inside the NVTX range, and the mean time of each is printed.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import inputs
from . import mlsdc as M


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--R", type=int, default=170)
    ap.add_argument("--nlon", type=int, default=512)
    ap.add_argument("--nlat", type=int, default=256)
    ap.add_argument("--precision", default="bf16x3", choices=list(M.PRECISIONS))
    ap.add_argument("--members", type=int, default=1)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--adjoint", action="store_true", help="the float64 F_E adjoint instead of F_E")
    ap.add_argument("--tc-config", default=None,
                    help="members_per_cta,stages,warp_specialised: replace the analysis's autotuned tensor-core "
                         "configuration (the synthesis keeps its own)")
    ap.add_argument("--kernels", default="auto", choices=["auto", "tc", "simt"],
                    help="tensor-core plans: the plan's choice, or both Legendre stages on tcgen05 / CUDA cores")
    ap.add_argument("--node", action="store_true", help="the node updates of an SDC level instead of F_E")
    ap.add_argument("--nodes", type=int, default=5, help="--node: Lobatto nodes of the level")
    ap.add_argument("--coriolis-implicit", action="store_true", help="--node: the implicit-Coriolis splitting")
    ap.add_argument("--dt", type=float, default=150.0)
    a = ap.parse_args(argv)
    if a.node:
        return node_main(a)
    plan = M.Plan(a.R, a.nlon, a.nlat, "fp64" if a.adjoint else a.precision, a.members)
    if a.kernels != "auto" and a.precision in ("tf32", "bf16x3") and not a.adjoint:
        plan.set_stage_kernels(a.kernels, a.kernels)
    if a.tc_config and a.precision in ("tf32", "bf16x3") and not a.adjoint:
        plan.set_tc_config(*[int(v) for v in a.tc_config.split(",")])
    prm = M.swe_params()
    base = inputs.initial_state(a.R)
    x = torch.from_numpy(np.stack([inputs.perturbed_member(base, a.R, a.R, k) for k in range(a.members)])).cuda()
    fe = torch.empty_like(x)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("mlsdc_profile")
    for _ in range(a.reps):
        if a.adjoint:
            for b in range(a.members):
                lam = x[b].clone()
                M.swe_explicit_rhs_adjoint(plan, prm, x[b], lam, fe[b])
        else:
            M.swe_explicit_rhs_batched(plan, prm, x, fe, a.members)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if a.adjoint:
        ms = M.mlsdc_profile_rhs_adjoint(plan, prm, x[0], x[0].clone(), fe[0], reps=20)
    else:
        ms = M.mlsdc_profile_rhs(plan, prm, x, fe, reps=20, members=a.members)
    print(json.dumps({"R": a.R, "nlon": a.nlon, "nlat": a.nlat, "precision": a.precision, "members": a.members,
                      "adjoint": a.adjoint, "stage_ms": ms, "stage_kernels_tc": plan.stage_kernels(a.members),
                      "tc_config": {"synthesis": plan.tc_config("synthesis"),
                                    "analysis": plan.tc_config("analysis")}}))


def node_main(a):
    plan = M.Plan(a.R, a.nlon, a.nlat, "fp64", a.members)
    lev = M.Level(plan, a.nodes, members=a.members, coriolis_implicit=a.coriolis_implicit)
    base = inputs.initial_state(a.R)
    x = torch.from_numpy(np.stack([inputs.perturbed_member(base, a.R, a.R, k) for k in range(a.members)])).cuda()
    if a.members == 1:
        x = x[0].contiguous()
    M.sdc_step(lev, x, a.dt, 1)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("mlsdc_profile")
    ms = M.mlsdc_profile_node(lev, a.dt, reps=a.reps)
    torch.cuda.nvtx.range_pop()
    ms20 = M.mlsdc_profile_node(lev, a.dt, reps=20)
    print(json.dumps({"R": a.R, "nodes": a.nodes, "members": a.members, "coriolis_implicit": a.coriolis_implicit,
                      "node_ms": ms20}))


if __name__ == "__main__":
    main()
