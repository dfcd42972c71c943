"""Time-refinement study of SDC and MLSDC-SH on the GPU, in the manner of the
paper's Sec. 5 experiments: errors of several schemes against a reference run
at a fixed spatial resolution, the observed order of convergence between
successive step sizes, and the measured cost of each run.

    python -m paper_1805_07923_gb300.study --case dome --R 85 --nlon 256 --nlat 128 \\
        --Rc 42 --Ic 128 --Jc 64 --hours 24 --dts 1200,900,600,450,300 --ref-dt 60

Schemes, in the paper's notation: SDC(M+1, K) is the single-level scheme with
M+1 Gauss-Lobatto nodes and K sweeps per step; MLSDC(M_f+1, M_c+1, N, 1/2) is
the two-level scheme with the coarse truncation R_c (half of R by default),
N iterations of one fine and one coarse sweep (the paper's choice of one
coarse sweep per iteration); MLSDC(5,3,2,N) adds a third level at R_3 (a
quarter of R by default) with 2 nodes (the V-cycle of mlsdc_levels_step).  Cases: `dome` (the Gaussian dome of Eq.
gaussian_bump, at rest, with the mean geopotential g h_bar = g 29400 m) and
`spectra` (the seeded n^-3/2 state of the benchmarks).  Errors are L_inf
norms over the Gaussian grid of Phi' and of zeta (the difference
synthesised with sh_inverse), relative to the L_inf norm of the reference
field.  Everything runs in float64, each step one CUDA-graph replay; the cost
of a run is its device time (CUDA events) and its F_E evaluation count.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import inputs
from . import mlsdc as M

SCHEMES = {
    # name: (nodes per level, finest first; sweeps (one level) or iterations)
    "SDC(3,4)": ((3,), 4),
    "MLSDC(3,2,2,1/2)": ((3, 2), 2),
    "SDC(5,8)": ((5,), 8),
    "MLSDC(5,3,4,1/2)": ((5, 3), 4),
}
EXTRA_SCHEMES = {  # run on request (--schemes)
    "MLSDC(5,3,7,1/2)": ((5, 3), 7),
    "MLSDC(5,3,2,4)": ((5, 3, 2), 4),
}
ALL_SCHEMES = {**SCHEMES, **EXTRA_SCHEMES}


def fe_evals_per_step(scheme: str) -> list[int]:
    """F_E evaluations per step on each level: the spread evaluates node 0
    once per level; a sweep evaluates every node after the first; an MLSDC
    iteration adds, on each coarser level, the restricted nodes and one
    sweep, and on an intermediate level one more sweep going up."""
    nodes, k = ALL_SCHEMES[scheme]
    if len(nodes) == 1:
        return [1 + k * (nodes[0] - 1)]
    out = [1 + k * (nodes[0] - 1)]
    for l in range(1, len(nodes)):
        sweeps = 1 + (1 if l < len(nodes) - 1 else 0)
        out.append(1 + k * (nodes[l] - 1) * (1 + sweeps))
    return out


class Study:
    def __init__(self, case: str, R: int, I: int, J: int, Rc: int, Ic: int, Jc: int, omega: float | None = None,
                 third: tuple[int, int, int] | None = None):
        self.case, self.R, self.Rc = case, R, Rc
        g = 9.80616
        if case == "dome":
            self.prm = M.swe_params(phibar=g * inputs.DOME_H_BAR)
        else:
            self.prm = M.swe_params()
        if omega is not None:
            self.prm.omega = omega
        self.pf = M.Plan(R, I, J, "fp64")
        self.pc = M.Plan(Rc, Ic, Jc, "fp64", 2)
        R3, I3, J3 = third if third else (Rc // 2, Ic // 2, Jc // 2)
        self.p3 = M.Plan(R3, I3, J3, "fp64")
        self.x0 = self._initial_state()
        self.buf = torch.empty_like(self.x0)  # one state buffer, so each step size captures one graph
        self._levels = {}
        self._captured = set()

    def _initial_state(self) -> torch.Tensor:
        R, p = self.R, self.pf
        if self.case == "spectra":
            return torch.from_numpy(inputs.initial_state(R)).cuda()
        mu, _ = p.grid()
        lam = 2.0 * np.pi * np.arange(p.I) / p.I
        phi, _ = inputs.gaussian_dome_grid(lam, mu)
        spec = torch.empty((1, p.nc), dtype=torch.complex128, device="cuda")
        M.sh_forward(p, torch.from_numpy(np.ascontiguousarray(phi)).cuda(), spec, 1)
        x = torch.zeros((3, p.nc), dtype=torch.complex128, device="cuda")
        x[0] = spec[0]
        return x

    def _runner(self, scheme: str):
        if scheme not in self._levels:
            nodes, k = ALL_SCHEMES[scheme]
            levels = [M.Level(p, n, self.prm) for p, n in zip((self.pf, self.pc, self.p3), nodes)]
            if len(levels) == 1:
                self._levels[scheme] = (levels[0],)
            elif len(levels) == 2:
                self._levels[scheme] = (levels, M.MLSDC(*levels))
            else:
                self._levels[scheme] = (levels, M.MLSDCLevels(levels))
        return self._levels[scheme]

    def _step(self, scheme, objs, x, dt, k):
        if len(objs) == 1:
            M.sdc_step(objs[0], x, dt, k)
        elif isinstance(objs[1], M.MLSDC):
            M.mlsdc_step(objs[1], x, dt, k, 1, use_graph=True)
        else:
            M.mlsdc_levels_step(objs[1], x, dt, k, 1, use_graph=True)

    def run(self, scheme: str, dt: float, seconds: float) -> tuple[torch.Tensor, float, int]:
        """The state after `seconds` of simulated time (a whole number of steps
        of size dt), the device milliseconds and the number of steps."""
        steps = int(round(seconds / dt))
        if abs(steps * dt - seconds) > 1e-9 * seconds:
            raise ValueError(f"{seconds} s is not a whole number of steps of {dt} s")
        nodes, k = ALL_SCHEMES[scheme]
        objs = self._runner(scheme)
        x = self.buf
        if len(nodes) > 1 and (scheme, dt) not in self._captured:
            x.copy_(self.x0)  # capture this step size's graph outside the timed region
            self._step(scheme, objs, x, dt, k)
            self._captured.add((scheme, dt))
        x.copy_(self.x0)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(steps):
            self._step(scheme, objs, x, dt, k)
        e1.record(st)
        e1.synchronize()
        return x.clone(), e0.elapsed_time(e1), steps

    def linf(self, x: torch.Tensor, field: int) -> float:
        g = torch.empty((1, self.pf.J, self.pf.I), dtype=torch.float64, device="cuda")
        M.sh_inverse(self.pf, x[field:field + 1].contiguous(), g, 1)
        return float(g.abs().max())


def observed_orders(dts, errs):
    out = [None]
    for i in range(1, len(dts)):
        a, b = errs[i - 1], errs[i]
        out.append(math.log(a / b) / math.log(dts[i - 1] / dts[i]) if a > 0 and b > 0 else None)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="dome", choices=["dome", "spectra"])
    ap.add_argument("--R", type=int, default=85)
    ap.add_argument("--nlon", type=int, default=256)
    ap.add_argument("--nlat", type=int, default=128)
    ap.add_argument("--Rc", type=int, default=42)
    ap.add_argument("--Ic", type=int, default=128)
    ap.add_argument("--Jc", type=int, default=64)
    ap.add_argument("--hours", type=float, default=24.0)
    ap.add_argument("--dts", default="1200,900,600,450,300")
    ap.add_argument("--ref-dt", type=float, default=60.0)
    ap.add_argument("--schemes", default=";".join(SCHEMES), help="scheme names separated by semicolons")
    a = ap.parse_args(argv)
    T = a.hours * 3600.0
    s = Study(a.case, a.R, a.nlon, a.nlat, a.Rc, a.Ic, a.Jc)
    ref, ref_ms, ref_steps = s.run("SDC(5,8)", a.ref_dt, T)
    norms = [s.linf(ref, 0), s.linf(ref, 1)]
    dts = [float(v) for v in a.dts.split(",")]
    rows = []
    for scheme in a.schemes.split(";"):
        errs_phi, errs_zeta = [], []
        for dt in dts:
            x, ms, steps = s.run(scheme, dt, T)
            d = x - ref
            errs_phi.append(s.linf(d, 0) / norms[0])
            errs_zeta.append(s.linf(d, 1) / norms[1])
            rows.append({"scheme": scheme, "dt": dt, "steps": steps, "err_phi": errs_phi[-1],
                         "err_zeta": errs_zeta[-1], "ms": ms,
                         "fe_per_level": [v * steps for v in fe_evals_per_step(scheme)]})
        for r, op, oz in zip(rows[-len(dts):], observed_orders(dts, errs_phi), observed_orders(dts, errs_zeta)):
            r["order_phi"], r["order_zeta"] = op, oz
    out = {"case": a.case, "R": a.R, "grid": [a.nlon, a.nlat], "Rc": a.Rc, "hours": a.hours,
           "reference": {"scheme": "SDC(5,8)", "dt": a.ref_dt, "steps": ref_steps, "ms": ref_ms},
           "phibar": s.prm.phibar, "rows": rows}
    print(json.dumps(out))
    print(f"| scheme | dt (s) | L_inf err Phi' | order | L_inf err zeta | order | F_E per level | GPU ms |")
    print("|---|---|---|---|---|---|---|---|")
    for r in rows:
        fo = lambda v: "" if v is None else f"{v:.2f}"
        print(f"| {r['scheme']} | {r['dt']:g} | {r['err_phi']:.2e} | {fo(r['order_phi'])} | {r['err_zeta']:.2e} | "
              f"{fo(r['order_zeta'])} | {' / '.join(str(v) for v in r['fe_per_level'])} | {r['ms']:.1f} |")


if __name__ == "__main__":
    main()
