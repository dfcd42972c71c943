"""Parity of the float64 CUDA path (through the C ABI) with the float64 oracle.

Bar: relative L2 (Parseval norm) <= 1e-12 per field for spectral results and
per step for SDC/MLSDC steps; grid results max-abs relative <= 1e-12.  Sizes
span several 32-wide work items and ragged tails (J/2 = 35, R = 45), the
smallest legal plan (R = 1 on 16 x 4) and the full T170/T85 sizes of the
headline workload.

Each spectral comparison is also made band by band (degrees n <= R/3,
R/3 < n <= 2R/3, n > 2R/3, each band's error relative to that band's own
norm), so an error confined to the weak high-degree coefficients of the
n^-3/2 spectra cannot hide under the field's norm: bound 1e-11 per band
(the field bound times the ~14x that uniform rounding gains when measured
against the high band's norm, with margin)."""
import numpy as np
import pytest
import torch

from oracle import sdc as osdc
from oracle import sht as osht
from oracle.swe import SWE, Params
from paper_1805_07923_gb300 import inputs
from paper_1805_07923_gb300 import mlsdc as M

pytestmark = pytest.mark.gpu

TOL = 1e-12
SIZES = [(1, 16, 4), (21, 64, 32), (45, 256, 70), (42, 128, 64), (85, 256, 128), (170, 512, 256)]

_oracles = {}


def oracle(R, I, J):
    key = (R, I, J)
    if key not in _oracles:
        _oracles[key] = SWE(R, I, J, Params())
    return _oracles[key]


def rel_l2(R, got, ref):
    return np.sqrt(osht.norm2(R, got - ref) / max(osht.norm2(R, ref), 1e-300))


BAND_TOL = 1e-11


def band_rel_l2(R, got, ref):
    """Relative L2 error in each third of the degrees, against the band's own norm."""
    m, n = osht.spec_mn(R)
    wt = np.where(m == 0, 1.0, 2.0)
    out = []
    for lo, hi in ((-1, R // 3), (R // 3, 2 * R // 3), (2 * R // 3, R)):
        sel = (n > lo) & (n <= hi)
        den = np.sum(wt[sel] * np.abs(ref[sel]) ** 2)
        if den > 0:
            out.append(float(np.sqrt(np.sum(wt[sel] * np.abs(got[sel] - ref[sel]) ** 2) / den)))
    return out


def check_bands(R, got, ref, tol=BAND_TOL, what=""):
    b = band_rel_l2(R, got, ref)
    assert max(b) <= tol, (what, b)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("R,I,J", SIZES)
def test_sh_inverse_matches_oracle(R, I, J):
    o = oracle(R, I, J)
    spec = np.stack([inputs.spectrum(R, 40 + k, k, 1.0, slope=-0.5) for k in range(3)])
    plan = M.Plan(R, I, J)
    g = torch.empty((3, J, I), dtype=torch.float64, device="cuda")
    M.sh_inverse(plan, dev(spec), g, 3)
    got = host(g)
    for k in range(3):
        ref = o.grid.synthesis(spec[k])
        assert np.max(np.abs(got[k] - ref)) <= TOL * np.max(np.abs(ref))


@pytest.mark.parametrize("R,I,J", SIZES)
def test_sh_forward_matches_oracle(R, I, J):
    o = oracle(R, I, J)
    rng = np.random.default_rng(R)
    grid = rng.standard_normal((2, J, I))          # not band-limited: aliasing included
    plan = M.Plan(R, I, J)
    s = torch.empty((2, o.nc), dtype=torch.complex128, device="cuda")
    M.sh_forward(plan, dev(grid), s, 2)
    got = host(s)
    for k in range(2):
        ref = o.grid.analysis(grid[k])
        assert rel_l2(R, got[k], ref) <= TOL
        check_bands(R, got[k], ref, what=("sh_forward", k))
        assert np.all(got[k][: R + 1].imag == 0)


@pytest.mark.parametrize("R,I,J", SIZES[1:4])
def test_round_trip_on_gpu(R, I, J):
    spec = inputs.spectrum(R, 9, 0, 1.0, slope=0.0)[None]
    plan = M.Plan(R, I, J)
    g = torch.empty((1, J, I), dtype=torch.float64, device="cuda")
    s = torch.empty((1, plan.nc), dtype=torch.complex128, device="cuda")
    M.sh_inverse(plan, dev(spec), g, 1)
    M.sh_forward(plan, g, s, 1)
    assert rel_l2(R, host(s)[0], spec[0]) <= TOL


def fp64_spread(o, x):
    """Relative difference, per field, between two correct float64 evaluations of
    F_E that differ only in rounding order (the oracle's matmul DFT versus a
    numpy FFT for the longitude transforms).  The divergence tendency is a
    near-cancellation of curl((zeta+f)V) and lap(V.V/2), so at T170 two
    correct evaluations already differ by ~5e-12."""
    g = o.grid
    R, I = g.R, g.I
    fa, fs = g.fourier_analysis, g.fourier_synthesis

    def fft_a(f):
        return np.fft.rfft(f, axis=-1)[..., : R + 1] / I

    def fft_s(F):
        full = np.zeros(F.shape[:-1] + (I // 2 + 1,), complex)
        full[..., : R + 1] = F
        full[..., 0] = full[..., 0].real
        return np.fft.irfft(full, n=I, axis=-1) * I

    ref = o.explicit_rhs(x)
    g.fourier_analysis, g.fourier_synthesis = fft_a, fft_s
    try:
        alt = o.explicit_rhs(x)
    finally:
        g.fourier_analysis, g.fourier_synthesis = fa, fs
    return ref, [rel_l2(R, alt[k], ref[k]) for k in range(3)], [band_rel_l2(R, alt[k], ref[k]) for k in range(3)]


@pytest.mark.parametrize("R,I,J", SIZES)
def test_explicit_rhs_matches_oracle(R, I, J):
    """Per field: relative L2 <= max(1e-12, 4 x the float64 rounding-order
    spread of the oracle itself); per degree band likewise, against the
    oracle's spread in that band (the divergence tendency's high band is
    where its cancellation is strongest)."""
    o = oracle(R, I, J)
    x = inputs.initial_state(R, seed=1805)
    plan = M.Plan(R, I, J)
    FE = torch.empty((3, o.nc), dtype=torch.complex128, device="cuda")
    M.swe_explicit_rhs(plan, M.swe_params(), dev(x), FE)
    got = host(FE)
    ref, spread, bspread = fp64_spread(o, x)
    for k in range(3):
        tol = max(TOL, 4.0 * spread[k])
        assert rel_l2(R, got[k], ref[k]) <= tol, (k, rel_l2(R, got[k], ref[k]), tol)
        gb = band_rel_l2(R, got[k], ref[k])
        for i, (e, s) in enumerate(zip(gb, bspread[k])):
            assert e <= max(BAND_TOL, 4.0 * s), ("F_E band", k, i, e, s)


@pytest.mark.parametrize("R,I,J", [(21, 64, 32), (85, 256, 128)])
def test_implicit_rhs_and_solve_match_oracle(R, I, J):
    o = oracle(R, I, J)
    x = inputs.initial_state(R, seed=3)
    plan = M.Plan(R, I, J)
    prm = M.swe_params()
    FI = torch.empty_like(dev(x))
    M.swe_implicit_rhs(plan, prm, dev(x), FI)
    ref = o.implicit_rhs(x)
    got = host(FI)
    for k in range(3):
        assert rel_l2(R, got[k], ref[k]) <= TOL
    for alpha in (0.0, 75.0, 1.0e4):
        xs = dev(x)
        M.swe_implicit_solve(plan, prm, alpha, xs, xs)      # in place
        ref = o.implicit_solve(x, alpha)
        got = host(xs)
        for k in range(3):
            assert rel_l2(R, got[k], ref[k]) <= TOL


@pytest.mark.parametrize("R,I,J,n_nodes,with_tau", [(21, 64, 32, 5, False), (42, 128, 64, 3, True)])
def test_sdc_sweep_matches_oracle(R, I, J, n_nodes, with_tau):
    o = oracle(R, I, J)
    lev_o = osdc.Level(o, n_nodes)
    base = inputs.initial_state(R, seed=11)
    Theta = [base + 0.01 * inputs.initial_state(R, seed=100 + m) for m in range(n_nodes)]
    FI = [o.implicit_rhs(t) for t in Theta]
    FE = [o.explicit_rhs(t) * (1.0 + 0.1 * m) for m, t in enumerate(Theta)]
    tau = [0.001 * inputs.initial_state(R, seed=200 + m) for m in range(n_nodes)] if with_tau else None
    tau_o = None
    if with_tau:
        tau[0] = np.zeros_like(tau[0])
        tau_o = tau
    dt = 450.0
    Tn, FIn, FEn = osdc.sweep(lev_o, dt, Theta, FI, FE, tau_o)
    plan = M.Plan(R, I, J)
    lev = M.Level(plan, n_nodes)
    Th_d, FI_d, FE_d = dev(np.stack(Theta)), dev(np.stack(FI)), dev(np.stack(FE))
    FIn_d, FEn_d = torch.zeros_like(FI_d), torch.zeros_like(FE_d)
    M.sdc_sweep(lev, dt, Th_d, FI_d, FE_d, FIn_d, FEn_d, dev(np.stack(tau)) if with_tau else None)
    gT, gI, gE = host(Th_d), host(FIn_d), host(FEn_d)
    for m in range(n_nodes):
        for k in range(3):
            assert rel_l2(R, gT[m][k], Tn[m][k]) <= TOL
            assert rel_l2(R, gI[m][k], FIn[m][k]) <= TOL
            assert rel_l2(R, gE[m][k], FEn[m][k]) <= TOL


def test_level_matrices_match_oracle():
    plan = M.Plan(21, 64, 32)
    for n in (2, 3, 5, 7):
        lev = M.Level(plan, n)
        t, Q, QE, QI = lev.matrices()
        lo = osdc.Level(None, n)
        assert np.max(np.abs(t - lo.t)) < 1e-15
        assert np.max(np.abs(Q - lo.Q)) < 1e-15
        assert np.max(np.abs(QE - lo.QE)) < 1e-15
        assert np.max(np.abs(QI - lo.QI)) < 1e-14


def test_sdc_step_config1():
    """Single-level SDC(3,4), T21 on 64 x 32, dt 600 s: every step and 20 steps."""
    R = 21
    o = oracle(R, 64, 32)
    lev_o = osdc.Level(o, 3)
    plan = M.Plan(R, 64, 32)
    lev = M.Level(plan, 3)
    u = inputs.initial_state(R)
    x = dev(u)
    for step in range(20):
        u_prev = host(x)
        M.sdc_step(lev, x, 600.0, 4)
        ref = osdc.sdc_step(lev_o, u_prev, 600.0, 4)
        got = host(x)
        for k in range(3):
            assert rel_l2(R, got[k], ref[k]) <= TOL, (step, k)
        u = osdc.sdc_step(lev_o, u, 600.0, 4)
    for k in range(3):
        assert rel_l2(R, host(x)[k], u[k]) <= 1e-11


def _mlsdc(Rf, If, Jf, Rc, Ic, Jc):
    pf, pc = M.Plan(Rf, If, Jf), M.Plan(Rc, Ic, Jc)
    lf, lc = M.Level(pf, 5), M.Level(pc, 3)
    return M.MLSDC(lf, lc), (pf, pc, lf, lc)


def test_mlsdc_step_config2():
    """MLSDC T85/T42 (256x128 / 128x64), 5/3 nodes, 4 iterations, 1 fine + 2
    coarse sweeps, dt 300 s: three steps, each against the oracle."""
    Rf, Rc = 85, 42
    of, oc = osdc.Level(oracle(Rf, 256, 128), 5), osdc.Level(oracle(Rc, 128, 64), 3)
    ml, keep = _mlsdc(Rf, 256, 128, Rc, 128, 64)
    x = dev(inputs.initial_state(Rf))
    for step in range(3):
        u_prev = host(x)
        M.mlsdc_step(ml, x, 300.0, 4, 2)
        ref = osdc.mlsdc_step(of, oc, u_prev, 300.0, 4, 2)
        got = host(x)
        for k in range(3):
            assert rel_l2(Rf, got[k], ref[k]) <= TOL, (step, k, rel_l2(Rf, got[k], ref[k]))
            check_bands(Rf, got[k], ref[k], what=(step, k))
    assert ml.launch_count() > 0


def test_mlsdc_step_headline_size():
    """One MLSDC step at the headline sizes: T170/T85 (512x256 / 256x128), dt 150 s."""
    Rf, Rc = 170, 85
    of, oc = osdc.Level(oracle(Rf, 512, 256), 5), osdc.Level(oracle(Rc, 256, 128), 3)
    ml, keep = _mlsdc(Rf, 512, 256, Rc, 256, 128)
    u = inputs.initial_state(Rf)
    x = dev(u)
    M.mlsdc_step(ml, x, 150.0, 4, 2, use_graph=True)
    ref = osdc.mlsdc_step(of, oc, u, 150.0, 4, 2)
    got = host(x)
    for k in range(3):
        assert rel_l2(Rf, got[k], ref[k]) <= TOL, (k, rel_l2(Rf, got[k], ref[k]))
        check_bands(Rf, got[k], ref[k], what=k)
        print(f"T170/T85 step field {k}: rel L2 {rel_l2(Rf, got[k], ref[k]):.2e}, "
              f"bands {band_rel_l2(Rf, got[k], ref[k])}")


def test_graph_replay_equals_direct_launches():
    ml, keep = _mlsdc(42, 128, 64, 21, 64, 32)
    u = inputs.initial_state(42)
    a, b = dev(u), dev(u)
    for _ in range(3):
        M.mlsdc_step(ml, a, 300.0, 4, 2, use_graph=False)
    for _ in range(3):
        M.mlsdc_step(ml, b, 300.0, 4, 2, use_graph=True)
    assert np.array_equal(host(a), host(b))


def test_mean_geopotential_conserved_on_gpu():
    ml, keep = _mlsdc(42, 128, 64, 21, 64, 32)
    u = inputs.initial_state(42)
    u[0, 0] = 77.0
    x = dev(u)
    for _ in range(10):
        M.mlsdc_step(ml, x, 300.0, 4, 2, use_graph=True)
    got = host(x)
    assert abs(got[0, 0] - 77.0) <= 1e-13 * 77.0
    assert abs(got[2, 0]) <= 1e-25
    assert M.mlsdc_check_finite(x)
    bad = x.clone()
    bad[1, 5] = float("nan")
    assert not M.mlsdc_check_finite(bad)


def test_bad_arguments_are_reported():
    plan = M.Plan(21, 64, 32)
    x = torch.zeros((3, plan.nc), dtype=torch.complex128, device="cuda")
    with pytest.raises(M.MlsdcError):
        M.swe_explicit_rhs(plan, M.swe_params(), x, x)       # aliasing
    with pytest.raises(M.MlsdcError):
        M.swe_implicit_solve(plan, M.swe_params(), -1.0, x, x)
    with pytest.raises(M.MlsdcError):
        M.Level(plan, 12)
    with pytest.raises(M.MlsdcError):
        M.sh_inverse(plan, x, torch.zeros(10, dtype=torch.float64, device="cuda"), 1)
