"""GPU parity of the Neo-Hookean beam (Sec. 3, "Hyperelasticity") against the
oracle through the C ABI: the residual entry by entry, the FD action, the
transfers between the beam grids, and whole solves with the paper's solver
(outer CG, V(5,5), coarse CG with L-BFGS and the spectral shift, which this
non-convex problem activates)."""
import numpy as np
import pytest

from gpu_common import dev, host, jf, rel, torch
from golden import make_beam_cg_envelope
from oracle import hyper, jfnk

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -52


def _state(m, seed, amp=0.2):
    """Dirichlet data plus a random displacement of amp * h (every element keeps
    J > 0, so the residual is finite)."""
    u = hyper.boundary_state(m)
    rng = np.random.default_rng(seed)
    mask = hyper.unknown_mask(u.shape)
    u[mask] += amp / m * rng.uniform(-1.0, 1.0, size=int(mask.sum()))
    return u


@pytest.mark.parametrize("m", [1, 3, 16])
def test_residual_parity(m):
    p = jf().Problem("beam3d", m, 1)
    u = _state(m, seed=m)
    F_ora = hyper.residual(u)
    assert np.all(np.isfinite(F_ora))
    F64 = host(p.residual(dev(u)))
    assert rel(F64, F_ora) <= 1e-12
    assert np.all(F64[hyper.dirichlet_mask(u.shape)] == 0.0)
    F32 = host(p.residual(dev(u, torch.float32)))
    assert rel(F32, F_ora) <= 1e-5


def test_jvp_parity():
    m = 4
    p = jf().Problem("beam3d", m, 1)
    u = _state(m, seed=5)
    v = np.random.default_rng(6).normal(size=u.shape)
    ud = dev(u)
    Jv = host(p.jvp(ud, p.residual(ud), dev(v)))
    lv = jfnk.HyperLevel(m)
    Jo = jfnk.fd_jv(lv, u, lv.F(u), v)
    # FD round-off bound c eps_p |F terms| / eps (c = 64), the terms of size mu |F| h^2
    eps = jfnk.fd_eps(u, np.where(lv.mask, v, 0.0), lv.mask)
    terms = hyper.MU * np.sqrt(lv.n_unknowns) * (1.0 / m) ** 2 * 4.0
    bound = 64 * EPS64 * terms / eps / np.linalg.norm(Jo)
    assert rel(Jv, Jo) <= max(bound, 1e-10), (rel(Jv, Jo), bound)


@pytest.mark.parametrize("mc", [1, 4])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_transfers_parity(mc, dt):
    tdt = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-14 if dt == "f64" else 1e-6
    p = jf().Problem("beam3d", 2 * mc, 2)
    rng = np.random.default_rng(7)
    f = rng.normal(size=hyper.shape_of(2 * mc))
    c = rng.normal(size=hyper.shape_of(mc))
    assert rel(host(p.transfer("restrict", dev(f, tdt), level=1)), hyper.restrict(f)) <= tol
    assert rel(host(p.transfer("project", dev(f, tdt), level=1)), hyper.project(f)) <= tol
    s0 = rng.normal(size=f.shape)
    s0[hyper.dirichlet_mask(s0.shape)] = 0.0
    out = dev(s0, tdt)
    p.transfer("prolong_add", dev(c, tdt), level=1, out=out)
    assert rel(host(out), s0 + hyper.prolong(c)) <= tol


@pytest.mark.parametrize("k", [1, 2])
def test_paper_solver_matches_oracle(k):
    """Refinement levels L1 (20 x 2 x 2 elements, 2 levels) and L2 (40 x 4 x 4, 3
    levels): the GPU and the oracle run the same algorithm to ||F|| < 1e-10 and
    reach the same discrete solution; the spectral shift is used on the GPU; the
    Newton counts of the paper's stopping rule agree to within one step."""
    m = 2 ** k
    u0 = hyper.boundary_state(m)
    p = jf().Problem("beam3d", m, k + 1, options=jf().paper_options(atol_newton=1e-10))
    u = dev(u0)
    st = p.solve(u)
    assert st["converged"]
    assert st["coarse_shifts"] > 0
    lvs = jfnk.build_hyper_hierarchy(k)
    uo, so = jfnk.newton_solve(lvs, u0, jfnk.paper_options(atol_newton=1e-10))
    assert so.converged
    # both stop at ||F|| < 1e-10, where the solution is within ~2e-10 of the
    # converged one (the oracle's own L1 solve at 1e-10 against 1e-13)
    assert rel(host(u), uo) <= 1e-8
    b = hyper.dirichlet_mask(u0.shape)
    assert np.array_equal(host(u)[b], u0[b])
    q = jf().Problem("beam3d", m, k + 1, options=jf().paper_options())
    u6 = dev(u0)
    st6 = q.solve(u6)
    _, so6 = jfnk.newton_solve(jfnk.build_hyper_hierarchy(k), u0, jfnk.paper_options())
    assert st6["converged"] and abs(st6["newton_its"] - so6.newton_its) <= 1


def test_fgmres_solve_with_fp32_preconditioner():
    """The default solver (FGMRES, GMRES coarse solve) with an FP32
    preconditioner also reaches the oracle's discrete solution."""
    k, m = 2, 4
    u0 = hyper.boundary_state(m)
    o = jf().default_options(rtol_newton=1e-10, pc_dtype=jf().F32, eps_mode_pc=jf().EPS_FP32)
    p = jf().Problem("beam3d", m, k + 1, options=o)
    u = dev(u0)
    st = p.solve(u)
    assert st["converged"]
    uo, so = jfnk.newton_solve(jfnk.build_hyper_hierarchy(k), u0, jfnk.paper_options(atol_newton=1e-10))
    assert rel(host(u), uo) <= 1e-8


@pytest.mark.parametrize("amp", [0.1, 0.4])
def test_vcycle_parity_with_cgqn_coarse_solve(amp):
    """One V-cycle of Alg. 1 on the beam (3 levels, the paper's settings: V(5,5),
    coarse CG-QN with the spectral shift) at a seeded state, with the GPU's
    lambda_l given to the oracle.  The first cycle collects the secant pairs, the
    second uses them; both agree with the oracle to the accuracy of the FD
    actions."""
    k, m = 2, 4
    u = _state(m, seed=8, amp=amp)
    o = jf().paper_options()
    p = jf().Problem("beam3d", m, k + 1, options=o)
    p.mg_setup(dev(u), 0)
    lvs = jfnk.build_hyper_hierarchy(k)
    oo = jfnk.paper_options()
    jfnk.setup_levels(lvs, u, oo, 0)
    for l in range(1, k + 1):
        lvs[l].lam_max = p.level_info(l)["lambda_max"]
        assert lvs[l].lam_max == pytest.approx(jfnk.power_method(lvs[l], lvs[l].x, lvs[l].Fx,
                                                                 lvs[l].power_v, 30, tol=1e-2)[0], rel=2e-2)
    rng = np.random.default_rng(9)
    for _ in range(2):
        b = np.where(hyper.unknown_mask(u.shape), rng.normal(size=u.shape), 0.0)
        s = host(p.mg_vcycle(dev(b)))
        so = jfnk.mg_vcycle(lvs, k, b, oo)
        assert rel(s, so) <= 1e-5, rel(s, so)


def test_vcycle_near_the_solution_is_finite_and_of_the_oracles_size():
    """At the oracle's iterate after four Newton steps of the paper's solver at
    L2 (a twisted state where the shifted coarse CG of Alg. 1 is active), the
    V-cycle is discontinuous in its input: the oracle's own output norm moves
    by up to two orders of magnitude under 1e-13 relative perturbations of b
    (test_oracle_hyper).  So GPU and oracle are compared by size only: the GPU
    output is finite, zero on the Dirichlet faces, and its norm lies within a
    factor 10 of the range the oracle spans over b and five such perturbations."""
    k, m = 2, 4
    lvs0 = jfnk.build_hyper_hierarchy(k)
    u, _ = jfnk.newton_solve(lvs0, hyper.boundary_state(m), jfnk.paper_options(max_newton=4))
    p = jf().Problem("beam3d", m, k + 1, options=jf().paper_options())
    p.mg_setup(dev(u), 0)
    lam = [p.level_info(l)["lambda_max"] for l in range(k + 1)]
    rng = np.random.default_rng(10)
    for _ in range(3):
        b = np.where(hyper.unknown_mask(u.shape), rng.normal(size=u.shape), 0.0)
        s = host(p.mg_vcycle(dev(b)))
        assert np.all(np.isfinite(s))
        assert np.all(s[hyper.dirichlet_mask(u.shape)] == 0.0)
        norms = []
        for j in range(6):
            lvs = jfnk.build_hyper_hierarchy(k)
            oo = jfnk.paper_options()
            jfnk.setup_levels(lvs, u, oo, 0)
            for l in range(1, k + 1):
                lvs[l].lam_max = lam[l]
            rhs = b if j == 0 else b * (1.0 + 1e-13 * np.random.default_rng(100 + j).normal(size=b.shape))
            norms.append(np.linalg.norm(jfnk.mg_vcycle(lvs, k, rhs, oo)))
        assert 0.1 * min(norms) <= np.linalg.norm(s) <= 10.0 * max(norms), (np.linalg.norm(s), norms)


@pytest.mark.parametrize("k", [1, 2])
def test_paper_solver_counts_within_the_oracles_envelope(k):
    """Bound on the beam's cost.  The shifted coarse CG of Alg. 1 makes the
    outer CG counts scatter with rounding: the oracle's own totals over 17
    starts that differ by 1e-13 range over 40-417 (L1) and 22-446 (L2)
    (tests/golden/beam_cg_envelope.txt).  From the same 17 starts the GPU must
    (i) converge with Newton counts inside the oracle's range +- 1, (ii) repeat
    the oracle's CG counts exactly on the leading Newton steps where every
    oracle run agrees, (iii) stay at or under max_linear in every step, and
    (iv) have a median total of at most 5x the oracle's median (a run of the
    same distribution fails this with probability below 1e-3, a systematic
    blow-up does not pass it)."""
    env = make_beam_cg_envelope.load()[k]
    runs = sorted(env)
    o = jf().paper_options()
    p = jf().Problem("beam3d", 2 ** k, k + 1, options=o)
    newton_o = [r[1] for r in runs]
    totals_o = sorted(r[2] for r in runs)
    hists_o = [r[3] for r in runs]
    lead = 0
    while all(len(h) > lead for h in hists_o) and len({h[lead] for h in hists_o}) == 1:
        lead += 1
    assert lead >= 3
    totals = []
    for run, _, _, _ in runs:
        u = dev(make_beam_cg_envelope.initial_state(k, run))
        st = p.solve(u)
        assert st["converged"], (run, st)
        assert min(newton_o) - 1 <= st["newton_its"] <= max(newton_o) + 1, (run, st["newton_its"])
        assert st["lin_hist"][:lead] == hists_o[0][:lead], (run, st["lin_hist"])
        assert max(st["lin_hist"]) <= o.max_linear
        totals.append(st["linear_its"])
    print(f"L{k} CG totals, GPU: {sorted(totals)}; oracle: {totals_o}")
    assert np.median(totals) <= 5 * np.median(totals_o), (sorted(totals), totals_o)
